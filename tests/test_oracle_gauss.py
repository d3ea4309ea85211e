"""Pins for the Gaussian-coupling oracle (the model of the paper's Sec. 4).

fexp against mpmath; the Metropolis acceptance fraction against exp(-beta
dE); exact enumeration of 2x2x2 and 2x2x3 boxes; the Boltzmann distribution
after fixed-temperature sweeps; and the paper's own 1D comparison: the
periodic Gaussian chain against exact transfer matrices."""
import math

import numpy as np
import pytest

import brute
from oracle import oracle as o
from paper_1006_0252_gb300 import inputs

S = o.GAUSS_SCALE


def test_fexp_within_two_float_ulp():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 80
    rng = np.random.default_rng(4)
    xs = [0.0, -0.0, -1e-30, -0.5, -math.log(2), -1.0, -20.0, -87.0, -100.0, -103.9]
    xs += list(-rng.uniform(0, 1, 2000)) + list(-rng.uniform(0, 104, 4000))
    for x in xs:
        xf = float(np.float32(x))
        got = o.fexp(xf)
        want = float(mp.exp(mp.mpf(xf)))
        if want < 1.2e-38:  # subnormal results: absolute error of a few subnormal steps
            assert abs(got - want) <= 4 * 1.4e-45 + 4 * np.spacing(np.float32(want))
        else:
            assert abs(got - want) <= 2 * float(np.spacing(np.float32(want))), (xf, got, want)
    assert o.fexp(0.0) == 1.0 and o.fexp(-200.0) == 0.0


def test_acceptance_fraction_is_boltzmann_factor():
    mp = pytest.importorskip("mpmath")
    for beta, dE in ((0.3, int(0.7 * S)), (1.0, int(2.5 * S)), (2.0, 12345), (5.0, int(0.1 * S))):
        # count accepted top-24-bit values exactly: u24 < p * 2^24
        lo, hi = 0, 1 << 24
        while lo < hi:  # smallest u24 rejected
            mid = (lo + hi) // 2
            if o.gauss_accept(beta, dE, mid << 8):
                lo = mid + 1
            else:
                hi = mid
        p = lo / 2 ** 24
        x = float(np.float32(np.float32(beta) * np.float32(dE)) * np.float32(1 / S))
        want = float(mp.exp(-x))
        assert abs(p - want) <= 2 ** -24 + 4e-7 * want, (beta, dE, p, want)
    assert o.gauss_accept(0.0, 1000, 0xFFFFFFFF)  # beta = 0 accepts every rise


def _exact(J, Lx, Ly, Lz, mask):
    bonds = brute.bonds_3d(J, Lx, Ly, Lz, mask)
    return brute.energies(bonds, Lx * Ly * Lz).astype(np.float64) / S


def _runs(J, dims, mask, R, betas, theta, seeds):
    F = np.zeros((len(seeds), len(betas)))
    Em = np.zeros((len(seeds), len(betas)))
    for a, s in enumerate(seeds):
        r = o.GaussRun(J, 3 if len(dims) == 3 else 1, *dims, periodic_mask=mask, R0=R, seed=s)
        st = r.state()
        F[a, 0], Em[a, 0] = st.minus_beta_F, st.sumE / st.R / S
        for k in range(1, len(betas)):
            r.step(float(betas[k]), theta, R)
            st = r.state()
            F[a, k], Em[a, k] = st.minus_beta_F, st.sumE / st.R / S
        r.close()
    return F, Em


@pytest.mark.parametrize("shape", [(2, 2, 2, 7), (2, 2, 3, 3)])
def test_gaussian_pa_matches_exact_enumeration(shape):
    Lx, Ly, Lz, mask = shape
    J = inputs.gaussian_couplings_lattice(Lx, Ly, Lz, 3)
    Es = _exact(J, Lx, Ly, Lz, mask)
    betas = inputs.linear_schedule(2.0, 21)
    F, Em = _runs(J, (Lx, Ly, Lz), mask, 3000, betas, 4, range(1, 7))
    for k, b in enumerate(betas):
        lnZ, Eex, varE = brute.exact(Es, float(b))
        Ew, Fw = o.weighted_average(F[:, k], Em[:, k])
        assert abs(Fw - lnZ) < 0.03, (b, Fw, lnZ)
        err = max(Em[:, k].std(ddof=1) / math.sqrt(len(Em)), 0.02 * math.sqrt(varE) + 1e-3)
        assert abs(Ew - Eex) < 6 * err + 0.02, (b, Ew, Eex)


def test_gaussian_sweeps_sample_boltzmann_distribution():
    st = pytest.importorskip("scipy.stats")
    J = inputs.gaussian_couplings_lattice(2, 2, 2, 5)
    Es = _exact(J, 2, 2, 2, 7)
    beta = 0.6
    r = o.GaussRun(J, 3, 2, 2, 2, 7, R0=20000, seed=8)
    r.sweep_fixed(beta, 40)
    sp = r.spins()
    idx = ((sp < 0).astype(np.int64) << np.arange(8)).sum(axis=1)
    counts = np.bincount(idx, minlength=256)
    p = np.exp(-beta * Es - (-beta * Es).max())
    p /= p.sum()
    e = p * len(idx)
    keep = e >= 5
    chi2 = (((counts - e) ** 2 / e)[keep]).sum()
    assert st.chi2.sf(chi2, int(keep.sum()) - 1) > 1e-4
    assert np.array_equal(r.energies(), np.rint(Es[idx] * S).astype(np.int64))


def _chain_exact(J, beta):
    """ln Z of the periodic chain (E = sum J s s') by the 2x2 transfer matrix,
    and <E> by a central difference of ln Z."""
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120

    def lnZ(b):
        M = mp.eye(2)
        for j in J:
            a = mp.mpf(int(j)) / S
            M = M * mp.matrix([[mp.exp(-b * a), mp.exp(b * a)], [mp.exp(b * a), mp.exp(-b * a)]])
        return mp.log(M[0, 0] + M[1, 1])

    b = mp.mpf(beta)
    h = mp.mpf("1e-12")
    return float(lnZ(b)), float(-(lnZ(b + h) - lnZ(b - h)) / (2 * h))


def test_periodic_gaussian_chain_against_transfer_matrix():
    """The paper's 1D check (Sec. 4): population annealing against exact
    transfer matrices for a periodic chain with Gaussian couplings."""
    N = 40
    J = inputs.gaussian_couplings_chain(N, 2, 1)
    betas = inputs.linear_schedule(2.0, 26)
    F, Em = _runs(J, (N,), 0, 2000, betas, 5, range(1, 5))
    for k in (0, 5, 12, 25):
        lnZ, Eex = _chain_exact(J, float(betas[k]))
        Ew, Fw = o.weighted_average(F[:, k], Em[:, k])
        assert abs(Fw - lnZ) < 0.08, (betas[k], Fw, lnZ)
        assert abs(Ew - Eex) < 0.25, (betas[k], Ew, Eex)


def test_gaussian_invariants():
    J = inputs.gaussian_couplings_3d(4, 1, 1)
    r = o.GaussRun(J, 3, 4, 4, 4, 7, R0=800, seed=3)
    assert r.state().minus_beta_F == 64 * math.log(2.0)
    sp = r.spins()
    E = r.energies()
    for s in range(0, 800, 97):
        assert E[s] == r.energy_of(sp[s])
    r.step(0.0, 2, 800)
    st = r.state()
    assert st.lnQ_last == 0.0 and st.Qprime_last == 800.0
    assert int(r.copies(800).sum()) == st.R
