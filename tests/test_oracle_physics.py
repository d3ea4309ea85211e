"""Pins for the oracle's population-annealing arithmetic (CPU only).

The oracle is held to what the paper and the mathematics fix, never to
itself: exact enumeration of 2x2x2 and 2x2x3 lattices (ln Z, <E>, the
Boltzmann distribution), the closed form of the open +-1 chain, the exact
invariants of Sec. 2 (ln Omega = N ln 2 at beta = 0, Q = 1 for a zero step,
population totals), and exact binomial overlap statistics at beta = 0."""
import math

import numpy as np
import pytest

import brute
from oracle import oracle as o
from paper_1006_0252_gb300 import inputs


def _box(Lx, Ly, Lz, mask, real=0, seed=1):
    J = inputs.couplings_lattice(Lx, Ly, Lz, real, seed)
    return J, brute.energies(brute.bonds_3d(J, Lx, Ly, Lz, mask), Lx * Ly * Lz)


def test_init_invariants_3d():
    J = inputs.couplings_3d(4, 0, 1)
    r = o.Run(J, 3, 4, 4, 4, 7, R0=500, seed=3)
    st = r.state()
    assert st.minus_beta_F == 64 * math.log(2.0)  # ln Omega, exact at beta = 0
    assert st.Nb == 192 and st.R == 500 and st.step == 0
    sp = r.spins()
    assert set(np.unique(sp)) <= {-1, 1}
    E = r.energies()
    bonds = brute.bonds_3d(J, 4, 4, 4, 7)
    for s in range(0, 500, 37):  # energies against the independent bond list
        assert E[s] == sum(Jb * sp[s, i] * sp[s, j] for i, j, Jb in bonds)
    assert len(set((E % 4).tolist())) == 1  # +-1 couplings, 3D: E is fixed mod 4
    assert abs(sp.mean()) < 5.0 / math.sqrt(sp.size)
    assert st.sumE == int(E.sum()) and st.sumE2 == int((E.astype(np.int64) ** 2).sum())


def test_init_spins_follow_keying_spec():
    J = inputs.couplings_3d(6, 2, 1)
    seed = 0x1234_5678_9ABC
    r = o.Run(J, 3, 6, 6, 6, 7, R0=7, seed=seed)
    sp = r.spins()
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for s in range(7):
        for i in range(0, 216, 5):
            w, p, _ = r.site_label(i)
            word = o.philox((w >> 2, s, 0, o.TAG_INIT), key)[w & 3]
            assert sp[s, i] == (-1 if (word >> p) & 1 else 1)


def test_keying_labels_are_a_bijection():
    for L in (2, 4, 6, 8, 10, 12, 14):
        J = inputs.couplings_3d(L, 0, 1)
        r = o.Run(J, 3, L, L, L, 7, R0=1, seed=1)
        seen = set()
        ranks = ([], [])
        for i in range(L ** 3):
            w, p, S = r.site_label(i)
            x, y, z = i % L, (i // L) % L, i // (L * L)
            c = (x + y + z) & 1
            assert 0 <= p < 32
            assert (w, p) not in seen
            seen.add((w, p))
            assert (p & 1) == (x & 1)
            seen.add(("m", w, p >> 1, c))
            ranks[c].append(w * S + (p >> 1))
        assert len(seen) == 2 * L ** 3  # (w, m, colour) is unique too
        # the sweep uniforms: the colour-c sites' ranks w S + m are exactly
        # 0 .. N/2 - 1, so every Philox output is used once and none is shared
        for c in (0, 1):
            assert sorted(ranks[c]) == list(range(L ** 3 // 2))
    r = o.Run(inputs.couplings_chain(70), 1, 70, R0=1, seed=1)
    assert r.site_label(69) == (2, 5, 16)
    r = o.Run(inputs.couplings_3d(6, 0, 1), 3, 6, 6, 6, 7, R0=1, seed=1)
    assert r.site_label(0)[2] == 9  # 3 lanes of 6 bits: 9 sites of each colour per word


def test_zero_step_has_unit_Q_and_poisson_population():
    J = inputs.couplings_3d(4, 1, 1)
    r = o.Run(J, 3, 4, 4, 4, 7, R0=2000, seed=5)
    f0 = r.state().minus_beta_F
    r.step(0.0, 2, 2000)
    st = r.state()
    assert st.lnQ_last == 0.0 and st.Qprime_last == 2000.0
    assert st.minus_beta_F == f0
    c = r.copies(2000)
    assert int(c.sum()) == st.R
    assert abs(st.R - 2000) < 5 * math.sqrt(2000)
    # copies are Poisson(1): mean 1, variance 1
    assert abs(c.mean() - 1.0) < 0.12 and abs(c.var() - 1.0) < 0.2


def test_population_total_tracks_target():
    J = inputs.couplings_3d(4, 0, 1)
    r = o.Run(J, 3, 4, 4, 4, 7, R0=1000, R_cap=2000, seed=9)
    for k, b in enumerate(inputs.linear_schedule(2.0, 21)[1:]):
        prev = r.state().R
        target = 1000 if k < 10 else 1500  # temperature-dependent R_beta of Sec. 4
        r.step(float(b), 3, target)
        st = r.state()
        assert int(r.copies(prev).sum()) == st.R
        assert abs(st.R - target) < 6 * math.sqrt(target)


def _pa_runs(J, dim, Lx, Ly, Lz, mask, R, betas, theta, seeds):
    """-beta F~ and E-bar per run at every beta of the schedule."""
    F = np.zeros((len(seeds), len(betas)))
    Em = np.zeros((len(seeds), len(betas)))
    for a, s in enumerate(seeds):
        r = o.Run(J, dim, Lx, Ly, Lz, mask, R0=R, seed=s)
        st = r.state()
        F[a, 0], Em[a, 0] = st.minus_beta_F, st.sumE / st.R
        for k in range(1, len(betas)):
            r.step(float(betas[k]), theta, R)
            st = r.state()
            F[a, k], Em[a, k] = st.minus_beta_F, st.sumE / st.R
        r.close()
    return F, Em


@pytest.mark.parametrize("shape", [(2, 2, 2, 7), (2, 2, 3, 3)])
def test_pa_matches_exact_enumeration(shape):
    Lx, Ly, Lz, mask = shape
    J, Es = _box(Lx, Ly, Lz, mask, real=4)
    betas = inputs.linear_schedule(2.0, 21)
    F, Em = _pa_runs(J, 3, Lx, Ly, Lz, mask, 3000, betas, 4, seeds=range(1, 7))
    for k, b in enumerate(betas):
        lnZ, Eex, varE = brute.exact(Es, float(b))
        Fbar = np.log(np.mean(np.exp(F[:, k] - F[:, k].max()))) + F[:, k].max()
        _, Fbar_or = o.weighted_average(F[:, k], Em[:, k])
        assert abs(Fbar - Fbar_or) < 1e-9
        # free energy (Eqs. (4), (7)): tiny systems, R = 3000 -> error ~ 1e-2
        assert abs(Fbar_or - lnZ) < 0.03, (b, Fbar_or, lnZ)
        # energy: population mean, error from the spread over runs
        Ew, _ = o.weighted_average(F[:, k], Em[:, k])
        err = max(Em[:, k].std(ddof=1) / math.sqrt(len(Em)), 0.02 * math.sqrt(varE) + 1e-3)
        assert abs(Ew - Eex) < 6 * err + 0.02, (b, Ew, Eex, err)


def test_metropolis_sweeps_sample_boltzmann_distribution():
    """Detailed balance of the checkerboard sweep: independent replicas after
    many sweeps at fixed beta follow exp(-beta E)/Z over all 256 states of a
    2x2x2 box, and over the energy levels of a 4x2x2 box (where energy rises
    of 4, 8 and 12 all occur)."""
    st = pytest.importorskip("scipy.stats")

    def chi2_p(counts, p):
        exp_counts = p * counts.sum()
        keep = exp_counts >= 5
        rest_o, rest_e = counts[~keep].sum(), exp_counts[~keep].sum()
        chi2 = (((counts - exp_counts) ** 2 / exp_counts)[keep]).sum()
        dof = int(keep.sum()) - 1
        if rest_e > 0:
            chi2 += (rest_o - rest_e) ** 2 / rest_e
            dof += 1
        return st.chi2.sf(chi2, dof)

    J, Es = _box(2, 2, 2, 7, real=2)
    beta = 0.45
    r = o.Run(J, 3, 2, 2, 2, 7, R0=20000, seed=21)
    r.sweep_fixed(beta, 40)
    sp = r.spins()
    idx = ((sp < 0).astype(np.int64) << np.arange(8)).sum(axis=1)
    p = np.exp(-beta * Es - (-beta * Es).max())
    assert chi2_p(np.bincount(idx, minlength=256), p / p.sum()) > 1e-4
    # the energy tracked through the sweeps equals the recomputed one
    assert np.array_equal(r.energies(), Es[idx])

    J, Es = _box(4, 2, 2, 7, real=1)
    levels, g = np.unique(Es, return_counts=True)
    for beta, seed in ((0.35, 5), (0.8, 6)):
        r = o.Run(J, 3, 4, 2, 2, 7, R0=20000, seed=seed)
        r.sweep_fixed(beta, 60)
        E = r.energies()
        counts = np.array([(E == e).sum() for e in levels])
        assert counts.sum() == len(E)
        lw = np.log(g) - beta * levels
        p = np.exp(lw - lw.max())
        assert chi2_p(counts, p / p.sum()) > 1e-4, beta


def test_open_chain_closed_form():
    """Open +-1 chain: ln Z = N ln 2 + (N-1) ln cosh beta, <E> = -(N-1) tanh beta."""
    N = 48
    J = inputs.couplings_chain(N, 3, 1, open_chain=True)
    betas = inputs.linear_schedule(2.0, 31)
    F, Em = _pa_runs(J, 1, N, 1, 1, 0, 2000, betas, 5, seeds=range(1, 5))
    for k, b in enumerate(betas):
        lnZ = N * math.log(2.0) + (N - 1) * math.log(math.cosh(b))
        Eex = -(N - 1) * math.tanh(b)
        Ew, Fw = o.weighted_average(F[:, k], Em[:, k])
        assert abs(Fw - lnZ) < 0.08, (b, Fw, lnZ)
        sd = math.sqrt((N - 1) / math.cosh(b) ** 2)
        assert abs(Ew - Eex) < 6 * sd / math.sqrt(2000) * 3 + 0.05, (b, Ew, Eex)


def test_closed_form_values_quoted_for_the_large_chain():
    # closed-form anchors for the N = 4096 open chain used by the benchmarks
    N = 4096
    lnZ = lambda b: N * math.log(2.0) + (N - 1) * math.log(math.cosh(b))
    assert abs(lnZ(0.0) - 2839.130851573536) < 1e-9
    assert abs(lnZ(1.0) - 4615.463352401532) < 1e-9
    assert abs(lnZ(4.0) - 16382.066636277568) < 1e-8
    assert abs(-(N - 1) * math.tanh(4.0) + 4092.2534824314794) < 1e-9


def test_weighted_estimator_is_unbiased_where_single_runs_are_not():
    """Sec. 3: with a small population each run's -beta F~ is biased low, the
    ln of the mean of exp(-beta F~) (Eq. (7)) is not."""
    N = 32
    J = inputs.couplings_chain(N, 5, 1, open_chain=True)
    betas = inputs.linear_schedule(3.0, 13)
    F, Em = _pa_runs(J, 1, N, 1, 1, 0, 12, betas, 1, seeds=range(100, 260))
    lnZ = N * math.log(2.0) + (N - 1) * math.log(math.cosh(3.0))
    _, Fw = o.weighted_average(F[:, -1], Em[:, -1])
    _, sF = o.bootstrap(F[:, -1], Em[:, -1], B=200, seed=4)
    unweighted = F[:, -1].mean()
    assert abs(Fw - lnZ) < 4 * sF + 0.02, (Fw, lnZ, sF)
    assert unweighted < lnZ - 2 * F[:, -1].std(ddof=1) / math.sqrt(len(F))


def test_overlap_exact_cases():
    st = pytest.importorskip("scipy.stats")
    J = inputs.couplings_3d(4, 0, 1)
    a = o.Run(J, 3, 4, 4, 4, 7, R0=3000, seed=11)
    b = o.Run(J, 3, 4, 4, 4, 7, R0=3000, seed=11)
    g, n, hist = o.overlap(a, b)
    assert g == 0.0 and n == 3000 and hist[-1] == 3000  # identical runs: q = 1
    c = o.Run(J, 3, 4, 4, 4, 7, R0=3000, seed=12)
    g, n, hist = o.overlap(a, c)
    # beta = 0: dot = N - 2 Binomial(N, 1/2); Prob(|dot| < 0.2 N) exactly
    N = 64
    ks = np.arange(N + 1)
    dots = N - 2 * ks
    p = st.binom.pmf(ks, N, 0.5)[np.abs(dots) < 0.2 * N].sum()
    assert abs(g - p) < 5 * math.sqrt(p * (1 - p) / n)


def test_error_paths_leave_state_untouched():
    J = inputs.couplings_3d(4, 0, 1)
    r = o.Run(J, 3, 4, 4, 4, 7, R0=100, R_cap=100, seed=1)
    before = r.state()
    with pytest.raises(o.OracleError) as e:
        r.step(0.1, 1, 10_000)
    assert e.value.code == o.ERR_CAPACITY
    after = r.state()
    assert after.R == before.R and after.minus_beta_F == before.minus_beta_F
    assert after.step == 0 and np.array_equal(r.spins().shape, (100, 64))
    with pytest.raises(o.OracleError) as e:
        r.step(-0.5, 1, 100)
    assert e.value.code == o.ERR_INVALID
    # odd periodic extent is not bipartite
    with pytest.raises(o.OracleError):
        o.Run(inputs.couplings_lattice(4, 3, 4), 3, 4, 3, 4, 7, R0=5, seed=1)
    o.Run(inputs.couplings_lattice(4, 3, 4), 3, 4, 3, 4, 5, R0=5, seed=1)  # open y is fine
    # extinction: target of one replica; some seed dies out on the first step
    hit = False
    for s in range(1, 40):
        r = o.Run(J, 3, 4, 4, 4, 7, R0=4, seed=s)
        try:
            r.step(0.2, 1, 1)
        except o.OracleError as err:
            assert err.code == o.ERR_EXTINCT
            assert r.state().R == 4
            hit = True
            break
    assert hit
