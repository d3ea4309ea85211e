"""Parity of general lattices (pa_create_lattice): Lx x Ly x Lz boxes with any
periodic/open axes, both coupling models, and chains given by extents, against
the oracle on the same seeded inputs (bit-exact spins, energies, copy counts,
population sizes and exact energy sums; -beta F~ within 1e-12)."""
import math

import numpy as np
import pytest

from oracle import oracle as o
from paper_1006_0252_gb300 import inputs, pa

pytestmark = pytest.mark.gpu

S = 2.0 ** -15


def close(a, b, rtol=1e-12):
    return abs(a - b) <= rtol * max(abs(a), abs(b), 1.0)


def same_state(g, c, where, gaussian):
    go, co = g.observables(), c.state()
    assert go["R"] == co.R, where
    assert go["step"] == co.step and go["sweeps"] == co.sweeps, where
    assert go["sumE"] == co.sumE, where
    if gaussian:
        assert close(go["E2_mean"], co.sumE2 / co.R), where
    else:
        assert go["sumE2"] == co.sumE2, where
    assert close(go["minus_beta_F"], co.minus_beta_F), (where, go["minus_beta_F"], co.minus_beta_F)
    assert np.array_equal(g.energies().astype(np.int64), c.energies().astype(np.int64)), where
    assert np.array_equal(g.spins(), c.spins()), where


# (Lx, Ly, Lz, periodic mask): small boxes for exact enumeration, open and
# mixed boundaries, odd open extents, flat and thin shapes, a cubic lattice
# with an open axis, a non-cubic fully periodic box, and words whose
# colour-c sites are not a multiple of 4 (uniforms shared across words)
BOXES = [(2, 2, 2, 7), (2, 2, 3, 3), (4, 2, 3, 1), (6, 4, 2, 0), (4, 4, 6, 7), (2, 3, 4, 5),
         (8, 1, 1, 1), (2, 1, 1, 0), (32, 2, 2, 7), (4, 4, 4, 3), (10, 6, 4, 6), (2, 2, 64, 7),
         (6, 2, 3, 1), (6, 3, 5, 1)]  # the last two: 9 and 15 colour-c sites per word


@pytest.mark.parametrize("gaussian", [False, True])
@pytest.mark.parametrize("box", BOXES)
def test_box_bit_exact(box, gaussian):
    Lx, Ly, Lz, mask = box
    if gaussian:
        J = inputs.gaussian_couplings_lattice(Lx, Ly, Lz, 4)
    else:
        J = inputs.couplings_lattice(Lx, Ly, Lz, 4, 3)
    R0 = 300
    cap = inputs.default_capacity(R0)
    g = pa.Run(J, Lx, 3, R0, 21, R_cap=cap, gaussian=gaussian, Ls=(Lx, Ly, Lz), periodic_mask=mask)
    Cls = o.GaussRun if gaussian else o.Run
    c = Cls(J, 3, Lx, Ly, Lz, mask, R0=R0, R_cap=cap, seed=21)
    same_state(g, c, f"{box} init", gaussian)
    for k, beta in enumerate([0.2, 0.5, 1.0, 1.0, 2.0, 3.5]):
        Rprev = c.state().R
        g.step(beta, 2)
        c.step(beta, 2, R0)
        assert np.array_equal(g.copies(Rprev), c.copies(Rprev)), (box, k)
        same_state(g, c, f"{box} step {k}", gaussian)


@pytest.mark.parametrize("gaussian", [False, True])
@pytest.mark.parametrize("N,mask", [(40, 1), (41, 0), (256, 1)])
def test_chain_by_extents(N, mask, gaussian):
    if gaussian:
        J = inputs.gaussian_couplings_chain(N, 1, 2)
    else:
        J = inputs.couplings_chain(N, 1, 2, open_chain=False)
    Jo = J.copy()
    if not mask & 1:
        Jo[N - 1] = 0  # an open chain: the stored wrap coupling is ignored
    g = pa.Run(J, N, 1, 257, 4, gaussian=gaussian, Ls=(N, 1, 1), periodic_mask=mask)
    c = (o.GaussRun if gaussian else o.Run)(Jo, 1, N, R0=257, seed=4)
    for k, beta in enumerate([0.3, 1.0, 2.5]):
        g.step(beta, 3)
        c.step(beta, 3, 257)
        same_state(g, c, f"chain {N} step {k}", gaussian)


def test_cubic_periodic_extents_use_the_cubic_lattice():
    """pa_create_lattice on L x L x L, all axes periodic, is the same run as
    pa_create (the cubic kernels)."""
    J = inputs.couplings_3d(6, 0, 1)
    a = pa.Run(J, 6, 3, 500, 3)
    b = pa.Run(J, 6, 3, 500, 3, Ls=(6, 6, 6), periodic_mask=7)
    for beta in (0.4, 1.2):
        a.step(beta, 2)
        b.step(beta, 2)
    assert a.observables() == b.observables()
    assert np.array_equal(a.spins(), b.spins())


def test_box_pa_matches_exact_enumeration():
    """The GPU's weighted estimates on the 2x2x3 box with open z (Sec. 3
    averages over independent runs) against exact enumeration of its 4096
    states."""
    import brute
    Lx, Ly, Lz, mask = 2, 2, 3, 3
    J = inputs.couplings_lattice(Lx, Ly, Lz, 4, 3)
    Es = brute.energies(brute.bonds_3d(J, Lx, Ly, Lz, mask), Lx * Ly * Lz).astype(np.float64)
    betas = inputs.linear_schedule(2.0, 11)
    F = np.zeros((8, len(betas)))
    Em = np.zeros((8, len(betas)))
    for r in range(8):
        g = pa.Run(J, Lx, 3, 2000, 100 + r, Ls=(Lx, Ly, Lz), periodic_mask=mask)
        for k in range(1, len(betas)):
            g.step(float(betas[k]), 4)
        tr = g.trajectory()
        F[r] = tr["minus_beta_F"]
        Em[r] = tr["sumE"] / tr["R"]
    # The spread of -beta F~ that independent equilibrium replicas would give,
    # from the exact partition functions: step l adds Var(ln Q_l) =
    # (Z(b_{l-1}) Z(b_{l-1} + 2 db) / Z(b_l)^2 - 1) / R (Eqs. (2)-(4) with Q the
    # mean of R independent weights); KAPPA allows for the correlation of the
    # copies a resampling makes (an effective population of at least R / 4).
    R, M, KAPPA = 2000, 8, 4.0
    lnz = lambda b: brute.exact(Es, float(b))[0]
    var_f = 0.0
    for k, b in enumerate(betas):
        if k > 0:
            db = float(betas[k] - betas[k - 1])
            var_f += (math.exp(lnz(betas[k - 1]) + lnz(betas[k - 1] + 2 * db) - 2 * lnz(betas[k])) - 1.0) / R
        lnZ, Eex, varE = brute.exact(Es, float(b))
        Ew, Fw = pa.pa_weighted_average(F[:, k], Em[:, k])
        bound_f = 4.0 * math.sqrt(KAPPA * var_f / M) + 1e-9
        assert abs(Fw - lnZ) < bound_f, (b, Fw, lnZ, bound_f)
        assert abs(Ew - Eex) < 0.1 + 4.0 * math.sqrt(varE / (M * R)), (b, Ew, Eex)


def test_box_checkpoint_and_errors():
    J = inputs.couplings_lattice(4, 2, 3, 0, 1)
    a = pa.Run(J, 4, 3, 400, 5, Ls=(4, 2, 3), periodic_mask=3)
    a.step(0.5, 2)
    blob = a.checkpoint()
    b = pa.Run(J, 4, 3, 400, 9, Ls=(4, 2, 3), periodic_mask=3)
    b.restore(blob)
    a.step(1.0, 2)
    b.step(1.0, 2)
    assert a.observables() == b.observables()
    # the same couplings with z open differ in their bond set: refused
    c = pa.Run(J, 4, 3, 400, 9, Ls=(4, 2, 3), periodic_mask=1)
    with pytest.raises(pa.PAError):
        c.restore(blob)
    with pytest.raises(pa.PAError) as e:  # odd Lx
        pa.Run(inputs.couplings_lattice(3, 2, 2, 0, 1), 3, 3, 100, 1, Ls=(3, 2, 2), periodic_mask=0)
    assert e.value.code == 1
    with pytest.raises(pa.PAError) as e:  # periodic z of odd length
        pa.Run(J, 4, 3, 100, 1, Ls=(4, 2, 3), periodic_mask=7)
    assert e.value.code == 1
    with pytest.raises(pa.PAError) as e:  # too many sites for the general kernel
        big = inputs.couplings_lattice(16, 16, 16, 0, 1)
        pa.Run(big, 16, 3, 100, 1, Ls=(16, 16, 16), periodic_mask=3)
    assert e.value.code == 7


@pytest.mark.parametrize("gaussian", [False, True])
def test_box_schedule_graph_equals_steps(gaussian):
    Lx, Ly, Lz, mask = 4, 2, 3, 3
    J = inputs.gaussian_couplings_lattice(Lx, Ly, Lz, 4) if gaussian else inputs.couplings_lattice(Lx, Ly, Lz, 4, 3)
    betas = np.linspace(0.3, 2.5, 8)
    a = pa.Run(J, Lx, 3, 500, 6, gaussian=gaussian, Ls=(Lx, Ly, Lz), periodic_mask=mask)
    for beta in betas:
        a.step(float(beta), 2)
    b = pa.Run(J, Lx, 3, 500, 6, gaussian=gaussian, Ls=(Lx, Ly, Lz), periodic_mask=mask)
    b.run_schedule(betas, 2, use_graph=True)
    assert a.observables() == b.observables()
    assert np.array_equal(a.spins(), b.spins())
