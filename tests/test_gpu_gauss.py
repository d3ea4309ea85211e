"""Parity of the CUDA path with the oracle for Gaussian couplings (the model of
the paper's Sec. 4), on the same seeded inputs.

Bit-exact: spins, fixed-point energies E_q, copy counts, population sizes,
the exact sum of E_q.  Within 1e-12 relative: ln Q, -beta F~ and the mean of
E^2 (the oracle adds (E_q 2^-15)^2 in replica order; the GPU sums E_q^2 as
exact integers and rounds once)."""
import math

import numpy as np
import pytest

from oracle import oracle as o
from paper_1006_0252_gb300 import inputs, pa

pytestmark = pytest.mark.gpu

RTOL = 1e-12
S = 2.0 ** -15


def close(a, b, rtol=RTOL):
    return abs(a - b) <= rtol * max(abs(a), abs(b), 1.0)


def make_pair(J, L, R0, seed, R_cap=None, tpb=0):
    cap = R_cap or inputs.default_capacity(R0)
    g = pa.Run(J, L, 3, R0, seed, R_cap=cap, threads_per_block=tpb, gaussian=True)
    c = o.GaussRun(J, 3, L, L, L, 7, R0=R0, R_cap=cap, seed=seed)
    return g, c


def energies_gauss(sp: np.ndarray, J: np.ndarray, L: int) -> np.ndarray:
    """E_q = sum_bonds J_q s_i s_j, independent numpy evaluation."""
    s = sp.reshape(-1, L, L, L).astype(np.int64)  # axes (z, y, x)
    Jx, Jy, Jz = (J[d].reshape(L, L, L).astype(np.int64) for d in range(3))
    E = (Jx * s * np.roll(s, -1, axis=3)).sum(axis=(1, 2, 3))
    E += (Jy * s * np.roll(s, -1, axis=2)).sum(axis=(1, 2, 3))
    E += (Jz * s * np.roll(s, -1, axis=1)).sum(axis=(1, 2, 3))
    return E


def assert_same_state(g, c, where, spins=True):
    go, co = g.observables(), c.state()
    assert go["R"] == co.R, where
    assert go["step"] == co.step and go["sweeps"] == co.sweeps, where
    assert go["sumE"] == co.sumE, where
    assert close(go["E_mean"], co.sumE * S / co.R), where
    assert close(go["E2_mean"], co.sumE2 / co.R), (where, go["E2_mean"], co.sumE2 / co.R)
    assert close(go["minus_beta_F"], co.minus_beta_F), (where, go["minus_beta_F"], co.minus_beta_F)
    assert close(go["lnQ_last"], co.lnQ_last, 1e-11) or abs(go["lnQ_last"] - co.lnQ_last) < 1e-12, where
    if spins:
        assert np.array_equal(g.energies().astype(np.int64), c.energies()), where
        assert np.array_equal(g.spins(), c.spins()), where


def test_init_matches_oracle_and_ln_omega():
    J = inputs.gaussian_couplings_3d(4, 0, 1)
    g, c = make_pair(J, 4, 1000, 1)
    assert g.free_energy() == 64 * math.log(2.0)
    assert_same_state(g, c, "init")
    assert np.array_equal(energies_gauss(g.spins(), J, 4), g.energies())


@pytest.mark.parametrize("L,tpb,split", [(4, 128, 4), (4, 64, 2), (8, 128, 4), (8, 64, 4), (8, 256, 2),
                                          (8, 128, 1), (12, 128, 4), (12, 64, 2), (6, 128, 1), (10, 32, 1),
                                          (8, 512, 1), (8, 512, 4), (8, 1024, 1), (8, 1024, 2), (8, 1024, 4),
                                          (6, 512, 1), (6, 1024, 1), (4, 1024, 4), (4, 512, 2)])
def test_threads_per_replica_bit_exact(L, tpb, split):
    """Every launch shape of the Gaussian cubic sweep gives the oracle's
    spins, energies and copy counts bit for bit (ragged population); blocks of
    512 and 1024 threads (L <= 8) decide through the per-site threshold
    tables."""
    J = inputs.gaussian_couplings_3d(L, 5, 1)
    R0 = 301 if L <= 8 else 133
    cap = inputs.default_capacity(R0)
    g = pa.Run(J, L, 3, R0, 13, R_cap=cap, threads_per_block=tpb, gaussian=True, threads_per_replica=split)
    c = o.GaussRun(J, 3, L, L, L, 7, R0=R0, R_cap=cap, seed=13)
    for k, beta in enumerate((0.3, 1.1, 2.6)):
        Rprev = c.state().R
        g.step(beta, 3)
        c.step(beta, 3, R0)
        assert np.array_equal(g.copies(Rprev), c.copies(Rprev)), k
        assert_same_state(g, c, f"L={L} tpb={tpb} split={split} step {k}")


@pytest.mark.parametrize("L", [4, 6, 8, 10, 12])
def test_every_lattice_size_bit_exact(L):
    J = inputs.gaussian_couplings_3d(L, 3, 7)
    R0 = 300 if L <= 10 else 130  # not a multiple of any block size
    g, c = make_pair(J, L, R0, 40 + L)
    betas = [0.15, 0.4, 0.4, 0.9, 1.6, 3.0]
    for k, beta in enumerate(betas):
        Rprev = c.state().R
        g.step(beta, 2)
        c.step(beta, 2, R0)
        assert np.array_equal(g.copies(Rprev), c.copies(Rprev)), (L, k)
        assert_same_state(g, c, f"L={L} step {k}")
    assert np.array_equal(energies_gauss(g.spins(), J, L), g.energies())


def test_paper_schedule_l4_two_runs():
    """The paper's 3D schedule shape (Sec. 4: 1/beta evenly spaced from 2 to
    0.2 after beta = 0) on L=4 with R=600, theta=5: every step bit-exact, then
    the overlap statistics between two runs match the oracle's."""
    J = inputs.gaussian_couplings_3d(4, 1, 1)
    T = np.linspace(2.0, 0.2, 40)
    betas = 1.0 / T
    pairs = [make_pair(J, 4, 600, s) for s in (1, 2)]
    for k, b in enumerate(betas):
        for g, c in pairs:
            Rprev = c.state().R
            g.step(float(b), 5)
            c.step(float(b), 5, 600)
            assert np.array_equal(g.copies(Rprev), c.copies(Rprev)), k
            assert_same_state(g, c, f"step {k}", spins=(k % 8 == 0 or k == len(betas) - 1))
    (ga, ca), (gb, cb) = pairs
    gg, gn, gh = pa.overlap(ga, gb)
    og, on, oh = o.overlap(ca, cb)
    assert gn == on and np.array_equal(gh, oh) and gg == og
    te = ga.trajectory_energy()
    tr = ga.trajectory()
    assert len(te["E_mean"]) == len(betas) + 1
    assert np.allclose(te["E_mean"], tr["sumE"] * S / tr["R"], rtol=0, atol=0)
    assert not tr["sumE2"].any()
    ob = ga.observables()
    assert te["E_mean"][-1] == ob["E_mean"] and te["E2_mean"][-1] == ob["E2_mean"]


def test_variable_target_zero_step_and_block_sizes():
    J = inputs.gaussian_couplings_3d(6, 1, 1)
    runs = [pa.Run(J, 6, 3, 800, 5, R_cap=2000, threads_per_block=t, gaussian=True)
            for t in (32, 64, 128, 256, 512, 1024)]
    c = o.GaussRun(J, 3, 6, 6, 6, 7, R0=800, R_cap=2000, seed=5)
    sched = [(0.3, 3, 800), (0.3, 2, 800), (0.9, 3, 1500), (1.4, 1, 1200)]
    for beta, th, Rt in sched:
        for g in runs:
            g.step(beta, th, R_target=Rt)
        c.step(beta, th, Rt)
        for g in runs:
            assert_same_state(g, c, f"beta {beta} target {Rt}")
    for g in runs:
        g.step(1.4, 1)
    c.step(1.4, 1, 800)
    assert runs[0].observables()["lnQ_last"] == 0.0 and c.state().lnQ_last == 0.0
    assert_same_state(runs[0], c, "zero step")


def test_large_step_heavy_replicas():
    """One large temperature step concentrates the weight on a few replicas,
    whose Poisson means need many pieces (block-cooperative sampling)."""
    J = inputs.gaussian_couplings_3d(6, 2, 1)
    g, c = make_pair(J, 6, 2000, 9, R_cap=4000)
    g.step(0.5, 3)
    c.step(0.5, 3, 2000)
    Rprev = c.state().R
    g.step(6.0, 2)
    c.step(6.0, 2, 2000)
    assert np.array_equal(g.copies(Rprev), c.copies(Rprev))
    assert c.copies(Rprev).max() > 8 * 32
    assert_same_state(g, c, "large step")


def test_checkpoint_restore_continues_exactly():
    J = inputs.gaussian_couplings_3d(8, 0, 2)
    a = pa.Run(J, 8, 3, 700, 3, gaussian=True)
    for b in (0.2, 0.5, 0.8):
        a.step(b, 2)
    blob = a.checkpoint()
    b_ = pa.Run(J, 8, 3, 700, 99, gaussian=True)
    b_.restore(blob)
    for b in (1.1, 1.5):
        a.step(b, 2)
        b_.step(b, 2)
    oa, ob = a.observables(), b_.observables()
    assert oa == ob
    assert np.array_equal(a.spins(), b_.spins())
    # a +-1 run of the same lattice refuses the Gaussian checkpoint
    pm = pa.Run(inputs.couplings_3d(8, 0, 2), 8, 3, 700, 3)
    with pytest.raises(pa.PAError):
        pm.restore(blob)


@pytest.mark.parametrize("beta", [0.0, 0.2, 1.0, 2.5, 5.0, 17.0])
def test_threshold_form_matches_oracle_decision(beta):
    """The threshold tables' integer decision (u >> 8) < thr is the oracle's
    float decision exactly: at every tabulated energy change the oracle
    accepts the largest u of 24-bit part thr - 1 and rejects the smallest of
    part thr, and dE <= 0 maps to 2^24 (always).  Energy changes near 0, of
    typical size, and large enough for the exponential to underflow."""
    rng = np.random.default_rng(int(beta * 100) + 7)
    dE = np.concatenate([np.arange(-40, 41), rng.integers(-(1 << 21), 1 << 21, 3000),
                         rng.integers(1, 1 << 16, 3000), rng.integers(1 << 20, 1 << 23, 300)]).astype(np.int32)
    thr = pa.gauss_thresholds(beta, dE)
    assert np.all(thr[dE <= 0] == 1 << 24)
    assert np.all(thr <= 1 << 24)
    def oracle(d, u):  # the oracle's rule: a fall or no change always, a rise by its float test
        return d <= 0 or o.gauss_accept(beta, d, u)

    for d, t in zip(dE.tolist(), thr.tolist()):
        if t >= 1:
            assert oracle(d, ((t - 1) << 8) | 0xFF), (beta, d, t)
        if t < (1 << 24):
            assert not oracle(d, t << 8), (beta, d, t)
    if beta >= 5.0:
        assert (thr == 0).any()  # the underflow branch is exercised


def test_host_side_argument_checks():
    J = inputs.gaussian_couplings_3d(4, 0, 1)
    with pytest.raises(pa.PAError) as e:
        pa.Run(inputs.gaussian_couplings_3d(14, 0, 1), 14, 3, 100, 1, gaussian=True)
    assert e.value.code == 7
    with pytest.raises(pa.PAError) as e:
        pa.Run(inputs.gaussian_couplings_chain(5000, 0, 1), 5000, 1, 100, 1, gaussian=True)
    assert e.value.code == 7
    bad = J.copy()
    bad[0, 0] = 1 << 20
    with pytest.raises(pa.PAError) as e:
        pa.Run(bad, 4, 3, 100, 1, gaussian=True)
    assert e.value.code == 1


def check_step(g, lat, J, L, beta_next, theta, R_target, rng, n_samples=40, n_last=0):
    pre = g.observables()
    pre_sp = g.spins()
    pre_E = g.energies().astype(np.int64)
    assert np.array_equal(energies_gauss(pre_sp, J, L), pre_E)
    g.step(beta_next, theta, R_target=R_target)
    post = g.observables()
    copies, Rn, Qp, lnQ = lat.resample(pre_E, pre["beta"], beta_next, R_target, pre["step"])
    assert np.array_equal(g.copies(len(pre_E)), copies)
    assert post["R"] == Rn
    assert close(post["lnQ_last"], lnQ, 1e-11) or abs(post["lnQ_last"] - lnQ) < 1e-12
    assert close(post["minus_beta_F"], pre["minus_beta_F"] + lnQ)
    src = np.repeat(np.arange(len(pre_E)), copies)
    post_sp = g.spins()
    post_E = g.energies().astype(np.int64)
    assert np.array_equal(energies_gauss(post_sp, J, L), post_E)
    assert int(post_E.sum()) == post["sumE"]
    e2 = float(((post_E * S) ** 2).sum()) / Rn
    assert close(post["E2_mean"], e2, 1e-11)
    # n_last more among the last 5000 slots, past the last whole wave of
    # resident threads, where the kernel may sweep a replica with 4 threads
    last = rng.integers(max(0, Rn - 5000), Rn, n_last)
    slots = np.unique(np.concatenate([[0, Rn - 1], rng.integers(0, Rn, n_samples), last]))
    for s in slots:
        sig, E = lat.sweep_replica(pre_sp[src[s]], int(s), pre["sweeps"], beta_next, theta)
        assert np.array_equal(post_sp[s], sig), s
        assert post_E[s] == E


def test_l8_r1e5_sampled():
    """L=8, R0=1e5 Gaussian run with the library's default launch
    configuration, the paper's temperature set (100 values of 1/beta evenly
    spaced in [0.2, 2] after beta = 0), theta=10: sampled steps checked against
    the oracle."""
    J = inputs.gaussian_couplings_3d(8, 0, 1)
    R0 = 100_000
    g = pa.Run(J, 8, 3, R0, 1, gaussian=True)
    lat = o.GaussRun(J, 3, 8, 8, 8, 7, R0=1, R_cap=1, seed=1)
    rng = np.random.default_rng(5)
    betas = 1.0 / np.linspace(2.0, 0.2, 100)
    check_step(g, lat, J, 8, float(betas[0]), 10, R0, rng, n_last=100)
    check_step(g, lat, J, 8, float(betas[1]), 10, R0, rng)
    for k in range(2, 99):
        g.step(float(betas[k]), 10)
    check_step(g, lat, J, 8, float(betas[99]), 10, R0, rng, n_last=100)
    tr = g.trajectory()
    assert len(tr["R"]) == 101 and np.all(np.abs(tr["R"][1:] - R0) < 10 * math.sqrt(R0))


def energies_chain_gauss(sp: np.ndarray, J: np.ndarray) -> np.ndarray:
    s = sp.astype(np.int64)
    return (J.astype(np.int64)[None, :] * s * np.roll(s, -1, axis=1)).sum(axis=1)


@pytest.mark.parametrize("N,open_chain", [(2, False), (33, True), (64, False), (70, True),
                                          (256, False), (4096, False)])
def test_chain_bit_exact(N, open_chain):
    J = inputs.gaussian_couplings_chain(N, 2, 5, open_chain=open_chain)
    R0 = 257 if N < 4096 else 60
    cap = inputs.default_capacity(R0)
    g = pa.Run(J, N, 1, R0, 11, R_cap=cap, gaussian=True)
    c = o.GaussRun(J, 1, N, R0=R0, R_cap=cap, seed=11)
    assert_same_state(g, c, f"N={N} init")
    for k, beta in enumerate([0.2, 0.5, 1.0, 1.0, 2.0, 3.5, 5.0]):
        Rprev = c.state().R
        g.step(beta, 3)
        c.step(beta, 3, R0)
        assert np.array_equal(g.copies(Rprev), c.copies(Rprev)), (N, k)
        assert_same_state(g, c, f"N={N} step {k}")
    assert np.array_equal(energies_chain_gauss(g.spins(), J), g.energies())


@pytest.mark.parametrize("N,open_chain,tpb", [(256, False, 32), (256, False, 256), (70, True, 128),
                                               (4096, False, 256)])
def test_chain_block_sizes_bit_exact(N, open_chain, tpb):
    """The chain kernel (threshold tables per site and pattern) at explicit
    block sizes; a size whose tables do not fit in shared memory (256 threads
    at N = 4096) falls back to the default block."""
    J = inputs.gaussian_couplings_chain(N, 4, 2, open_chain=open_chain)
    R0 = 301 if N < 4096 else 60
    cap = inputs.default_capacity(R0)
    g = pa.Run(J, N, 1, R0, 21, R_cap=cap, threads_per_block=tpb, gaussian=True)
    shape = pa.pa_sweep_shape(g._h)
    assert shape == ((tpb, 1) if N < 4096 else (64, 1)), shape
    c = o.GaussRun(J, 1, N, R0=R0, R_cap=cap, seed=21)
    for k, beta in enumerate([0.3, 1.2, 4.0]):
        Rprev = c.state().R
        g.step(beta, 4)
        c.step(beta, 4, R0)
        assert np.array_equal(g.copies(Rprev), c.copies(Rprev)), (N, k)
        assert_same_state(g, c, f"N={N} tpb={tpb} step {k}")


def test_odd_periodic_chain_rejected():
    J = inputs.gaussian_couplings_chain(33, 0, 1, open_chain=False)
    with pytest.raises(pa.PAError) as e:
        pa.Run(J, 33, 1, 100, 1, gaussian=True)
    assert e.value.code == 1


def test_gaussian_batch_matches_runs_alone():
    """Runs of the paper's two Gaussian studies (3D L=8, periodic chain N=256)
    at reduced population, batched in one graph launch per segment: each run
    is bit-identical to the same run alone."""
    specs3 = inputs.config_gauss_3d(n_real=2, runs_per_real=2, R0=700, theta=3)
    specs1 = inputs.config_gauss_1d(n_real=2, runs_per_real=2, R0=500, theta=3)
    for specs in (specs3, specs1):
        b = pa.Batch(specs)
        b.autotune()
        betas = specs[0].betas
        b.run(betas[1:5], thetas=specs[0].theta, use_graph=True)
        b.run(betas[5:9], thetas=specs[0].theta, use_graph=True)
        assert not b.sync().any()
        tr = b.trajectory(9)
        en = b.energy(9)
        for r, s in enumerate(specs):
            J = s.couplings()
            alone = pa.Run(J, s.L, s.dim, s.R0, s.seed, gaussian=True)
            for k in range(1, 9):
                alone.step(float(betas[k]), s.theta)
            ta = alone.trajectory()
            te = alone.trajectory_energy()
            assert np.array_equal(ta["R"], tr["R"][r]) and np.array_equal(ta["sumE"], tr["sumE"][r])
            assert np.array_equal(ta["minus_beta_F"], tr["minus_beta_F"][r])
            assert np.array_equal(te["E_mean"], en["E_mean"][r])
            assert np.array_equal(te["E2_mean"], en["E2_mean"][r])
            assert np.array_equal(alone.spins(), b.spins(r, s.R0 * 2))
            alone.close()
        b.close()
    # one of the batched runs, stepped alone, against the oracle
    s = specs3[0]
    alone = pa.Run(s.couplings(), 8, 3, s.R0, s.seed, gaussian=True)
    c = o.GaussRun(s.couplings(), 3, 8, 8, 8, 7, R0=s.R0, seed=s.seed)
    for k in range(1, 9):
        alone.step(float(s.betas[k]), s.theta)
        c.step(float(s.betas[k]), s.theta, s.R0)
    assert_same_state(alone, c, "batched run alone")


def test_mixed_models_in_one_batch_rejected():
    s3 = inputs.config_gauss_3d(n_real=1, runs_per_real=1, R0=300, theta=2)[0]
    pm = inputs.RunSpec(3, 8, 0, 1, 300, s3.betas, 2)
    with pytest.raises(pa.PAError):
        pa.Batch([s3, pm])


def test_device_detected_errors_and_reset():
    """Capacity overflow leaves the Gaussian run as it was (sticky error);
    extinction happens for exactly the seeds where the oracle dies out; a
    reset gives the same run as a fresh one with that seed."""
    J = inputs.gaussian_couplings_3d(4, 0, 1)
    g = pa.Run(J, 4, 3, 100, 3, R_cap=300, gaussian=True)
    g.step(0.1, 1, R_target=100)
    before = g.observables()
    g.step(0.2, 1, R_target=100000)
    with pytest.raises(pa.PAError) as e:
        g.sync()
    assert e.value.code == pa.PA_ERR_CAPACITY
    lib = pa.load()
    obs = pa.Obs()
    assert lib.pa_observables(g._h, obs) == pa.PA_ERR_CAPACITY
    assert obs.step == before["step"] and obs.R == before["R"] and obs.sumE == before["sumE"]
    assert obs.minus_beta_F == before["minus_beta_F"]
    # reset clears the error and starts over: identical to a fresh run with the new seed
    g.reset(11)
    f = pa.Run(J, 4, 3, 100, 11, R_cap=300, gaussian=True)
    for beta in (0.3, 0.9):
        g.step(beta, 2)
        f.step(beta, 2)
    assert g.observables() == f.observables()
    assert np.array_equal(g.spins(), f.spins())
    for s in range(1, 25):
        gg = pa.Run(J, 4, 3, 4, s, gaussian=True)
        gg.step(0.2, 1, R_target=1)
        cc = o.GaussRun(J, 3, 4, 4, 4, 7, R0=4, seed=s)
        try:
            cc.step(0.2, 1, 1)
            died = False
        except o.OracleError as err:
            died = err.code == o.ERR_EXTINCT
        code = lib.pa_sync(gg._h)
        assert (code == pa.PA_ERR_EXTINCT) == died, s
        if not died:
            assert code == pa.PA_OK
            assert gg.observables()["R"] == cc.state().R


def test_schedule_graph_equals_steps():
    """A Gaussian run's schedule replayed as one CUDA graph (pa_run_schedule)
    gives the bits of the same steps taken one at a time, for a cubic
    lattice and a chain."""
    for J, L, dim in ((inputs.gaussian_couplings_3d(6, 2, 1), 6, 3),
                      (inputs.gaussian_couplings_chain(96, 1, 3, open_chain=False), 96, 1)):
        betas = np.linspace(0.2, 3.0, 10)
        a = pa.Run(J, L, dim, 800, 5, gaussian=True)
        for beta in betas:
            a.step(float(beta), 3)
        b = pa.Run(J, L, dim, 800, 5, gaussian=True)
        b.run_schedule(betas, 3, use_graph=True)
        ta, tb = a.trajectory(), b.trajectory()
        for key in ta:
            assert np.array_equal(ta[key], tb[key]), (dim, key)
        assert np.array_equal(a.spins(), b.spins()) and np.array_equal(a.energies(), b.energies())
        a.close()
        b.close()
