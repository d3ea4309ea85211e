"""Parity of the CUDA path with the oracle on the same seeded inputs.

Bit-exact: spins, energies, copy counts, population sizes, integer energy
sums, overlap counts.  Within 1e-12 relative: ln Q, -beta F~ and the
weighted averages (the GPU takes log/exp from CUDA's libdevice, the oracle
from the C library; every quantity that decides an integer is computed with
the deterministic exp on both sides)."""
import math

import numpy as np
import pytest

from oracle import oracle as o
from paper_1006_0252_gb300 import inputs, pa

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def close(a, b, rtol=RTOL):
    return abs(a - b) <= rtol * max(abs(a), abs(b), 1.0)


def make_pair(J, L, dim, R0, seed, R_cap=None, tpb=0):
    cap = R_cap or inputs.default_capacity(R0)
    g = pa.Run(J, L, dim, R0, seed, R_cap=cap, threads_per_block=tpb)
    if dim == 3:
        c = o.Run(J, 3, L, L, L, 7, R0=R0, R_cap=cap, seed=seed)
    else:
        c = o.Run(J, 1, L, R0=R0, R_cap=cap, seed=seed)
    return g, c


def assert_same_state(g, c, where, spins=True):
    go, co = g.observables(), c.state()
    assert go["R"] == co.R, where
    assert go["step"] == co.step and go["sweeps"] == co.sweeps, where
    assert go["sumE"] == co.sumE and go["sumE2"] == co.sumE2, where
    assert close(go["minus_beta_F"], co.minus_beta_F), (where, go["minus_beta_F"], co.minus_beta_F)
    assert close(go["lnQ_last"], co.lnQ_last, 1e-11) or abs(go["lnQ_last"] - co.lnQ_last) < 1e-12, where
    if spins:
        assert np.array_equal(g.energies(), c.energies()), where
        assert np.array_equal(g.spins(), c.spins()), where


def test_init_matches_oracle_and_ln_omega():
    J = inputs.couplings_3d(4, 0, 1)
    g, c = make_pair(J, 4, 3, 1000, 1)
    assert g.free_energy() == 64 * math.log(2.0)
    assert_same_state(g, c, "init")


def test_small_3d_full_schedule_bit_exact():
    """3D L=4, R0=1000, 101 betas 0..5, theta=10, two runs (seeds 1, 2): every
    step, every replica; then the overlap Gamma of Sec. 4 between the runs."""
    specs = inputs.config_small_3d()
    pairs = [make_pair(s.couplings(), 4, 3, s.R0, s.seed) for s in specs]
    b = specs[0].betas
    for k in range(1, len(b)):
        for g, c in pairs:
            Rprev = c.state().R
            g.step(float(b[k]), 10)
            c.step(float(b[k]), 10, 1000)
            assert np.array_equal(g.copies(Rprev), c.copies(Rprev)), k
            assert_same_state(g, c, f"step {k}", spins=(k % 10 == 0 or k < 4))
    (ga, ca), (gb, cb) = pairs
    gg, gn, gh = pa.overlap(ga, gb)
    og, on, oh = o.overlap(ca, cb)
    assert gn == on and np.array_equal(gh, oh) and gg == og
    traj = ga.trajectory()
    assert len(traj["R"]) == 101 and traj["R"][-1] == ca.state().R


@pytest.mark.parametrize("L,tpb,split", [(4, 64, 2), (4, 128, 4), (4, 256, 4), (4, 32, 1), (8, 64, 8),
                                          (8, 128, 4), (8, 256, 2), (8, 128, 1), (8, 128, 8), (12, 64, 4),
                                          (12, 128, 2), (12, 256, 4), (12, 32, 1), (16, 64, 8), (16, 128, 4),
                                          (16, 64, 2)])
def test_threads_per_replica_bit_exact(L, tpb, split):
    """Every launch shape of the +-1 cubic sweep (block size x threads per
    replica) gives the oracle's spins, energies and copy counts bit for bit;
    the population is not a multiple of any block's replicas (ragged tail)."""
    J = inputs.couplings_3d(L, 5, 1)
    R0 = 301 if L <= 8 else 133
    cap = inputs.default_capacity(R0)
    g = pa.Run(J, L, 3, R0, 11, R_cap=cap, threads_per_block=tpb, threads_per_replica=split)
    c = o.Run(J, 3, L, L, L, 7, R0=R0, R_cap=cap, seed=11)
    for k, beta in enumerate((0.3, 1.1, 2.6, 4.0)):
        Rprev = c.state().R
        g.step(beta, 3)
        c.step(beta, 3, R0)
        assert np.array_equal(g.copies(Rprev), c.copies(Rprev)), k
        assert_same_state(g, c, f"L={L} tpb={tpb} split={split} step {k}")


@pytest.mark.parametrize("N,tpb,split,open_chain", [(4096, 128, 8, True), (4096, 256, 8, True), (4096, 64, 4, True),
                                                     (1000, 128, 4, True),
                                                     (1000, 256, 8, False), (96, 128, 2, True), (70, 64, 4, False),
                                                     (70, 32, 1, True), (4096, 32, 1, True)])
def test_chain_threads_per_replica_bit_exact(N, tpb, split, open_chain):
    """The +-1 chain sweep on word ranges (P threads per replica, ranges of
    ceil(words / P) words, the last one short or empty) against the oracle."""
    J = inputs.couplings_chain(N, 3, 1, open_chain=open_chain)
    R0 = 301
    cap = inputs.default_capacity(R0)
    g = pa.Run(J, N, 1, R0, 17, R_cap=cap, threads_per_block=tpb, threads_per_replica=split)
    c = o.Run(J, 1, N, R0=R0, R_cap=cap, seed=17)
    for k, beta in enumerate((0.3, 1.2, 2.5)):
        Rprev = c.state().R
        g.step(beta, 3)
        c.step(beta, 3, R0)
        assert np.array_equal(g.copies(Rprev), c.copies(Rprev)), k
        assert_same_state(g, c, f"N={N} tpb={tpb} split={split} step {k}")


def test_threads_per_replica_rejected_where_rows_do_not_split():
    with pytest.raises(pa.PAError):
        pa.Run(inputs.couplings_3d(6, 0, 1), 6, 3, 100, 1, threads_per_replica=2)
    with pytest.raises(pa.PAError):
        pa.Run(inputs.couplings_3d(8, 0, 1), 8, 3, 100, 1, threads_per_replica=3)
    with pytest.raises(pa.PAError):
        pa.Run(inputs.couplings_3d(8, 0, 1), 8, 3, 100, 1, threads_per_block=32, threads_per_replica=4)


@pytest.mark.parametrize("L", [2, 4, 6, 8, 10, 12, 14, 16])
def test_every_lattice_size_bit_exact(L):
    J = inputs.couplings_3d(L, 3, 7)
    R0 = 300 if L <= 10 else 130  # not a multiple of any block size
    g, c = make_pair(J, L, 3, R0, 40 + L)
    betas = [0.15, 0.4, 0.4, 0.9, 1.6]
    for k, beta in enumerate(betas):
        g.step(beta, 2)
        c.step(beta, 2, R0)
        assert_same_state(g, c, f"L={L} step {k}")


@pytest.mark.parametrize("N,open_chain", [(2, False), (33, True), (64, False), (70, True),
                                          (96, False), (4096, True)])
def test_chain_bit_exact(N, open_chain):
    J = inputs.couplings_chain(N, 2, 5, open_chain=open_chain)
    R0 = 257 if N < 4096 else 60
    g, c = make_pair(J, N, 1, R0, 11)
    for k, beta in enumerate([0.2, 0.5, 1.0, 1.0, 2.0, 3.5]):
        g.step(beta, 3)
        c.step(beta, 3, R0)
        assert_same_state(g, c, f"N={N} step {k}")


def test_variable_target_zero_step_and_block_sizes():
    J = inputs.couplings_3d(6, 1, 1)
    runs = [pa.Run(J, 6, 3, 800, 5, R_cap=2000, threads_per_block=t) for t in (32, 64, 128, 256)]
    c = o.Run(J, 3, 6, 6, 6, 7, R0=800, R_cap=2000, seed=5)
    sched = [(0.3, 3, 800), (0.3, 2, 800), (0.9, 3, 1500), (1.4, 1, 1200)]
    for beta, th, Rt in sched:
        for g in runs:
            g.step(beta, th, R_target=Rt)
        c.step(beta, th, Rt)
        for g in runs:
            assert_same_state(g, c, f"beta {beta} target {Rt}")
    # a zero-width step: Q' = R~ exactly, ln Q = 0 (Eq. (2) with beta' = beta)
    for g in runs:
        g.step(1.4, 1)
    c.step(1.4, 1, 800)
    assert runs[0].observables()["lnQ_last"] == 0.0 and c.state().lnQ_last == 0.0
    assert_same_state(runs[0], c, "zero step")


def test_device_detected_errors_leave_state_untouched():
    J = inputs.couplings_3d(4, 0, 1)
    g = pa.Run(J, 4, 3, 100, 3, R_cap=300)
    g.step(0.1, 1, R_target=100)
    before = g.observables()
    g.step(0.2, 1, R_target=100000)  # population far above R_cap
    with pytest.raises(pa.PAError) as e:
        g.sync()
    assert e.value.code == pa.PA_ERR_CAPACITY
    lib = pa.load()
    obs = pa.Obs()
    assert lib.pa_observables(g._h, obs) == pa.PA_ERR_CAPACITY
    assert obs.step == before["step"] and obs.R == before["R"]
    assert obs.minus_beta_F == before["minus_beta_F"] and obs.sumE == before["sumE"]
    # the error is sticky: later steps do nothing
    g.step(0.3, 1, R_target=100)
    assert lib.pa_observables(g._h, obs) == pa.PA_ERR_CAPACITY and obs.step == before["step"]
    # extinction happens for exactly the seeds where the oracle dies out
    for s in range(1, 25):
        gg = pa.Run(J, 4, 3, 4, s)
        gg.step(0.2, 1, R_target=1)
        cc = o.Run(J, 3, 4, 4, 4, 7, R0=4, seed=s)
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


def test_host_detected_errors():
    J = inputs.couplings_3d(4, 0, 1)
    g = pa.Run(J, 4, 3, 50, 1)
    g.step(0.5, 1)
    with pytest.raises(pa.PAError) as e:
        g.step(0.4, 1)  # beta must not decrease
    assert e.value.code == pa.PA_ERR_INVALID
    with pytest.raises(pa.PAError) as e:
        g.step(0.6, -1)
    assert e.value.code == pa.PA_ERR_INVALID
    g.sync()  # nothing was queued by the refused calls
    assert g.observables()["step"] == 1
    with pytest.raises(pa.PAError) as e:
        pa.Run(inputs.couplings_lattice(5, 5, 5), 5, 3, 10, 1)
    assert e.value.code == pa.PA_ERR_INVALID
    with pytest.raises(pa.PAError) as e:
        pa.Run(inputs.couplings_3d(18), 18, 3, 10, 1)
    assert e.value.code == pa.PA_ERR_UNSUPPORTED
    Jz = J.copy()
    Jz[0, 0] = 0
    with pytest.raises(pa.PAError) as e:
        pa.Run(Jz, 4, 3, 10, 1)
    assert e.value.code == pa.PA_ERR_INVALID
    Jc = inputs.couplings_chain(33, open_chain=False)
    with pytest.raises(pa.PAError) as e:
        pa.Run(Jc, 33, 1, 10, 1)  # odd periodic chain
    assert e.value.code == pa.PA_ERR_INVALID


def test_walk_division_matches_the_division_instruction():
    """The Poisson walk divides P_{k-1} a by k with an integer-arithmetic
    division; bit for bit the same as the correctly rounded division
    instruction on 2^26 pairs per seed (every exponent class, k = 1..512)."""
    for seed in (0, 1, 2):
        assert pa.pa_check_division(1 << 26, seed) == 0
    assert pa.pa_check_division(0) == 0
    with pytest.raises(pa.PAError):
        pa.pa_check_division(-1)


def test_kernel_timing_hook_counts_sampled_launches():
    """pa_kernel_time: every k-th sweep launch timed, all kernels counted
    (six per +-1 step: prepare, copies, scan, scatter, sweep, commit)."""
    J = inputs.couplings_3d(6, 0, 1)
    r = pa.Run(J, 6, 3, 3000, 1)
    beta = 0.0
    for every, want in ((1, 8), (4, 2), (3, 3)):
        pa.pa_kernel_time(r._h, True, every)
        for k in range(8):
            beta += 0.05
            r.step(beta, 2)
        ms, n, launches = pa.pa_kernel_time(r._h, False)
        assert n == want and launches == 6 * 8 and ms > 0.0, (every, n, launches, ms)
    with pytest.raises(pa.PAError):
        pa.pa_kernel_time(r._h, True, -1)
    r.close()


def test_run_schedule_equals_steps_with_and_without_graph():
    """pa_run_schedule (one graph or step by step, then replayed after
    pa_reset) gives the bits of the same steps taken one pa_step_target at a
    time; a bad schedule is refused before any work."""
    J = inputs.couplings_3d(8, 1, 1)
    betas = inputs.linear_schedule(3.0, 25)[1:]
    thetas = np.array([2 + (k % 3) for k in range(24)])
    targets = np.array([4000 + 50 * k for k in range(24)])
    ref = pa.Run(J, 8, 3, 4000, 9, R_cap=6000)
    for k in range(24):
        ref.step(float(betas[k]), int(thetas[k]), R_target=int(targets[k]))
    want = (ref.trajectory(), ref.spins(), ref.energies())
    for use_graph in (False, True):
        r = pa.Run(J, 8, 3, 4000, 9, R_cap=6000)
        for rep in range(2):  # the second pass replays the kept graph
            if rep:
                r.reset(9)
            r.run_schedule(betas[:12], thetas[:12], targets[:12], use_graph=use_graph)
            r.run_schedule(betas[12:], thetas[12:], targets[12:], use_graph=use_graph)
            got = (r.trajectory(), r.spins(), r.energies())
            for key in want[0]:
                assert np.array_equal(want[0][key], got[0][key]), (use_graph, rep, key)
            assert np.array_equal(want[1], got[1]) and np.array_equal(want[2], got[2])
        before = r.observables()
        with pytest.raises(pa.PAError):
            r.run_schedule([3.5, 3.4])  # decreasing
        with pytest.raises(pa.PAError):
            r.run_schedule([3.5], R_targets=[0])
        assert r.observables() == before
        r.close()


def test_kernel_timing_inside_graph_replays():
    """Sweep timing of replayed graphs: the events captured with the graph
    are read after every replay, so each replay adds its sampled launches."""
    J = inputs.couplings_3d(6, 0, 1)
    r = pa.Run(J, 6, 3, 3000, 1)
    betas = np.linspace(0.1, 1.6, 16)
    pa.pa_kernel_time(r._h, True, 4)
    for rep in range(3):
        r.reset(rep + 1)
        r.run_schedule(betas, 2, use_graph=True)
        r.trajectory()
    ms, n, launches = pa.pa_kernel_time(r._h, False)
    assert n == 3 * 4 and ms > 0.0, (n, ms)
    assert launches == 3 * (4 + 6 * 16), launches  # init (4 kernels) + six per step
    r.close()


def test_exponentials_within_two_ulp_of_cuda():
    """The deterministic exp of the FP64 path and the float exp of the
    Gaussian acceptance stay within 2 ulp of CUDA's exp and expf (both are
    within about 1 ulp of the exact value: the oracle's pins against mpmath
    bound ours, CUDA documents its own)."""
    md, mf = pa.pa_check_exp(1 << 24, 3)
    assert md <= 2 and mf <= 2, (md, mf)


def test_philox_matches_curand():
    """The device Philox4x32-10 (both forms) equals cuRAND's Philox4_32_10
    generator on 2^22 seeded (seed, subsequence, offset) triples."""
    for seed in (0, 1):
        assert pa.pa_check_philox(1 << 22, seed) == 0
    with pytest.raises(pa.PAError):
        pa.pa_check_philox(-1)


def test_weighted_average_and_bootstrap_match_oracle():
    rng = np.random.default_rng(17)
    for M in (1, 2, 31, 64, 257):
        x = rng.normal(2500.0, 0.9, M)
        A = rng.normal(-600.0, 4.0, M)
        R = rng.integers(20000, 80000, M).astype(np.float64)
        for args in ((x, A, R), (x, A, None), (x, None, None)):
            gm, gf = pa.pa_weighted_average(*args)
            om, of = o.weighted_average(*args)
            assert close(gm, om) and close(gf, of), (M, gm, om, gf, of)
        if M >= 2:
            gs = pa.pa_bootstrap(x, A, R, B=64, seed=9)
            os_ = o.bootstrap(x, A, R, B=64, seed=9)
            assert close(gs[0], os_[0], 1e-9) and close(gs[1], os_[1], 1e-9)


def test_batch_graph_matches_oracle_and_standalone_runs():
    specs = [inputs.RunSpec(3, 4, 0, 1, 500, None, 3), inputs.RunSpec(3, 6, 1, 2, 700, None, 3),
             inputs.RunSpec(3, 4, 0, 3, 400, None, 3), inputs.RunSpec(1, 70, 2, 4, 300, None, 3),
             inputs.RunSpec(3, 8, 2, 5, 260, None, 3)]
    nst = 6
    betas = np.array([[0.1 * (k + 1) * (1 + 0.3 * r) for k in range(nst)] for r in range(len(specs))])
    for r, s in enumerate(specs):
        s.betas = np.concatenate([[0.0], betas[r]])
    b = pa.Batch(specs)
    b.run(betas[:, :3], thetas=3, use_graph=True)
    b.run(betas[:, 3:], thetas=3, use_graph=True)
    assert not b.sync().any()
    tr = b.trajectory(nst + 1)
    for r, s in enumerate(specs):
        J = s.couplings()
        if s.dim == 3:
            c = o.Run(J, 3, s.L, s.L, s.L, 7, R0=s.R0, R_cap=inputs.default_capacity(s.R0), seed=s.seed)
        else:
            c = o.Run(J, 1, s.L, R0=s.R0, R_cap=inputs.default_capacity(s.R0), seed=s.seed)
        alone = pa.Run(J, s.L, s.dim, s.R0, s.seed)
        for k in range(nst):
            c.step(float(betas[r, k]), 3, s.R0)
            alone.step(float(betas[r, k]), 3)
            st = c.state()
            assert tr["R"][r, k + 1] == st.R and tr["sumE"][r, k + 1] == st.sumE
            assert close(tr["minus_beta_F"][r, k + 1], st.minus_beta_F)
        sp = b.spins(r, c.state().R)
        assert np.array_equal(sp, c.spins())
        assert np.array_equal(sp, alone.spins())  # same result alone and in the batch


def test_pair_weighted_overlap_matches_oracle():
    """Gamma of Sec. 4 from pairs of runs, weighted by Eq. (11)."""
    J = inputs.couplings_3d(4, 2, 1)
    betas = [0.3, 0.8, 1.5]
    x1, x2, gam = [], [], []
    ox1, ox2, ogam = [], [], []
    for p in range(4):
        a, ca = make_pair(J, 4, 3, 400, 100 + 2 * p)
        b, cb = make_pair(J, 4, 3, 400, 101 + 2 * p)
        for beta in betas:
            for g, c in ((a, ca), (b, cb)):
                g.step(beta, 3)
                c.step(beta, 3, 400)
        x1.append(a.free_energy()); x2.append(b.free_energy())
        gam.append(pa.overlap(a, b)[0])
        ox1.append(ca.state().minus_beta_F); ox2.append(cb.state().minus_beta_F)
        ogam.append(o.overlap(ca, cb)[0])
    assert gam == ogam
    got = pa.pair_weighted_average(x1, x2, gam)
    want, _ = o.weighted_average_pairs(ox1, ox2, ogam)
    assert close(got, want)


def test_pair_weighted_average_matches_oracle():
    """Eqs. (10)-(11) through the C ABI: pair weights e^{x1 + x2} (times R1 R2),
    host and device-array forms, against the oracle at 1e-12."""
    rng = np.random.default_rng(29)
    for M in (1, 2, 31, 64, 257):
        x1 = rng.normal(2500.0, 0.9, M)
        x2 = rng.normal(2490.0, 0.9, M)
        G = rng.uniform(0.0, 0.4, M)
        R1 = rng.integers(1000, 3000, M).astype(np.float64)
        R2 = rng.integers(1000, 3000, M).astype(np.float64)
        for args in ((x1, x2, G, R1, R2), (x1, x2, G, None, None), (x1, x2, None, None, None)):
            gm, gf = pa.pa_weighted_average_pairs(*args)
            om, of = o.weighted_average_pairs(*args)
            assert close(gm, om) and close(gf, of), (M, gm, om, gf, of)
    # device form: G = 3 groups of M = 40 pairs in one launch
    torch = pytest.importorskip("torch")
    Gn, M = 3, 40
    x1 = rng.normal(900.0, 0.5, (Gn, M))
    x2 = rng.normal(905.0, 0.5, (Gn, M))
    A = rng.normal(-50.0, 1.0, (Gn, M))
    R1 = rng.integers(500, 900, (Gn, M)).astype(np.float64)
    R2 = rng.integers(500, 900, (Gn, M)).astype(np.float64)
    dev = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (x1, x2, A, R1, R2)]
    mean = torch.zeros(Gn, dtype=torch.float64, device="cuda")
    fbar = torch.zeros(Gn, dtype=torch.float64, device="cuda")
    code = pa.load().pa_weighted_average_pairs_dev(Gn, M, *[d.data_ptr() for d in dev], mean.data_ptr(),
                                                   fbar.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert code == pa.PA_OK
    torch.cuda.synchronize()
    for g in range(Gn):
        om, of = o.weighted_average_pairs(x1[g], x2[g], A[g], R1[g], R2[g])
        assert close(mean[g].item(), om) and close(fbar[g].item(), of)
    # argument errors: one R array without the other, a non-positive R
    with pytest.raises(pa.PAError):
        pa.pa_weighted_average_pairs([0.0], [0.0], [1.0], [1.0], None)
    with pytest.raises(pa.PAError):
        pa.pa_weighted_average_pairs([0.0], [0.0], [1.0], [0.0], [1.0])


def test_large_temperature_steps_bit_exact():
    """A few large jumps in beta: low-energy replicas get Poisson means in the
    hundreds (many pieces, sampled by a whole block) and the population is
    dominated by few ancestors."""
    J = inputs.couplings_3d(6, 4, 1)
    g, c = make_pair(J, 6, 3, 3000, 9, R_cap=8000)
    for beta in (0.6, 1.8, 3.5, 3.5, 6.0):
        g.step(beta, 2)
        c.step(beta, 2, 3000)
        assert_same_state(g, c, f"beta {beta}")
