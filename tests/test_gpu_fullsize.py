"""Parity at the benchmark sizes, in the launch configuration the benchmark
times, on outputs the oracle can compute one at a time.

For a checked step the GPU's pre-step population is copied out; the oracle
recomputes every copy count, R~' and ln Q from the pre-step energies (all
replicas), and re-runs the sweeps of sampled new slots from their source
replicas (each with its own random stream); the GPU's post-step spins and
energies of those slots must match bit for bit.  Every replica's energy is
also checked against its spins with an independent numpy evaluation."""
import math

import numpy as np
import pytest

from oracle import oracle as o
from paper_1006_0252_gb300 import inputs, pa

pytestmark = pytest.mark.gpu


def close(a, b, rtol=1e-12):
    return abs(a - b) <= rtol * max(abs(a), abs(b), 1.0)


def energies_3d(sp: np.ndarray, J: np.ndarray, L: int) -> np.ndarray:
    s = sp.reshape(-1, L, L, L).astype(np.int32)  # axes (z, y, x)
    Jx, Jy, Jz = (J[d].reshape(L, L, L).astype(np.int32) for d in range(3))
    E = (Jx * s * np.roll(s, -1, axis=3)).sum(axis=(1, 2, 3))
    E += (Jy * s * np.roll(s, -1, axis=2)).sum(axis=(1, 2, 3))
    E += (Jz * s * np.roll(s, -1, axis=1)).sum(axis=(1, 2, 3))
    return E


def energies_chain(sp: np.ndarray, J: np.ndarray) -> np.ndarray:
    out = np.empty(len(sp), dtype=np.int64)
    Jc = J.astype(np.int16)[None, :]
    for a in range(0, len(sp), 8192):
        s = sp[a:a + 8192].astype(np.int16)
        out[a:a + 8192] = (Jc * s * np.roll(s, -1, axis=1)).sum(axis=1, dtype=np.int64)
    return out


def check_step(g, lat, beta_next, theta, R_target, energy_fn, rng, n_samples=40, n_last=0):
    pre = g.observables()
    pre_sp = g.spins()
    pre_E = g.energies()
    assert np.array_equal(energy_fn(pre_sp), pre_E)
    g.step(beta_next, theta, R_target=R_target)
    post = g.observables()
    copies, Rn, Qp, lnQ = lat.resample(pre_E, pre["beta"], beta_next, R_target, pre["step"])
    assert np.array_equal(g.copies(len(pre_E)), copies)
    assert post["R"] == Rn
    assert close(post["lnQ_last"], lnQ, 1e-11) or abs(post["lnQ_last"] - lnQ) < 1e-12
    assert close(post["minus_beta_F"], pre["minus_beta_F"] + lnQ)
    src = np.repeat(np.arange(len(pre_E)), copies)
    post_sp = g.spins()
    post_E = g.energies()
    assert np.array_equal(energy_fn(post_sp), post_E)
    assert int(post_E.astype(np.int64).sum()) == post["sumE"]
    # n_last more among the last 5000 slots: past the last whole wave of
    # resident threads, where the kernel may sweep a replica with 4 threads
    last = rng.integers(max(0, Rn - 5000), Rn, n_last)
    slots = np.unique(np.concatenate([[0, Rn - 1], rng.integers(0, Rn, n_samples), last]))
    for s in slots:
        sig, E = lat.sweep_replica(pre_sp[src[s]], int(s), pre["sweeps"], beta_next, theta)
        assert np.array_equal(post_sp[s], sig), s
        assert post_E[s] == E


def test_l8_full_size_sampled():
    spec = inputs.config_l8()
    J = spec.couplings()
    g = pa.Run(J, 8, 3, spec.R0, spec.seed)  # the benchmark's launch configuration
    lat = o.Run(J, 3, 8, 8, 8, 7, R0=1, R_cap=1, seed=spec.seed)
    rng = np.random.default_rng(1)
    efn = lambda sp: energies_3d(sp, J, 8)
    b = spec.betas
    check_step(g, lat, float(b[1]), spec.theta, spec.R0, efn, rng, n_last=200)
    check_step(g, lat, float(b[2]), spec.theta, spec.R0, efn, rng)
    for k in range(3, 100):
        g.step(float(b[k]), spec.theta)
    check_step(g, lat, float(b[100]), spec.theta, spec.R0, efn, rng)
    for k in range(101, 200):
        g.step(float(b[k]), spec.theta)
    check_step(g, lat, float(b[200]), spec.theta, spec.R0, efn, rng)
    tr = g.trajectory()
    assert len(tr["R"]) == 201 and np.all(np.abs(tr["R"][1:] - spec.R0) < 10 * math.sqrt(spec.R0))


def test_l12_wave_tail_sampled():
    """L = 12 with a population just above one wave of resident threads (the
    tail swept 4 threads per replica): sampled slots, most of them in the
    tail, against the oracle."""
    J = inputs.couplings_3d(12, 0, 1)
    g = pa.Run(J, 12, 3, 80000, 5)
    lat = o.Run(J, 3, 12, 12, 12, 7, R0=1, R_cap=1, seed=5)
    rng = np.random.default_rng(4)
    efn = lambda sp: energies_3d(sp, J, 12)
    check_step(g, lat, 0.3, 4, 80000, efn, rng, 8, n_last=60)
    g.step(0.6, 4)
    check_step(g, lat, 0.9, 4, 81000, efn, rng, 8, n_last=60)


def test_chain_full_size_sampled():
    spec = inputs.config_chain(1)[0]
    J = spec.couplings()
    g = pa.Run(J, spec.L, 1, spec.R0, spec.seed)
    lat = o.Run(J, 1, spec.L, R0=1, R_cap=1, seed=spec.seed)
    rng = np.random.default_rng(2)
    efn = lambda sp: energies_chain(sp, J)
    b = spec.betas
    check_step(g, lat, float(b[1]), spec.theta, spec.R0, efn, rng, 12)
    for k in range(2, 200):
        g.step(float(b[k]), spec.theta)
    check_step(g, lat, float(b[200]), spec.theta, spec.R0, efn, rng, 12)


def _whole_schedule(spec, R0, spin_every):
    """Every step of spec's schedule at population R0, GPU (the benchmark's
    launch shape) against the oracle: R~, the exact energy sums, -beta F~ and
    ln Q every step, all spins and energies every `spin_every` steps."""
    J = spec.couplings()
    cap = inputs.default_capacity(R0)
    g = pa.Run(J, spec.L, spec.dim, R0, spec.seed, R_cap=cap)
    if spec.dim == 3:
        c = o.Run(J, 3, spec.L, spec.L, spec.L, 7, R0=R0, R_cap=cap, seed=spec.seed)
    else:
        c = o.Run(J, 1, spec.L, R0=R0, R_cap=cap, seed=spec.seed)
    b = spec.betas
    for k in range(1, len(b)):
        g.step(float(b[k]), spec.theta)
        c.step(float(b[k]), spec.theta, R0)
        go, co = g.observables(), c.state()
        assert go["R"] == co.R and go["sumE"] == co.sumE and go["sumE2"] == co.sumE2, k
        assert close(go["minus_beta_F"], co.minus_beta_F), (k, go["minus_beta_F"], co.minus_beta_F)
        assert close(go["lnQ_last"], co.lnQ_last, 1e-11) or abs(go["lnQ_last"] - co.lnQ_last) < 1e-12, k
        if k % spin_every == 0 or k == len(b) - 1:
            assert np.array_equal(g.energies(), c.energies()), k
            assert np.array_equal(g.spins(), c.spins()), k


def test_l8_whole_schedule_at_r2000():
    """The benchmark workload's schedule (3D L=8, couplings seed 1, 201 betas
    0..5, theta = 10), all 200 steps at R0 = 2000, bit for bit."""
    _whole_schedule(inputs.config_l8(), 2000, 50)


def test_chain_whole_schedule_small_population():
    """The open-chain workload's schedule (N = 4096, 401 betas 0..4, theta = 5,
    eight threads per replica), all 400 steps at R0 = 150, bit for bit."""
    _whole_schedule(inputs.config_chain(1)[0], 150, 100)


def test_batched_mix_matches_runs_alone():
    """Mixed L in {6, 8, 10}, R0 in [2e4, 8e4], one autotuned graph launch per
    schedule segment: every run is bit-identical to the same run alone."""
    specs = inputs.config_batched(n_real=3, runs_per_real=2)
    b = pa.Batch(specs)
    b.autotune()
    betas = specs[0].betas
    b.run(betas[1:4], thetas=10, use_graph=True)
    b.run(betas[4:7], thetas=10, use_graph=True)
    assert not b.sync().any()
    tr = b.trajectory(7)
    rng = np.random.default_rng(3)
    for r, s in enumerate(specs):
        J = s.couplings()
        alone = pa.Run(J, s.L, 3, s.R0, s.seed)
        if r % 2 == 0:  # oracle-checked first step of one run per lattice size
            lat = o.Run(J, 3, s.L, s.L, s.L, 7, R0=1, R_cap=1, seed=s.seed)
            check_step(alone, lat, float(betas[1]), 10, s.R0, lambda sp: energies_3d(sp, J, s.L), rng, 16)
            start = 2
        else:
            start = 1
        for k in range(start, 7):
            alone.step(float(betas[k]), 10)
        ta = alone.trajectory()
        assert np.array_equal(ta["R"], tr["R"][r]) and np.array_equal(ta["sumE"], tr["sumE"][r])
        assert np.array_equal(ta["minus_beta_F"], tr["minus_beta_F"][r])
        assert np.array_equal(alone.spins(), b.spins(r, s.R0 * 2))
        alone.close()
