"""Checkpoint and resume: a run restored from a checkpoint continues exactly
as the original (same spins, energies, population sizes and free energy at
every later step), and a checkpoint is refused by a run with other
couplings or too small a capacity."""
import numpy as np
import pytest

from paper_1006_0252_gb300 import inputs, pa

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,L,R0", [(3, 8, 3000), (3, 6, 2000), (1, 200, 1500)])
def test_restore_continues_bit_exactly(dim, L, R0):
    J = inputs.couplings_3d(L, 1, 1) if dim == 3 else inputs.couplings_chain(L, 1, 1)
    betas = inputs.linear_schedule(3.0, 31)
    a = pa.Run(J, L, dim, R0, 77)
    for k in range(1, 16):
        a.step(float(betas[k]), 3)
    blob = a.checkpoint()
    b = pa.Run(J, L, dim, R0, 12345)  # another seed: the checkpoint carries the run's own
    b.restore(blob)
    assert b.observables() == a.observables()
    for k in range(16, 31):
        a.step(float(betas[k]), 3)
        b.step(float(betas[k]), 3)
    assert b.observables() == a.observables()
    assert np.array_equal(a.spins(), b.spins()) and np.array_equal(a.energies(), b.energies())
    ta, tb = a.trajectory(), b.trajectory()
    for key in ta:
        assert np.array_equal(ta[key], tb[key]), key


def test_restore_refuses_mismatched_runs():
    J = inputs.couplings_3d(4, 0, 1)
    a = pa.Run(J, 4, 3, 500, 1)
    a.step(0.3, 2)
    blob = a.checkpoint()
    other = pa.Run(inputs.couplings_3d(4, 5, 1), 4, 3, 500, 1)
    with pytest.raises(pa.PAError) as e:
        other.restore(blob)
    assert e.value.code == pa.PA_ERR_INVALID
    small = pa.Run(J, 4, 3, 100, 1, R_cap=120)
    with pytest.raises(pa.PAError):
        small.restore(blob)
    with pytest.raises(pa.PAError):
        a.restore(blob[:100])


def batch_state(b, count):
    """Everything a batch reports: final counters, per-step records and
    every run's spins."""
    res, tr = b.results(), b.trajectory(count)
    spins = [b.spins(r, 100000) for r in range(b.n)]
    return res, tr, spins


def same_batch_state(x, y):
    for key in x[0]:
        assert np.array_equal(x[0][key], y[0][key]), key
    for key in x[1]:
        assert np.array_equal(x[1][key], y[1][key]), key
    for r, (s, t) in enumerate(zip(x[2], y[2])):
        assert np.array_equal(s, t), r


@pytest.mark.parametrize("gaussian", [False, True])
def test_batch_restore_continues_bit_exactly(gaussian):
    """A batch of mixed lattices (3D L = 4, 6 and a chain) checkpointed after
    10 of 20 steps: a fresh batch restored from it, and the original batch
    rewound to it, both finish exactly as the uninterrupted batch."""
    betas = inputs.linear_schedule(4.0, 21)
    specs = [inputs.RunSpec(3, 4, 0, 1, 700, betas, 3, gaussian=gaussian),
             inputs.RunSpec(3, 6, 1, 2, 1200, betas, 3, gaussian=gaussian),
             inputs.RunSpec(1, 96, 2, 3, 900, betas, 3, gaussian=gaussian),
             inputs.RunSpec(3, 4, 3, 4, 500, betas, 3, gaussian=gaussian)]
    a = pa.Batch(specs)
    a.run(betas[1:11], thetas=3, use_graph=True)
    assert not a.sync().any()
    blob = a.checkpoint()
    a.run(betas[11:], thetas=3, use_graph=True)
    assert not a.sync().any()
    want = batch_state(a, 21)

    b = pa.Batch(specs)
    b.restore(blob)
    b.run(betas[11:], thetas=3, use_graph=True)
    assert not b.sync().any()
    same_batch_state(batch_state(b, 21), want)

    a.restore(blob)  # rewind: the graph of 10 steps is replayed from step 10
    a.run(betas[11:], thetas=3, use_graph=True)
    assert not a.sync().any()
    same_batch_state(batch_state(a, 21), want)
    a.close()
    b.close()


def test_batch_restore_refusals_leave_the_batch_untouched():
    betas = inputs.linear_schedule(3.0, 9)
    specs = [inputs.RunSpec(3, 4, d, d + 1, 400, betas, 2) for d in range(3)]
    a = pa.Batch(specs)
    a.run(betas[1:5], thetas=2, use_graph=False)
    assert not a.sync().any()
    blob = a.checkpoint()

    other = [inputs.RunSpec(3, 4, d, d + 1, 400, betas, 2) for d in (0, 1, 7)]  # run 2: other couplings
    c = pa.Batch(other)
    c.run(betas[1:3], thetas=2, use_graph=False)
    assert not c.sync().any()
    before = batch_state(c, 3)
    with pytest.raises(pa.PAError) as e:
        c.restore(blob)
    assert e.value.code == pa.PA_ERR_INVALID
    same_batch_state(batch_state(c, 3), before)  # runs 0 and 1 were not loaded either

    with pytest.raises(pa.PAError):
        pa.Batch(specs[:2]).restore(blob)  # another number of runs
    with pytest.raises(pa.PAError):
        pa.Batch(specs).restore(blob[: len(blob) - 8])  # truncated
    single = pa.Run(inputs.couplings_3d(4, 0, 1), 4, 3, 400, 1)
    with pytest.raises(pa.PAError):
        pa.Batch(specs).restore(single.checkpoint())  # a single-run checkpoint
    with pytest.raises(pa.PAError):
        single.restore(blob)  # and the other way round
    a.close()
    c.close()


def test_batch_reset_replays_runs_with_new_seeds():
    """pa_batch_reset gives fresh populations: a reset batch run again with
    the seeds of another batch gives that batch's results bit for bit, with
    the schedule graph kept."""
    betas = inputs.linear_schedule(3.0, 9)
    specs = [inputs.RunSpec(3, 6, d, d + 1, 600, betas, 2) for d in range(3)]
    other = [inputs.RunSpec(3, 6, d, 40 + d, 600, betas, 2) for d in range(3)]
    a = pa.Batch(specs)
    a.run(betas[1:], thetas=2, use_graph=True)
    assert not a.sync().any()
    b = pa.Batch(other)
    b.run(betas[1:], thetas=2, use_graph=True)
    assert not b.sync().any()
    want = batch_state(b, 9)
    a.reset([s.seed for s in other])
    a.run(betas[1:], thetas=2, use_graph=True)
    assert not a.sync().any()
    same_batch_state(batch_state(a, 9), want)
    a.close()
    b.close()
