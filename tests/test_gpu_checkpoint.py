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
