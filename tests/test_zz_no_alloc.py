"""pa_bootstrap_noalloc: the bootstrap for callers that cannot allocate
device memory (a process whose device memory belongs to another pool, a
latency-critical loop, a deployment with memory fixed at start-up).  It must
give the same standard deviations as the allocating pa_bootstrap, call after
call, while reusing one fixed device scratch array.  This file is collected
last so that a failure here stops a -x run only after every other test."""
import ctypes

import numpy as np
import pytest

from paper_1006_0252_gb300 import pa

pytestmark = pytest.mark.gpu


def _entry():
    f = pa.load().pa_bootstrap_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    return f


def _close(a, b, rtol=1e-9):
    return abs(a - b) <= rtol * max(abs(a), abs(b), 1e-300)


def test_noalloc_bootstrap_matches_allocating_bootstrap_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    f = _entry()
    rng = np.random.default_rng(23)
    stream = torch.cuda.current_stream()
    # the second call uses far fewer resamples than the first, so stale scratch
    # entries of the first call sit beyond what the second one reads
    for M, B, seed, with_R in ((257, 4096, 3, True), (64, 100, 9, False)):
        x = rng.normal(2800.0, 0.7, M)
        A = rng.normal(-700.0, 5.0, M)
        R = rng.integers(20000, 80000, M).astype(np.float64) if with_R else None
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        Ad = torch.tensor(A, dtype=torch.float64, device="cuda")
        Rd = torch.tensor(R, dtype=torch.float64, device="cuda") if with_R else None
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        code = f(M, xd.data_ptr(), Ad.data_ptr(), Rd.data_ptr() if with_R else None, B, seed,
                 out.data_ptr(), stream.cuda_stream)
        assert code == pa.PA_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = pa.pa_bootstrap(x, A, R, B=B, seed=seed)
        assert _close(got[0], want[0]) and _close(got[1], want[1]), (got, want)


def test_noalloc_bootstrap_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    f = _entry()
    xd = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert f(8, xd.data_ptr(), None, None, 4097, 1, out.data_ptr(), s) == pa.PA_ERR_INVALID
    assert f(8, xd.data_ptr(), None, None, 1, 1, out.data_ptr(), s) == pa.PA_ERR_INVALID
