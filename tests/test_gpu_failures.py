"""Failure handling injected on the host, never by faulting the GPU: an
allocator hook that refuses one chosen allocation (run creation, batch
creation, a scratch buffer of a live run, server admission), and request
cancellation in the server.  Each refusal must surface as PA_ERR_OOM (or a
queued request), leak nothing, leave the handle's state untouched, and let
later calls work; cancelling one served request must leave the results of the
others bit for bit the same."""
import ctypes

import numpy as np
import pytest

from paper_1006_0252_gb300 import inputs, pa

pytestmark = pytest.mark.gpu


class RefusingAllocator:
    """Routes device memory to PyTorch's caching allocator, counting calls;
    refuses the calls whose 1-based index is in `refuse` (a set, changeable)."""

    def __init__(self, torch, refuse=()):
        self.torch = torch
        self.calls = 0
        self.refuse = set(refuse)
        self.live = {}

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls in self.refuse:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, nbytes, stream, ctx):
            self.live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

        self._fa = pa.ALLOC_FN(_alloc)
        self._ff = pa.FREE_FN(_free)

    def opts(self, max_steps=0):
        o = pa.Opts()
        o.alloc, o.free = self._fa, self._ff
        s = self.torch.cuda.current_stream().cuda_stream
        o.stream = s if s else None
        o.max_steps = max_steps
        return o


def _torch():
    return pytest.importorskip("torch")


def _create(J, L, R0, seed, opts):
    h = ctypes.c_void_p()
    Jc = np.ascontiguousarray(J, dtype=np.int8)
    code = pa.load().pa_create_ex(Jc.ctypes.data_as(ctypes.c_void_p), L, 3, R0, seed, ctypes.byref(opts),
                                  ctypes.byref(h))
    return code, h


def test_run_creation_refused_at_every_allocation():
    torch = _torch()
    J = inputs.couplings_3d(6, 1, 1)
    probe = RefusingAllocator(torch)
    code, h = _create(J, 6, 700, 5, probe.opts())
    assert code == pa.PA_OK
    n_allocs = probe.calls
    pa.load().pa_destroy(h)
    torch.cuda.synchronize()
    assert n_allocs >= 2 and not probe.live
    for k in range(1, n_allocs + 1):
        a = RefusingAllocator(torch, refuse={k})
        code, h = _create(J, 6, 700, 5, a.opts())
        torch.cuda.synchronize()
        assert code == pa.PA_ERR_OOM, (k, code)
        assert not h.value
        assert not a.live, f"refusal at allocation {k} leaked {len(a.live)} buffers"
    # later calls work and give the run everyone else gets
    ok = RefusingAllocator(torch)
    code, h = _create(J, 6, 700, 5, ok.opts())
    assert code == pa.PA_OK
    ref = pa.Run(J, 6, 3, 700, 5)
    for beta in (0.4, 0.9):
        assert pa.load().pa_step(h, beta, 2) == pa.PA_OK
        ref.step(beta, 2)
    obs = pa.Obs()
    assert pa.load().pa_observables(h, ctypes.byref(obs)) == pa.PA_OK
    assert obs.R == ref.observables()["R"] and obs.sumE == ref.observables()["sumE"]
    pa.load().pa_destroy(h)
    torch.cuda.synchronize()
    assert not ok.live


def test_batch_creation_refused_at_every_allocation():
    torch = _torch()
    specs = [inputs.RunSpec(3, 4, 0, 1, 300, None, 2), inputs.RunSpec(3, 6, 1, 2, 400, None, 2),
             inputs.RunSpec(1, 64, 2, 3, 200, None, 2)]
    probe = RefusingAllocator(torch)
    pa.Batch(specs, opts=probe.opts()).close()
    n_allocs = probe.calls
    torch.cuda.synchronize()
    assert n_allocs >= 2 and not probe.live
    for k in range(1, n_allocs + 1):
        a = RefusingAllocator(torch, refuse={k})
        with pytest.raises(pa.PAError) as err:
            pa.Batch(specs, opts=a.opts())
        torch.cuda.synchronize()
        assert err.value.code == pa.PA_ERR_OOM, (k, err.value)
        assert not a.live, f"refusal at allocation {k} leaked {len(a.live)} buffers"


def test_scratch_refusal_leaves_the_run_untouched():
    """pa_copy_spins takes a scratch buffer from the allocator: refused, it
    reports PA_ERR_OOM and the run continues exactly like a twin that never
    saw the refusal."""
    torch = _torch()
    J = inputs.couplings_3d(4, 2, 1)
    a = RefusingAllocator(torch)
    code, h = _create(J, 4, 500, 9, a.opts())
    assert code == pa.PA_OK
    twin = pa.Run(J, 4, 3, 500, 9)
    L = pa.load()
    assert L.pa_step(h, 0.5, 2) == pa.PA_OK
    twin.step(0.5, 2)
    a.refuse = {a.calls + 1}
    buf = np.empty((600, 64), dtype=np.int8)
    n = ctypes.c_int64()
    code = L.pa_copy_spins(h, buf.ctypes.data_as(ctypes.c_void_p), 600, ctypes.byref(n))
    assert code == pa.PA_ERR_OOM
    a.refuse = set()
    for beta in (1.0, 1.7):
        assert L.pa_step(h, beta, 3) == pa.PA_OK
        twin.step(beta, 3)
    assert L.pa_copy_spins(h, buf.ctypes.data_as(ctypes.c_void_p), 600, ctypes.byref(n)) == pa.PA_OK
    assert np.array_equal(buf[: n.value], twin.spins())
    L.pa_destroy(h)
    torch.cuda.synchronize()
    assert not a.live


def _req(k, L=6, R0=900, nb=6, theta=2):
    J = inputs.couplings_3d(L, 10 + k, 1)
    betas = inputs.linear_schedule(0.25 * nb, nb + 1)[1:]
    return dict(L=L, J=J, R0=R0, seed=700 + k, betas=betas, theta=theta)


def _alone(q):
    r = pa.Run(q["J"], q["L"], 3, q["R0"], q["seed"])
    for b in q["betas"]:
        r.step(float(b), q["theta"])
    return r.observables()


def test_server_admission_refused_then_admitted():
    """A refused admission keeps the request queued; once memory comes back
    the request runs and gives the result of the same run alone."""
    torch = _torch()
    a = RefusingAllocator(torch)
    srv = pa.Server(max_runs=4, opts=a.opts())
    q = _req(0)
    rid = srv.submit(3, q["L"], q["J"], q["R0"], q["seed"], q["betas"], q["theta"])
    a.refuse = {a.calls + 1}  # the run's slab, requested by the first tick
    act, qd, fin = srv.tick(1)
    assert act == 0 and qd == 1 and srv.result(rid)["status"] == 0
    assert srv.memory()["used_bytes"] == 0
    a.refuse = set()
    while True:
        act, qd, fin = srv.tick(3)
        if act == 0 and qd == 0:
            break
    res = srv.result(rid)
    want = _alone(q)
    assert res["status"] == 2
    assert res["R"] == want["R"] and res["sumE"] == want["sumE"] and res["minus_beta_F"] == want["minus_beta_F"]
    srv.close()
    torch.cuda.synchronize()
    assert not a.live


def test_server_cancel_releases_memory_and_spares_the_others():
    srv = pa.Server(max_runs=3)
    reqs = [_req(k, R0=600 + 100 * k) for k in range(5)]
    ids = [srv.submit(3, q["L"], q["J"], q["R0"], q["seed"], q["betas"], q["theta"]) for q in reqs]
    srv.tick(2)  # three admitted, two queued
    mem = srv.memory()
    assert mem["runs_resident"] == 3
    running = [i for i in ids if srv.result(i)["status"] == 1]
    queued = [i for i in ids if srv.result(i)["status"] == 0]
    assert len(running) == 3 and len(queued) == 2
    srv.cancel(running[1])
    srv.cancel(queued[0])
    after = srv.memory()
    assert after["runs_resident"] == 2 and after["used_bytes"] < mem["used_bytes"]
    for c in (running[1], queued[0]):
        assert srv.result(c)["status"] == 4
    srv.cancel(running[1])  # a second cancel is a no-op
    with pytest.raises(pa.PAError):
        srv.cancel(10 ** 9)
    while True:
        act, qd, fin = srv.tick(2)
        if act == 0 and qd == 0:
            break
    assert srv.memory()["used_bytes"] == 0
    for q, i in zip(reqs, ids):
        res = srv.result(i)
        if i in (running[1], queued[0]):
            assert res["status"] == 4
            continue
        want = _alone(q)
        assert res["status"] == 2
        assert res["R"] == want["R"] and res["sumE"] == want["sumE"] and res["sumE2"] == want["sumE2"]
        assert res["minus_beta_F"] == want["minus_beta_F"]
    srv.close()
