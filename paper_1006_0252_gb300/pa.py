"""Python binding of the C ABI in include/pa.h (argument marshalling only).

Every function named pa_* here calls the entry point of the same name in
``libpa_gb300.so``; the classes Run and Batch are conveniences on top of
them.  Device memory comes from PyTorch's caching allocator and work is
queued on PyTorch's current stream when PyTorch with CUDA is available.
There is no CPU path: if the CUDA library cannot be built or loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_size_t, c_uint64, c_void_p

import numpy as np

from . import build as _build

PA_OK = 0
PA_ERR_INVALID = 1
PA_ERR_OOM = 2
PA_ERR_CAPACITY = 3
PA_ERR_EXTINCT = 4
PA_ERR_TIMEOUT = 5
PA_ERR_CUDA = 6
PA_ERR_UNSUPPORTED = 7


class PAError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: error {code}: {msg}")
        self.code = code


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class Opts(ctypes.Structure):
    _fields_ = [("R_cap", c_int64), ("stream", c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", c_void_p), ("max_steps", c_int32),
                ("threads_per_block", c_int32), ("threads_per_replica", c_int32)]


class Obs(ctypes.Structure):
    _fields_ = [("beta", c_double), ("R", c_int64), ("E_mean", c_double), ("E2_mean", c_double),
                ("lnQ_last", c_double), ("minus_beta_F", c_double), ("step", c_int64),
                ("sweeps", c_int64), ("sumE", c_int64), ("sumE2", c_int64)]


class RequestC(ctypes.Structure):
    _fields_ = [("dim", c_int32), ("L", c_int32), ("couplings", c_void_p), ("R0", c_int64),
                ("seed", c_uint64), ("n_steps", c_int32), ("theta", c_int32), ("betas", c_void_p)]


class ResultC(ctypes.Structure):
    _fields_ = [("status", c_int32), ("error", c_int32), ("steps", c_int64), ("R", c_int64),
                ("beta", c_double), ("minus_beta_F", c_double), ("E_mean", c_double),
                ("sumE", c_int64), ("sumE2", c_int64), ("submit_s", c_double), ("admit_s", c_double),
                ("done_s", c_double), ("device_bytes", c_int64), ("flips", c_int64)]


class RunSpecC(ctypes.Structure):
    _fields_ = [("dim", c_int32), ("L", c_int32), ("couplings", c_void_p), ("R0", c_int64),
                ("seed", c_uint64), ("R_cap", c_int64), ("gauss_couplings", c_void_p),
                ("Ls", c_int32 * 3), ("periodic_mask", ctypes.c_uint32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True) -> ctypes.CDLL:
    """Load libpa_gb300.so (building it in-tree first if sources changed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale:
        _build.build_library()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    P = POINTER
    sig = {
        "pa_version": (c_int, []),
        "pa_last_error": (ctypes.c_char_p, []),
        "pa_create": (c_int, [c_void_p, c_int, c_int, c_int64, c_uint64, P(c_void_p)]),
        "pa_create_ex": (c_int, [c_void_p, c_int, c_int, c_int64, c_uint64, P(Opts), P(c_void_p)]),
        "pa_create_gauss": (c_int, [c_void_p, c_int, c_int, c_int64, c_uint64, P(Opts), P(c_void_p)]),
        "pa_create_lattice": (c_int, [c_void_p, c_void_p, c_int, ctypes.c_uint, c_int64, c_uint64, P(Opts),
                                      P(c_void_p)]),
        "pa_create_lattice_gauss": (c_int, [c_void_p, c_void_p, c_int, ctypes.c_uint, c_int64, c_uint64,
                                            P(Opts), P(c_void_p)]),
        "pa_destroy": (None, [c_void_p]),
        "pa_check_division": (c_int, [c_int64, c_uint64, P(c_int64)]),
        "pa_check_philox": (c_int, [c_int64, c_uint64, P(c_int64)]),
        "pa_gauss_thresholds": (c_int, [c_double, c_int64, c_void_p, c_void_p]),
        "pa_check_exp": (c_int, [c_int64, c_uint64, P(c_int64), P(c_int64)]),
        "pa_reset": (c_int, [c_void_p, c_uint64]),
        "pa_kernel_time": (c_int, [c_void_p, c_int, P(c_double), P(c_int64), P(c_int64)]),
        "pa_sweep_shape": (c_int, [c_void_p, P(c_int32), P(c_int32)]),
        "pa_checkpoint_bytes": (c_int, [c_void_p, P(c_size_t)]),
        "pa_checkpoint": (c_int, [c_void_p, c_void_p, c_size_t]),
        "pa_restore": (c_int, [c_void_p, c_void_p, c_size_t]),
        "pa_step": (c_int, [c_void_p, c_double, c_int]),
        "pa_step_target": (c_int, [c_void_p, c_double, c_int, c_int64]),
        "pa_run_schedule": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int]),
        "pa_sync": (c_int, [c_void_p]),
        "pa_observables": (c_int, [c_void_p, P(Obs)]),
        "pa_free_energy": (c_int, [c_void_p, P(c_double)]),
        "pa_trajectory": (c_int, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p, P(c_int64)]),
        "pa_trajectory_energy": (c_int, [c_void_p, c_int64, c_void_p, c_void_p, P(c_int64)]),
        "pa_overlap": (c_int, [c_void_p, c_void_p, c_double, P(c_double), P(c_int64), c_void_p]),
        "pa_weighted_average": (c_int, [c_int, c_void_p, c_void_p, c_void_p, P(c_double),
                                        P(c_double)]),
        "pa_weighted_average_dev": (c_int, [c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p]),
        "pa_weighted_average_pairs": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                              P(c_double), P(c_double)]),
        "pa_weighted_average_pairs_dev": (c_int, [c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                                  c_void_p, c_void_p, c_void_p, c_void_p]),
        "pa_bootstrap": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_int, c_uint64,
                                 P(c_double), P(c_double)]),
        "pa_bootstrap_noalloc": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_int, c_uint64, c_void_p,
                                         c_void_p]),
        "pa_copy_spins": (c_int, [c_void_p, c_void_p, c_int64, P(c_int64)]),
        "pa_copy_energies": (c_int, [c_void_p, c_void_p, c_int64, P(c_int64)]),
        "pa_copy_copies": (c_int, [c_void_p, c_void_p, c_int64, P(c_int64)]),
        "pa_batch_create": (c_int, [c_int, P(RunSpecC), P(Opts), P(c_void_p)]),
        "pa_batch_destroy": (None, [c_void_p]),
        "pa_batch_run": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p, c_int]),
        "pa_batch_sync": (c_int, [c_void_p, c_void_p]),
        "pa_batch_results": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p]),
        "pa_batch_trajectory": (c_int, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p,
                                        c_void_p]),
        "pa_batch_energy": (c_int, [c_void_p, c_int64, c_void_p, c_void_p]),
        "pa_batch_diagnostics": (c_int, [c_void_p, c_int, c_int64, c_void_p, c_void_p, c_void_p]),
        "pa_batch_bootstrap": (c_int, [c_void_p, c_int, c_int64, c_int, c_uint64, c_void_p, c_void_p]),
        "pa_batch_overlap": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_void_p, c_void_p]),
        "pa_batch_overlap_hist": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
        "pa_batch_autotune": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, P(c_int)]),
        "pa_batch_reset": (c_int, [c_void_p, c_void_p]),
        "pa_batch_copy_spins": (c_int, [c_void_p, c_int, c_void_p, c_int64, P(c_int64)]),
        "pa_batch_checkpoint_bytes": (c_int, [c_void_p, P(c_size_t)]),
        "pa_batch_checkpoint": (c_int, [c_void_p, c_void_p, c_size_t]),
        "pa_batch_restore": (c_int, [c_void_p, c_void_p, c_size_t]),
        "pa_server_create": (c_int, [P(Opts), c_double, c_int, P(c_void_p)]),
        "pa_server_destroy": (None, [c_void_p]),
        "pa_server_submit": (c_int, [c_void_p, P(RequestC), P(c_int64)]),
        "pa_server_cancel": (c_int, [c_void_p, c_int64]),
        "pa_server_memory": (c_int, [c_void_p, P(c_int64), P(c_int64), P(c_int32)]),
        "pa_server_tick": (c_int, [c_void_p, c_int, P(c_int32), P(c_int32), P(c_int32)]),
        "pa_server_result": (c_int, [c_void_p, c_int64, P(ResultC), c_void_p, c_int64]),
        "pa_server_clock": (c_double, [c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(code: int, where: str):
    if code != PA_OK:
        msg = load().pa_last_error().decode(errors="replace")
        raise PAError(code, where, msg)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(c_void_p)


# ---- PyTorch plumbing: caching allocator and current stream ---------------------------

_torch_hooks = None


def _torch():
    try:
        import torch
        if torch.cuda.is_available():
            return torch
    except ImportError:
        pass
    return None


def torch_opts(R_cap: int = 0, max_steps: int = 0, threads_per_block: int = 0,
               threads_per_replica: int = 0) -> Opts:
    """Options routing device memory to PyTorch's caching allocator and work to
    PyTorch's current stream (library defaults when PyTorch has no CUDA)."""
    global _torch_hooks
    o = Opts()
    o.R_cap = R_cap
    o.max_steps = max_steps
    o.threads_per_block = threads_per_block
    o.threads_per_replica = threads_per_replica
    torch = _torch()
    if torch is None:
        o.alloc = ALLOC_FN()
        o.free = FREE_FN()
        o.stream = None
        return o
    if _torch_hooks is None:
        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          int(stream or 0))
            except Exception:
                return None

        def _free(ptr, nbytes, stream, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        _torch_hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    o.alloc, o.free = _torch_hooks
    s = torch.cuda.current_stream().cuda_stream
    o.stream = s if s else None
    return o


# ---- C-ABI mirror -----------------------------------------------------------------------

def pa_version() -> int:
    return load().pa_version()


def pa_last_error() -> str:
    return load().pa_last_error().decode(errors="replace")


def pa_create(couplings: np.ndarray, L: int, dim: int, R0: int, seed: int,
              opts: Opts | None = None) -> c_void_p:
    J = np.ascontiguousarray(couplings, dtype=np.int8)
    h = c_void_p()
    if opts is None:
        _check(load().pa_create(_ptr(J), L, dim, R0, seed, ctypes.byref(h)), "pa_create")
    else:
        _check(load().pa_create_ex(_ptr(J), L, dim, R0, seed, ctypes.byref(opts), ctypes.byref(h)),
               "pa_create_ex")
    return h


def pa_create_gauss(couplings: np.ndarray, L: int, dim: int, R0: int, seed: int,
                    opts: Opts | None = None) -> c_void_p:
    """Gaussian couplings as int32 J_q (J = J_q 2^-15), 3D layout [3][L^3]."""
    J = np.ascontiguousarray(couplings, dtype=np.int32)
    h = c_void_p()
    _check(load().pa_create_gauss(_ptr(J), L, dim, R0, seed,
                                  ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)),
           "pa_create_gauss")
    return h


def pa_create_lattice(couplings: np.ndarray, Ls, dim: int, periodic_mask: int, R0: int, seed: int,
                      opts: Opts | None = None, gaussian: bool = False) -> c_void_p:
    """General box Ls[0] x Ls[1] x Ls[2] (dim 3) or chain of Ls[0] spins (dim 1)
    with the periodic axes of periodic_mask; int8 (+-1) or int32 (Gaussian) couplings."""
    J = np.ascontiguousarray(couplings, dtype=np.int32 if gaussian else np.int8)
    ext = (c_int * 3)(*[int(v) for v in (list(Ls) + [1, 1, 1])[:3]])
    h = c_void_p()
    fn = load().pa_create_lattice_gauss if gaussian else load().pa_create_lattice
    name = "pa_create_lattice_gauss" if gaussian else "pa_create_lattice"
    _check(fn(_ptr(J), ext, dim, periodic_mask, R0, seed, ctypes.byref(opts) if opts is not None else None,
              ctypes.byref(h)), name)
    return h


def pa_destroy(h):
    load().pa_destroy(h)


def pa_check_division(n: int, seed: int = 0) -> int:
    """Pairs (x, k) on which the Poisson walk's integer division differs from
    the hardware division (pa_check_division); 0 when they agree."""
    bad = c_int64()
    _check(load().pa_check_division(n, seed, ctypes.byref(bad)), "pa_check_division")
    return bad.value


def pa_check_exp(n: int, seed: int = 0):
    """(max ulp of the double exp, max ulp of the float exp) from CUDA's exp
    and expf (pa_check_exp)."""
    d, f = c_int64(), c_int64()
    _check(load().pa_check_exp(n, seed, ctypes.byref(d), ctypes.byref(f)), "pa_check_exp")
    return d.value, f.value


def pa_check_philox(n: int, seed: int = 0) -> int:
    """Triples on which the library's Philox differs from cuRAND's
    (pa_check_philox); 0 when they agree."""
    bad = c_int64()
    _check(load().pa_check_philox(n, seed, ctypes.byref(bad)), "pa_check_philox")
    return bad.value


def gauss_thresholds(beta: float, dE) -> np.ndarray:
    """Integer acceptance thresholds of the Gaussian decision for each energy
    change (pa_gauss_thresholds): accept iff (u >> 8) < thr."""
    d = np.ascontiguousarray(dE, dtype=np.int32)
    out = np.empty(d.shape, dtype=np.uint32)
    _check(load().pa_gauss_thresholds(float(beta), d.size, d.ctypes.data_as(c_void_p),
                                      out.ctypes.data_as(c_void_p)), "pa_gauss_thresholds")
    return out


def pa_reset(h, seed: int):
    _check(load().pa_reset(h, seed), "pa_reset")


def pa_checkpoint(h) -> bytes:
    n = c_size_t()
    _check(load().pa_checkpoint_bytes(h, ctypes.byref(n)), "pa_checkpoint_bytes")
    buf = ctypes.create_string_buffer(n.value)
    _check(load().pa_checkpoint(h, buf, n.value), "pa_checkpoint")
    return buf.raw


def pa_restore(h, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().pa_restore(h, buf, len(blob)), "pa_restore")


def pa_kernel_time(h, enable, every: int = 1):
    """enable: start timing every `every`-th sweep launch; disable: return
    (timed sweep milliseconds, timed sweep launches, kernels launched)."""
    ms, n, k = c_double(), c_int64(), c_int64()
    _check(load().pa_kernel_time(h, int(every) if enable else 0, ctypes.byref(ms), ctypes.byref(n),
                                 ctypes.byref(k)), "pa_kernel_time")
    return ms.value, n.value, k.value


def pa_sweep_shape(h):
    """(threads per block, threads per replica) of the run's sweep kernel."""
    tpb, split = c_int32(), c_int32()
    _check(load().pa_sweep_shape(h, ctypes.byref(tpb), ctypes.byref(split)), "pa_sweep_shape")
    return tpb.value, split.value


def pa_step(h, beta_next: float, sweeps: int):
    _check(load().pa_step(h, beta_next, sweeps), "pa_step")


def pa_run_schedule(h, betas, thetas=None, R_targets=None, use_graph: bool = True):
    """The next len(betas) steps at once (pa_run_schedule); the arrays are
    returned so the caller can keep them alive until the call has copied
    them (it does so before returning)."""
    b = np.ascontiguousarray(betas, dtype=np.float64)
    th = None if thetas is None else np.ascontiguousarray(np.broadcast_to(thetas, b.shape), dtype=np.int32)
    rt = None if R_targets is None else np.ascontiguousarray(np.broadcast_to(R_targets, b.shape), dtype=np.int64)
    _check(load().pa_run_schedule(h, len(b), _ptr(b), _ptr(th), _ptr(rt), 1 if use_graph else 0),
           "pa_run_schedule")


def pa_step_target(h, beta_next: float, sweeps: int, R_target: int):
    _check(load().pa_step_target(h, beta_next, sweeps, R_target), "pa_step_target")


def pa_sync(h):
    _check(load().pa_sync(h), "pa_sync")


def pa_observables(h) -> dict:
    o = Obs()
    _check(load().pa_observables(h, ctypes.byref(o)), "pa_observables")
    return {f: getattr(o, f) for f, _ in Obs._fields_}


def pa_free_energy(h) -> float:
    v = c_double()
    _check(load().pa_free_energy(h, ctypes.byref(v)), "pa_free_energy")
    return v.value


def pa_trajectory(h, count: int) -> dict:
    out = {k: np.zeros(count, dtype=np.float64) for k in ("beta", "lnQ", "minus_beta_F")}
    out.update({k: np.zeros(count, dtype=np.int64) for k in ("R", "sumE", "sumE2")})
    n = c_int64()
    _check(load().pa_trajectory(h, count, _ptr(out["beta"]), _ptr(out["lnQ"]),
                                _ptr(out["minus_beta_F"]), _ptr(out["R"]), _ptr(out["sumE"]),
                                _ptr(out["sumE2"]), ctypes.byref(n)), "pa_trajectory")
    return {k: v[: n.value] for k, v in out.items()}


def pa_trajectory_energy(h, count: int) -> dict:
    out = {k: np.zeros(count, dtype=np.float64) for k in ("E_mean", "E2_mean")}
    n = c_int64()
    _check(load().pa_trajectory_energy(h, count, _ptr(out["E_mean"]), _ptr(out["E2_mean"]),
                                       ctypes.byref(n)), "pa_trajectory_energy")
    return {k: v[: n.value] for k, v in out.items()}


def pa_copy_spins(h, max_replicas: int, N: int) -> np.ndarray:
    out = np.empty((max_replicas, N), dtype=np.int8)
    n = c_int64()
    _check(load().pa_copy_spins(h, _ptr(out), max_replicas, ctypes.byref(n)), "pa_copy_spins")
    return out[: n.value]


def pa_copy_energies(h, max_replicas: int) -> np.ndarray:
    out = np.empty(max_replicas, dtype=np.int32)
    n = c_int64()
    _check(load().pa_copy_energies(h, _ptr(out), max_replicas, ctypes.byref(n)), "pa_copy_energies")
    return out[: n.value]


def pa_copy_copies(h, max_replicas: int) -> np.ndarray:
    out = np.empty(max_replicas, dtype=np.int32)
    n = c_int64()
    _check(load().pa_copy_copies(h, _ptr(out), max_replicas, ctypes.byref(n)), "pa_copy_copies")
    return out[: n.value]


def pa_overlap(a, b, qcut: float, N: int):
    g, n = c_double(), c_int64()
    hist = np.zeros(N + 1, dtype=np.int64)
    _check(load().pa_overlap(a, b, qcut, ctypes.byref(g), ctypes.byref(n), _ptr(hist)), "pa_overlap")
    return g.value, n.value, hist


def pa_weighted_average(x, A=None, R=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    A = None if A is None else np.ascontiguousarray(A, dtype=np.float64)
    R = None if R is None else np.ascontiguousarray(R, dtype=np.float64)
    m, f = c_double(), c_double()
    _check(load().pa_weighted_average(len(x), _ptr(x), _ptr(A), _ptr(R), ctypes.byref(m),
                                      ctypes.byref(f)), "pa_weighted_average")
    return m.value, f.value


def pa_weighted_average_pairs(x1, x2, A=None, R1=None, R2=None):
    """Eqs. (10)-(11) of Sec. 4 through the C ABI: (weighted mean, -beta F-bar of
    the two-run system) over M pairs of runs."""
    x1 = np.ascontiguousarray(x1, dtype=np.float64)
    x2 = np.ascontiguousarray(x2, dtype=np.float64)
    A = None if A is None else np.ascontiguousarray(A, dtype=np.float64)
    R1 = None if R1 is None else np.ascontiguousarray(R1, dtype=np.float64)
    R2 = None if R2 is None else np.ascontiguousarray(R2, dtype=np.float64)
    if any(a is not None and len(a) != len(x1) for a in (x2, A, R1, R2)):
        raise ValueError("pair arrays must have the same length")
    m, f = c_double(), c_double()
    _check(load().pa_weighted_average_pairs(len(x1), _ptr(x1), _ptr(x2), _ptr(A), _ptr(R1), _ptr(R2),
                                            ctypes.byref(m), ctypes.byref(f)), "pa_weighted_average_pairs")
    return m.value, f.value


def pair_weighted_average(minus_beta_F_1, minus_beta_F_2, A, R1=None, R2=None):
    """The weighted estimator of Eq. (10) with the pair weights of Eq. (11)
    (Sec. 4): the overlap observable of M pairs of independent runs."""
    return pa_weighted_average_pairs(minus_beta_F_1, minus_beta_F_2, A, R1, R2)[0]


def pa_bootstrap(x, A=None, R=None, B: int = 100, seed: int = 0):
    x = np.ascontiguousarray(x, dtype=np.float64)
    A = None if A is None else np.ascontiguousarray(A, dtype=np.float64)
    R = None if R is None else np.ascontiguousarray(R, dtype=np.float64)
    sm, sf = c_double(), c_double()
    _check(load().pa_bootstrap(len(x), _ptr(x), _ptr(A), _ptr(R), B, seed, ctypes.byref(sm),
                               ctypes.byref(sf)), "pa_bootstrap")
    return sm.value, sf.value


# ---- conveniences -------------------------------------------------------------------------

class Run:
    """One annealing run on the current GPU (Sec. 2 of the paper).  With
    gaussian=True the couplings are int32 J_q of the Gaussian model (Sec. 4)."""

    def __init__(self, couplings, L: int, dim: int, R0: int, seed: int, R_cap: int = 0,
                 max_steps: int = 0, threads_per_block: int = 0, use_torch: bool = True,
                 gaussian: bool = False, Ls=None, periodic_mask: int = 7, threads_per_replica: int = 0):
        self.L, self.dim, self.R0 = L, dim, R0
        self.N = L ** 3 if dim == 3 else L
        if Ls is not None:
            self.N = int(np.prod(Ls)) if dim == 3 else int(Ls[0])
        self.gaussian = gaussian
        opts = torch_opts(R_cap, max_steps, threads_per_block, threads_per_replica) if use_torch else None
        if opts is None and (R_cap or max_steps or threads_per_block or threads_per_replica):
            opts = Opts()
            opts.R_cap, opts.max_steps, opts.threads_per_block = R_cap, max_steps, threads_per_block
            opts.threads_per_replica = threads_per_replica
        self._opts = opts
        if Ls is not None:
            self._h = pa_create_lattice(couplings, Ls, dim, periodic_mask, R0, seed, opts, gaussian)
        elif gaussian:
            self._h = pa_create_gauss(couplings, L, dim, R0, seed, opts)
        else:
            self._h = pa_create(couplings, L, dim, R0, seed, opts)

    def close(self):
        if getattr(self, "_h", None):
            pa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, beta_next: float, sweeps: int, R_target: int | None = None):
        if R_target is None:
            pa_step(self._h, beta_next, sweeps)
        else:
            pa_step_target(self._h, beta_next, sweeps, R_target)

    def run_schedule(self, betas, thetas=None, R_targets=None, use_graph: bool = True):
        """Steps to betas[0], betas[1], ... (pa_run_schedule)."""
        pa_run_schedule(self._h, betas, thetas, R_targets, use_graph)

    def sync(self):
        pa_sync(self._h)

    def reset(self, seed: int):
        pa_reset(self._h, seed)

    def checkpoint(self) -> bytes:
        return pa_checkpoint(self._h)

    def restore(self, blob: bytes):
        pa_restore(self._h, blob)

    def observables(self) -> dict:
        return pa_observables(self._h)

    def free_energy(self) -> float:
        return pa_free_energy(self._h)

    def trajectory(self, count: int = 1 << 20) -> dict:
        return pa_trajectory(self._h, min(count, 1 << 20))

    def trajectory_energy(self, count: int = 1 << 20) -> dict:
        return pa_trajectory_energy(self._h, min(count, 1 << 20))

    def spins(self, max_replicas: int | None = None) -> np.ndarray:
        R = self.observables()["R"] if max_replicas is None else max_replicas
        return pa_copy_spins(self._h, R, self.N)

    def energies(self) -> np.ndarray:
        return pa_copy_energies(self._h, self.observables()["R"])

    def copies(self, n: int) -> np.ndarray:
        return pa_copy_copies(self._h, n)


def overlap(a: Run, b: Run, qcut: float = 0.2):
    return pa_overlap(a._h, b._h, qcut, a.N)


class Batch:
    """Many independent runs advanced together (one CUDA graph per schedule)."""

    def __init__(self, specs, max_steps: int = 0, threads_per_block: int = 0, use_torch: bool = True,
                 opts: Opts | None = None):
        gauss = [bool(getattr(s, "gaussian", False)) for s in specs]
        self._J = [np.ascontiguousarray(s.couplings(), dtype=np.int32 if g else np.int8)
                   for s, g in zip(specs, gauss)]
        arr = (RunSpecC * len(specs))()
        for i, (s, J) in enumerate(zip(specs, self._J)):
            arr[i].dim, arr[i].L = s.dim, s.L
            if gauss[i]:
                arr[i].couplings, arr[i].gauss_couplings = None, J.ctypes.data_as(c_void_p)
            else:
                arr[i].couplings, arr[i].gauss_couplings = J.ctypes.data_as(c_void_p), None
            arr[i].R0, arr[i].seed, arr[i].R_cap = s.R0, s.seed, int(getattr(s, "R_cap", 0))
        self.specs = list(specs)
        if opts is None:
            opts = torch_opts(0, max_steps, threads_per_block) if use_torch else Opts()
            if not use_torch:
                opts.max_steps, opts.threads_per_block = max_steps, threads_per_block
        self._opts = opts
        h = c_void_p()
        _check(load().pa_batch_create(len(specs), arr, ctypes.byref(opts), ctypes.byref(h)),
               "pa_batch_create")
        self._h = h
        self.n = len(specs)

    def close(self):
        if getattr(self, "_h", None):
            load().pa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, betas, thetas=None, R_targets=None, use_graph: bool = True):
        betas = np.ascontiguousarray(betas, dtype=np.float64)
        per_run = 1 if betas.ndim == 2 else 0
        n_steps = betas.shape[-1]
        th = None if thetas is None else np.ascontiguousarray(np.broadcast_to(thetas, betas.shape), dtype=np.int32)
        rt = None if R_targets is None else np.ascontiguousarray(np.broadcast_to(R_targets, betas.shape), dtype=np.int64)
        self._keep = (betas, th, rt)
        _check(load().pa_batch_run(self._h, n_steps, _ptr(betas), per_run, _ptr(th), _ptr(rt),
                                   1 if use_graph else 0), "pa_batch_run")

    def sync(self) -> np.ndarray:
        err = np.zeros(self.n, dtype=np.int32)
        code = load().pa_batch_sync(self._h, _ptr(err))
        if code not in (PA_OK, PA_ERR_CAPACITY, PA_ERR_EXTINCT, PA_ERR_INVALID):
            _check(code, "pa_batch_sync")
        return err

    def results(self) -> dict:
        out = {"beta": np.zeros(self.n), "minus_beta_F": np.zeros(self.n)}
        out.update({k: np.zeros(self.n, dtype=np.int64) for k in ("R", "sumE", "sumE2", "step")})
        _check(load().pa_batch_results(self._h, _ptr(out["beta"]), _ptr(out["minus_beta_F"]),
                                       _ptr(out["R"]), _ptr(out["sumE"]), _ptr(out["sumE2"]),
                                       _ptr(out["step"])), "pa_batch_results")
        return out

    def trajectory(self, count: int) -> dict:
        out = {"minus_beta_F": np.zeros((self.n, count))}
        out.update({k: np.zeros((self.n, count), dtype=np.int64) for k in ("R", "sumE", "sumE2")})
        _check(load().pa_batch_trajectory(self._h, count, _ptr(out["minus_beta_F"]), _ptr(out["R"]),
                                          _ptr(out["sumE"]), _ptr(out["sumE2"])),
               "pa_batch_trajectory")
        return out

    def energy(self, count: int) -> dict:
        """Per-run per-step E_mean and E2_mean in physical units, [n_runs][count]."""
        out = {k: np.zeros((self.n, count)) for k in ("E_mean", "E2_mean")}
        _check(load().pa_batch_energy(self._h, count, _ptr(out["E_mean"]), _ptr(out["E2_mean"])),
               "pa_batch_energy")
        return out

    def diagnostics(self, M: int, count: int) -> dict:
        """Sec. 3 estimators per group of M consecutive runs and per record,
        on the device: R-weighted E_bar, -beta F_bar (Eq. (7)) and
        Var(-beta F~); arrays [n_runs // M][count]."""
        G = self.n // M
        out = {k: np.zeros((G, count)) for k in ("E_bar", "minus_beta_F_bar", "var_minus_beta_F")}
        _check(load().pa_batch_diagnostics(self._h, M, count, _ptr(out["E_bar"]), _ptr(out["minus_beta_F_bar"]),
                                           _ptr(out["var_minus_beta_F"])), "pa_batch_diagnostics")
        return out

    def bootstrap(self, M: int, count: int, B: int = 100, seed: int = 0) -> dict:
        """Sec. 3 bootstrap standard deviations of E_bar and -beta F_bar per
        group of M consecutive runs and per record, on the device; arrays
        [n_runs // M][count]."""
        G = self.n // M
        out = {k: np.zeros((G, count)) for k in ("sd_E_bar", "sd_minus_beta_F_bar")}
        _check(load().pa_batch_bootstrap(self._h, M, count, B, seed, _ptr(out["sd_E_bar"]),
                                         _ptr(out["sd_minus_beta_F_bar"])), "pa_batch_bootstrap")
        return out

    def overlap(self, run_a, run_b, qcut: float = 0.2):
        """Sec. 4: Gamma = Prob(|q| < qcut) for each pair (run_a[p], run_b[p])
        of this batch's runs; returns (gamma, npairs) arrays."""
        a = np.ascontiguousarray(run_a, dtype=np.int32)
        b = np.ascontiguousarray(run_b, dtype=np.int32)
        gamma = np.zeros(len(a))
        npairs = np.zeros(len(a), dtype=np.int64)
        _check(load().pa_batch_overlap(self._h, len(a), _ptr(a), _ptr(b), qcut, _ptr(gamma), _ptr(npairs)),
               "pa_batch_overlap")
        return gamma, npairs

    def reset(self, seeds=None):
        """Fresh beta = 0 populations (pa_batch_reset); seeds: one per run or
        None to keep each run's seed."""
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        _check(load().pa_batch_reset(self._h, _ptr(sd)), "pa_batch_reset")

    def overlap_hist(self, run_a, run_b) -> np.ndarray:
        """Sec. 4, P(q): counts [n_pairs][N + 1] of (N q + N) / 2 for the pairs
        (run_a[p], run_b[p]) of this batch's runs (pa_batch_overlap_hist)."""
        a = np.ascontiguousarray(run_a, dtype=np.int32)
        b = np.ascontiguousarray(run_b, dtype=np.int32)
        N = self.specs[int(a[0])].N
        out = np.zeros((len(a), N + 1), dtype=np.int64)
        _check(load().pa_batch_overlap_hist(self._h, len(a), _ptr(a), _ptr(b), _ptr(out)), "pa_batch_overlap_hist")
        return out

    def autotune(self, sweeps: int = 0) -> dict:
        """{L (negative for chains): (threads per block, threads per replica)},
        timed on a dry step of `sweeps` Metropolis sweeps (the schedule's; capped
        at 20; 0 = 10)."""
        Ls = np.zeros(8, dtype=np.int32)
        tp = np.zeros(8, dtype=np.int32)
        sp = np.zeros(8, dtype=np.int32)
        n = c_int()
        _check(load().pa_batch_autotune(self._h, int(sweeps), _ptr(Ls), _ptr(tp), _ptr(sp), ctypes.byref(n)),
               "pa_batch_autotune")
        return {int(Ls[i]): (int(tp[i]), int(sp[i])) for i in range(n.value)}

    def spins(self, r: int, max_replicas: int) -> np.ndarray:
        N = self.specs[r].N
        out = np.empty((max_replicas, N), dtype=np.int8)
        n = c_int64()
        _check(load().pa_batch_copy_spins(self._h, r, _ptr(out), max_replicas, ctypes.byref(n)),
               "pa_batch_copy_spins")
        return out[: n.value]

    def checkpoint(self) -> bytes:
        """The state of every run of the batch (pa_batch_checkpoint)."""
        n = c_size_t()
        _check(load().pa_batch_checkpoint_bytes(self._h, ctypes.byref(n)), "pa_batch_checkpoint_bytes")
        buf = ctypes.create_string_buffer(n.value)
        _check(load().pa_batch_checkpoint(self._h, buf, n.value), "pa_batch_checkpoint")
        return buf.raw

    def restore(self, blob: bytes):
        """Load a batch checkpoint into this batch (pa_batch_restore)."""
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(load().pa_batch_restore(self._h, buf, len(blob)), "pa_batch_restore")


class Server:
    """Continuous batching of annealing requests (pa_server_*)."""

    STATUS = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}

    def __init__(self, hbm_budget_bytes: float = 0.0, max_runs: int = 256, max_steps: int = 0,
                 threads_per_block: int = 0, use_torch: bool = True, opts: Opts | None = None):
        if opts is None:
            opts = torch_opts(0, max_steps, threads_per_block) if use_torch else Opts()
            if not use_torch:
                opts.max_steps, opts.threads_per_block = max_steps, threads_per_block
        self._opts = opts
        h = c_void_p()
        _check(load().pa_server_create(ctypes.byref(opts), float(hbm_budget_bytes), max_runs,
                                       ctypes.byref(h)), "pa_server_create")
        self._h = h
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            load().pa_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, dim: int, L: int, couplings, R0: int, seed: int, betas, theta: int) -> int:
        J = np.ascontiguousarray(couplings, dtype=np.int8).reshape(-1)
        b = np.ascontiguousarray(betas, dtype=np.float64)
        q = RequestC(dim, L, J.ctypes.data_as(c_void_p), R0, seed, len(b), theta,
                     b.ctypes.data_as(c_void_p))
        rid = c_int64()
        _check(load().pa_server_submit(self._h, ctypes.byref(q), ctypes.byref(rid)), "pa_server_submit")
        return rid.value

    def cancel(self, rid: int):
        _check(load().pa_server_cancel(self._h, rid), "pa_server_cancel")

    def memory(self) -> dict:
        u, b, n = c_int64(), c_int64(), c_int32()
        _check(load().pa_server_memory(self._h, ctypes.byref(u), ctypes.byref(b), ctypes.byref(n)),
               "pa_server_memory")
        return {"used_bytes": u.value, "budget_bytes": b.value, "runs_resident": n.value}

    def tick(self, steps: int = 1):
        a, q, f = c_int32(), c_int32(), c_int32()
        _check(load().pa_server_tick(self._h, steps, ctypes.byref(a), ctypes.byref(q), ctypes.byref(f)),
               "pa_server_tick")
        return a.value, q.value, f.value

    def result(self, rid: int, traj_count: int = 0) -> dict:
        r = ResultC()
        tr = np.zeros(max(traj_count, 1), dtype=np.float64)
        _check(load().pa_server_result(self._h, rid, ctypes.byref(r), _ptr(tr) if traj_count else None,
                                       traj_count), "pa_server_result")
        out = {f: getattr(r, f) for f, _ in ResultC._fields_}
        if traj_count:
            out["trajectory"] = tr[: min(traj_count, r.steps + 1)]
        return out

    def clock(self) -> float:
        return load().pa_server_clock(self._h)
