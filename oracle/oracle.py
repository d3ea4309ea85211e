"""ctypes wrapper around the plain C oracle (``pa_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, literal CPU statement of
population annealing with weighted averages (Machta 2010, Sec. 2-4) that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline / reference legs may import this module; the
product package never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pa_oracle.c")
SRC_GAUSS = os.path.join(HERE, "pa_oracle_gauss.c")
LIB = os.path.join(HERE, "libpa_oracle.so")
# A prebuilt copy (used by the mutation tests to load a deliberately broken
# oracle) may be named here; it is then loaded as is.
_LIB_OVERRIDE = os.environ.get("PA_ORACLE_LIB")

OK, ERR_INVALID, ERR_OOM, ERR_CAPACITY, ERR_EXTINCT, ERR_STATE = 0, 1, 2, 3, 4, 5
TAG_INIT, TAG_RESAMPLE, TAG_SWEEP, TAG_BOOT = 0x1A000000, 0x2B000000, 0x3C000000, 0x4D000000


def build(force: bool = False, src: str = SRC, out: str = LIB, src_gauss: str = SRC_GAUSS) -> str:
    """Compile the oracle with every floating-point operation rounded as written."""
    if out != LIB:
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                        "-fPIC", "-shared", "-I", HERE, "-o", out, src, src_gauss, "-lm"], check=True)
        return out
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(SRC_GAUSS),
                                             os.path.getmtime(os.path.join(HERE, "pa_oracle.h")))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, SRC, SRC_GAUSS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _State(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("R", ctypes.c_int64),
                ("minus_beta_F", ctypes.c_double), ("lnQ_last", ctypes.c_double),
                ("Qprime_last", ctypes.c_double), ("step", ctypes.c_int64),
                ("sweeps", ctypes.c_int64), ("sumE", ctypes.c_int64),
                ("sumE2", ctypes.c_int64), ("N", ctypes.c_int64), ("Nb", ctypes.c_int64),
                ("R_cap", ctypes.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_LIB_OVERRIDE or build())
        L = _lib
        P = ctypes.POINTER
        L.or_philox.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.or_pexp.argtypes = [ctypes.c_double]
        L.or_pexp.restype = ctypes.c_double
        L.or_u53.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.or_u53.restype = ctypes.c_double
        L.or_poisson_piece.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_poisson_piece.restype = ctypes.c_int32
        L.or_threshold.argtypes = [ctypes.c_double, ctypes.c_int]
        L.or_threshold.restype = ctypes.c_uint32
        L.or_site_label.argtypes = [ctypes.c_void_p, ctypes.c_int64, P(ctypes.c_int64),
                                    P(ctypes.c_int), P(ctypes.c_int)]
        L.or_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_uint, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_uint64, P(ctypes.c_void_p)]
        L.or_destroy.argtypes = [ctypes.c_void_p]
        L.or_destroy.restype = None
        L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64]
        L.or_sweep_fixed.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        L.or_get_state.argtypes = [ctypes.c_void_p, P(_State)]
        L.or_resample.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                  P(ctypes.c_int64), P(ctypes.c_double), P(ctypes.c_double)]
        L.or_sweep_replica.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                       P(ctypes.c_int64)]
        for name in ("or_copy_spins", "or_copy_energies", "or_copy_copies"):
            getattr(L, name).argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            getattr(L, name).restype = ctypes.c_int64
        L.or_energy_of.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.or_energy_of.restype = ctypes.c_int64
        L.or_overlap.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                 P(ctypes.c_double), P(ctypes.c_int64), ctypes.c_void_p]
        L.or_weighted_average.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, P(ctypes.c_double),
                                          P(ctypes.c_double)]
        L.or_weighted_average_pairs.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]
        L.or_bootstrap.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                   P(ctypes.c_double), P(ctypes.c_double)]
        L.or_variance.argtypes = [ctypes.c_int, ctypes.c_void_p]
        L.or_variance.restype = ctypes.c_double
        L.og_fexp.argtypes = [ctypes.c_float]
        L.og_fexp.restype = ctypes.c_float
        L.og_accept.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_uint32]
        L.og_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_uint, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_uint64, P(ctypes.c_void_p)]
        L.og_destroy.argtypes = [ctypes.c_void_p]
        L.og_destroy.restype = None
        L.og_step.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64]
        L.og_sweep_fixed.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        L.og_get_state.argtypes = [ctypes.c_void_p, P(_State), P(ctypes.c_double)]
        for name in ("og_copy_spins", "og_copy_energies", "og_copy_copies"):
            getattr(L, name).argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            getattr(L, name).restype = ctypes.c_int64
        L.og_energy.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.og_energy.restype = ctypes.c_int64
        L.og_resample.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                  P(ctypes.c_int64), P(ctypes.c_double), P(ctypes.c_double)]
        L.og_sweep_replica.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                       P(ctypes.c_int64)]
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---- primitives --------------------------------------------------------------------

def philox(ctr, key) -> tuple[int, int, int, int]:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox(c, k, o)
    return tuple(int(v) for v in o)


def pexp(x: float) -> float:
    return lib().or_pexp(float(x))


def u53(w0: int, w1: int) -> float:
    return lib().or_u53(w0, w1)


def poisson_piece(u: float, am: float, p0: float) -> int:
    return lib().or_poisson_piece(u, am, p0)


def threshold(beta: float, dE: int) -> int:
    return lib().or_threshold(beta, dE)


def weighted_average(x, A=None, R=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    A = None if A is None else np.ascontiguousarray(A, dtype=np.float64)
    R = None if R is None else np.ascontiguousarray(R, dtype=np.float64)
    mean, fbar = ctypes.c_double(), ctypes.c_double()
    st = lib().or_weighted_average(len(x), _ptr(x), _ptr(A), _ptr(R),
                                   ctypes.byref(mean), ctypes.byref(fbar))
    if st != OK:
        raise ValueError(f"or_weighted_average: {st}")
    return mean.value, fbar.value


def weighted_average_pairs(x1, x2, A=None, R1=None, R2=None):
    """Sec. 4, Eqs. (10)-(11): (weighted mean, ln[(1/M) sum e^{x1+x2}]) over pairs of runs."""
    x1 = np.ascontiguousarray(x1, dtype=np.float64)
    x2 = np.ascontiguousarray(x2, dtype=np.float64)
    A, R1, R2 = (None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (A, R1, R2))
    mean, fbar = ctypes.c_double(), ctypes.c_double()
    st = lib().or_weighted_average_pairs(len(x1), _ptr(x1), _ptr(x2), _ptr(A), _ptr(R1), _ptr(R2),
                                         ctypes.byref(mean), ctypes.byref(fbar))
    if st != OK:
        raise ValueError(f"or_weighted_average_pairs: {st}")
    return mean.value, fbar.value


def bootstrap(x, A=None, R=None, B: int = 100, seed: int = 0):
    x = np.ascontiguousarray(x, dtype=np.float64)
    A = None if A is None else np.ascontiguousarray(A, dtype=np.float64)
    R = None if R is None else np.ascontiguousarray(R, dtype=np.float64)
    sm, sf = ctypes.c_double(), ctypes.c_double()
    st = lib().or_bootstrap(len(x), _ptr(x), _ptr(A), _ptr(R), B, seed,
                            ctypes.byref(sm), ctypes.byref(sf))
    if st != OK:
        raise ValueError(f"or_bootstrap: {st}")
    return sm.value, sf.value


def variance(x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().or_variance(len(x), _ptr(x))


# ---- runs --------------------------------------------------------------------------

@dataclass
class State:
    beta: float
    R: int
    minus_beta_F: float
    lnQ_last: float
    Qprime_last: float
    step: int
    sweeps: int
    sumE: int
    sumE2: int
    N: int
    Nb: int
    R_cap: int


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


class Run:
    """One population-annealing run held by the oracle."""

    def __init__(self, J: np.ndarray, dim: int, Lx: int, Ly: int = 1, Lz: int = 1,
                 periodic_mask: int = 7, R0: int = 1000, R_cap: int | None = None,
                 seed: int = 1):
        self._J = np.ascontiguousarray(J, dtype=np.int8)
        if R_cap is None:
            R_cap = default_capacity(R0)
        h = ctypes.c_void_p()
        st = lib().or_create(dim, Lx, Ly, Lz, periodic_mask, _ptr(self._J), R0, R_cap,
                             seed, ctypes.byref(h))
        if st != OK:
            raise OracleError(st, "or_create")
        self._h = h
        self.dim, self.N = dim, Lx * Ly * Lz

    def close(self):
        if getattr(self, "_h", None):
            lib().or_destroy(self._h)
            self._h = None

    __del__ = close

    def step(self, beta_next: float, theta: int, R_target: int):
        st = lib().or_step(self._h, beta_next, theta, R_target)
        if st != OK:
            raise OracleError(st, "or_step")

    def sweep_fixed(self, beta: float, theta: int):
        st = lib().or_sweep_fixed(self._h, beta, theta)
        if st != OK:
            raise OracleError(st, "or_sweep_fixed")

    def state(self) -> State:
        s = _State()
        lib().or_get_state(self._h, ctypes.byref(s))
        return State(**{f: getattr(s, f) for f, _ in _State._fields_})

    def spins(self) -> np.ndarray:
        st = self.state()
        out = np.empty((st.R, self.N), dtype=np.int8)
        lib().or_copy_spins(self._h, _ptr(out), st.R)
        return out

    def energies(self) -> np.ndarray:
        st = self.state()
        out = np.empty(st.R, dtype=np.int32)
        lib().or_copy_energies(self._h, _ptr(out), st.R)
        return out

    def copies(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.int32)
        k = lib().or_copy_copies(self._h, _ptr(out), n)
        return out[:k]

    def energy_of(self, sigma: np.ndarray) -> int:
        s = np.ascontiguousarray(sigma, dtype=np.int8)
        return int(lib().or_energy_of(self._h, _ptr(s)))

    def resample(self, E: np.ndarray, beta: float, beta_next: float, R_target: int, step: int):
        """Copy counts, R~', Q' and ln Q for a population with energies E."""
        E = np.ascontiguousarray(E, dtype=np.int32)
        copies = np.empty(len(E), dtype=np.int32)
        Rn, Qp, lnQ = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        st = lib().or_resample(self._h, _ptr(E), len(E), beta, beta_next, R_target, step,
                               _ptr(copies), ctypes.byref(Rn), ctypes.byref(Qp), ctypes.byref(lnQ))
        if st != OK:
            raise OracleError(st, "or_resample")
        return copies, Rn.value, Qp.value, lnQ.value

    def sweep_replica(self, sigma: np.ndarray, slot: int, T0: int, beta: float, theta: int):
        """theta sweeps of one replica in slot `slot` from global sweep T0."""
        s = np.ascontiguousarray(sigma, dtype=np.int8).copy()
        E = ctypes.c_int64()
        st = lib().or_sweep_replica(self._h, _ptr(s), slot, T0, beta, theta, ctypes.byref(E))
        if st != OK:
            raise OracleError(st, "or_sweep_replica")
        return s, E.value

    def site_label(self, i: int) -> tuple[int, int, int]:
        """(w, p, S): packed word, bit position, colour-c sites per word."""
        w, p, S = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        st = lib().or_site_label(self._h, i, ctypes.byref(w), ctypes.byref(p), ctypes.byref(S))
        if st != OK:
            raise OracleError(st, "or_site_label")
        return w.value, p.value, S.value


def overlap(a, b, qcut: float = 0.2):
    """Sec. 4: Gamma = Prob(|q| < qcut) over replica pairs (k of run a, k of
    run b), q = (1/N) sum_i s_i s'_i; also the counts of (N q + N) / 2."""
    if not (isinstance(a, Run) and isinstance(b, Run)):
        # Gaussian-coupling runs: the same definition on their spin arrays
        sa, sb = a.spins(), b.spins()
        n = min(len(sa), len(sb))
        N = sa.shape[1]
        dot = (sa[:n].astype(np.int64) * sb[:n].astype(np.int64)).sum(axis=1)
        hist = np.bincount((dot + N) // 2, minlength=N + 1).astype(np.int64)
        count = int((np.abs(dot.astype(np.float64)) < qcut * N).sum())
        return (count / n if n > 0 else 0.0), int(n), hist
    g, n = ctypes.c_double(), ctypes.c_int64()
    hist = np.zeros(a.N + 1, dtype=np.int64)
    st = lib().or_overlap(a._h, b._h, qcut, ctypes.byref(g), ctypes.byref(n), _ptr(hist))
    if st != OK:
        raise OracleError(st, "or_overlap")
    return g.value, n.value, hist


def default_capacity(R0: int) -> int:
    """Population cap R0 + 10 ceil(sqrt(R0)) + 64 (the paper leaves it open)."""
    import math
    r = math.isqrt(int(R0))
    if r * r < R0:
        r += 1
    return int(R0) + 10 * r + 64


# ---- Gaussian couplings ------------------------------------------------------------

GAUSS_SCALE = 2.0 ** 15  # physical J = J_q / GAUSS_SCALE


def fexp(x: float) -> float:
    return lib().og_fexp(float(x))


def gauss_accept(beta: float, dE_q: int, u: int) -> bool:
    return bool(lib().og_accept(beta, dE_q, u))


class GaussRun:
    """One population-annealing run with fixed-point Gaussian couplings."""

    def __init__(self, J: np.ndarray, dim: int, Lx: int, Ly: int = 1, Lz: int = 1,
                 periodic_mask: int = 7, R0: int = 1000, R_cap: int | None = None, seed: int = 1):
        self._J = np.ascontiguousarray(J, dtype=np.int32)
        if R_cap is None:
            R_cap = default_capacity(R0)
        h = ctypes.c_void_p()
        st = lib().og_create(dim, Lx, Ly, Lz, periodic_mask, _ptr(self._J), R0, R_cap, seed,
                             ctypes.byref(h))
        if st != OK:
            raise OracleError(st, "og_create")
        self._h = h
        self.dim, self.N = dim, Lx * Ly * Lz

    def close(self):
        if getattr(self, "_h", None):
            lib().og_destroy(self._h)
            self._h = None

    __del__ = close

    def step(self, beta_next: float, theta: int, R_target: int):
        st = lib().og_step(self._h, beta_next, theta, R_target)
        if st != OK:
            raise OracleError(st, "og_step")

    def sweep_fixed(self, beta: float, theta: int):
        st = lib().og_sweep_fixed(self._h, beta, theta)
        if st != OK:
            raise OracleError(st, "og_sweep_fixed")

    def state(self) -> State:
        s = _State()
        e2 = ctypes.c_double()
        lib().og_get_state(self._h, ctypes.byref(s), ctypes.byref(e2))
        st = State(**{f: getattr(s, f) for f, _ in _State._fields_})
        st.sumE2 = e2.value  # physical units for Gaussian runs
        return st

    def spins(self) -> np.ndarray:
        R = self.state().R
        out = np.empty((R, self.N), dtype=np.int8)
        lib().og_copy_spins(self._h, _ptr(out), R)
        return out

    def energies(self) -> np.ndarray:
        R = self.state().R
        out = np.empty(R, dtype=np.int64)
        lib().og_copy_energies(self._h, _ptr(out), R)
        return out

    def copies(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.int32)
        k = lib().og_copy_copies(self._h, _ptr(out), n)
        return out[:k]

    def energy_of(self, sigma: np.ndarray) -> int:
        s = np.ascontiguousarray(sigma, dtype=np.int8)
        return int(lib().og_energy(self._h, _ptr(s)))

    def resample(self, E: np.ndarray, beta: float, beta_next: float, R_target: int, step: int):
        E = np.ascontiguousarray(E, dtype=np.int64)
        copies = np.empty(len(E), dtype=np.int32)
        Rn, Qp, lnQ = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        st = lib().og_resample(self._h, _ptr(E), len(E), beta, beta_next, R_target, step,
                               _ptr(copies), ctypes.byref(Rn), ctypes.byref(Qp), ctypes.byref(lnQ))
        if st != OK:
            raise OracleError(st, "og_resample")
        return copies, Rn.value, Qp.value, lnQ.value

    def sweep_replica(self, sigma: np.ndarray, slot: int, T0: int, beta: float, theta: int):
        s = np.ascontiguousarray(sigma, dtype=np.int8).copy()
        E = ctypes.c_int64()
        st = lib().og_sweep_replica(self._h, _ptr(s), slot, T0, beta, theta, ctypes.byref(E))
        if st != OK:
            raise OracleError(st, "og_sweep_replica")
        return s, E.value
