"""Seeded synthetic inputs for population-annealing workloads.

This module holds none of the method's arithmetic: it only produces the
quenched couplings, population sizes, annealing schedules and request streams
that both the CUDA path and the CPU oracle consume.  Random bits come from
SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), written out here with numpy
integer operations so the streams are identical on every machine and numpy
version.

The paper's own realisations (Gaussian couplings, Sec. 4) were never
published; the workloads here use +-1 couplings of the same lattice shapes,
and Gaussian couplings (Box-Muller on SplitMix64, rounded to a 2^-15
fixed-point grid) for the Gaussian model.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n outputs of SplitMix64 started from a state derived from (seed, stream)."""
    with np.errstate(over="ignore"):
        start = _mix(np.array([(seed * 0x100000001B3 + stream * 0xD1342543DE82EF95)
                               & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        k = np.arange(1, n + 1, dtype=np.uint64)
        return _mix(start + k * _GAMMA)


def couplings_3d(L: int, realization: int = 0, seed: int = 1) -> np.ndarray:
    """+-1 couplings, equiprobable, for an L^3 periodic cubic lattice.

    Layout [3][N]: J[d][i] couples site i = x + L(y + L z) to its +d
    neighbour (d = x, y, z), with periodic wrap."""
    N = L ** 3
    bits = splitmix64(seed, 3 * N, stream=realization) >> np.uint64(63)
    return np.where(bits == 1, 1, -1).astype(np.int8).reshape(3, N)


def couplings_lattice(Lx: int, Ly: int, Lz: int, realization: int = 0,
                      seed: int = 1) -> np.ndarray:
    """+-1 couplings in the [3][N] layout for a general Lx x Ly x Lz box."""
    N = Lx * Ly * Lz
    bits = splitmix64(seed, 3 * N, stream=realization) >> np.uint64(63)
    return np.where(bits == 1, 1, -1).astype(np.int8).reshape(3, N)


def couplings_chain(N: int, realization: int = 0, seed: int = 1,
                    open_chain: bool = True) -> np.ndarray:
    """+-1 couplings of a chain of N spins; J[i] joins i and i+1, J[N-1] is the
    wrap bond and is 0 for an open chain."""
    bits = splitmix64(seed, N, stream=1000 + realization) >> np.uint64(63)
    J = np.where(bits == 1, 1, -1).astype(np.int8)
    if open_chain:
        J[N - 1] = 0
    return J


GAUSS_SCALE_BITS = 15  # Gaussian couplings as integers J_q, physical J = J_q * 2^-15


def _gaussians(n: int, seed: int, stream: int) -> np.ndarray:
    """n standard normal deviates by the Box-Muller transform of SplitMix64
    uniforms (two uniforms per pair)."""
    m = (n + 1) // 2
    raw = splitmix64(seed, 2 * m, stream=stream)
    u1 = ((raw[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53  # (0, 1]
    u2 = (raw[1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    g = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return g.reshape(2, m).T.reshape(-1)[:n]


def gaussian_couplings_fixed(g: np.ndarray) -> np.ndarray:
    """Round Gaussian couplings to the fixed-point grid 2^-15 (int32)."""
    q = np.rint(np.clip(g, -7.99, 7.99) * 2.0 ** GAUSS_SCALE_BITS)
    return q.astype(np.int32)


def gaussian_couplings_3d(L: int, realization: int = 0, seed: int = 1) -> np.ndarray:
    """Gaussian couplings (mean 0, variance 1) of an L^3 periodic lattice, the
    model of the paper's Sec. 4, as fixed-point int32 in the [3][N] layout."""
    N = L ** 3
    return gaussian_couplings_fixed(_gaussians(3 * N, seed, 2000 + realization)).reshape(3, N)


def gaussian_couplings_lattice(Lx: int, Ly: int, Lz: int, realization: int = 0, seed: int = 1) -> np.ndarray:
    N = Lx * Ly * Lz
    return gaussian_couplings_fixed(_gaussians(3 * N, seed, 2000 + realization)).reshape(3, N)


def gaussian_couplings_chain(N: int, realization: int = 0, seed: int = 1,
                             open_chain: bool = False) -> np.ndarray:
    """Gaussian couplings of a chain of N spins (periodic, as in the paper's
    1D study, unless open_chain), fixed-point int32; J[N-1] is the wrap bond."""
    J = gaussian_couplings_fixed(_gaussians(N, seed, 3000 + realization))
    if open_chain:
        J[N - 1] = 0
    return J


def uniform_ints(n: int, lo: int, hi: int, seed: int, stream: int = 0) -> np.ndarray:
    """n integers uniform in [lo, hi] (inclusive) by the multiply-shift map."""
    r = splitmix64(seed, n, stream=stream) >> np.uint64(32)
    span = np.uint64(hi - lo + 1)
    return (lo + ((r * span) >> np.uint64(32))).astype(np.int64)


def linear_schedule(beta_max: float, n_values: int) -> np.ndarray:
    """beta_k = beta_max * k / (n_values - 1), k = 0 .. n_values-1 (beta_0 = 0)."""
    K = n_values - 1
    return np.array([(beta_max * k) / K for k in range(n_values)], dtype=np.float64)


def default_capacity(R0: int) -> int:
    """Population cap R0 + 10 ceil(sqrt(R0)) + 64: about ten standard deviations
    of the Poisson population size above its target."""
    r = math.isqrt(int(R0))
    if r * r < R0:
        r += 1
    return int(R0) + 10 * r + 64


@dataclass
class RunSpec:
    """One annealing run: lattice, couplings realisation, seed and schedule."""
    dim: int
    L: int
    realization: int
    seed: int
    R0: int
    betas: np.ndarray
    theta: int
    coupling_seed: int = 1
    gaussian: bool = False      # Gaussian couplings (int32 fixed point) instead of +-1
    open_chain: bool = True     # 1D only: open (+-1 default) or periodic chain
    R_cap: int = 0              # population capacity (0: the library default for R0)

    @property
    def N(self) -> int:
        return self.L ** 3 if self.dim == 3 else self.L

    def couplings(self) -> np.ndarray:
        if self.gaussian:
            if self.dim == 3:
                return gaussian_couplings_3d(self.L, self.realization, self.coupling_seed)
            return gaussian_couplings_chain(self.L, self.realization, self.coupling_seed,
                                            open_chain=self.open_chain)
        if self.dim == 3:
            return couplings_3d(self.L, self.realization, self.coupling_seed)
        return couplings_chain(self.L, self.realization, self.coupling_seed,
                               open_chain=self.open_chain)

    @property
    def flips(self) -> int:
        """Attempted flips if the population stayed at R0: R0 * N * theta per step."""
        return self.R0 * self.N * self.theta * (len(self.betas) - 1)


# ---- the five workloads --------------------------------------------------------------

def config_small_3d() -> list[RunSpec]:
    """3D L=4 periodic, couplings from seed 1, R0 = 1000, 101 betas 0..5, theta = 10.
    Two independent runs (PA seeds 1 and 2) share the couplings so that the
    overlap q of Sec. 4 can be formed."""
    b = linear_schedule(5.0, 101)
    return [RunSpec(3, 4, 0, s, 1000, b, 10) for s in (1, 2)]


def config_l8() -> RunSpec:
    """3D L=8 periodic, R0 = 100000, 201 betas 0..5, theta = 10, one realisation."""
    return RunSpec(3, 8, 0, 1, 100_000, linear_schedule(5.0, 201), 10)


def config_batched(n_real: int = 16, runs_per_real: int = 64, n_betas: int = 101,
                   r_lo: int = 20_000, r_hi: int = 80_000) -> list[RunSpec]:
    """16 realisations x 64 runs, L in {6, 8, 10} by realisation, R0 uniform in
    [20000, 80000] (seed 3), 101 betas 0..5, theta = 10; PA seed (d << 8 | r)."""
    sizes = uniform_ints(n_real * runs_per_real, r_lo, r_hi, seed=3)
    b = linear_schedule(5.0, n_betas)
    out = []
    for d in range(n_real):
        L = (6, 8, 10)[d % 3]
        for r in range(runs_per_real):
            out.append(RunSpec(3, L, d, (d << 8) | r, int(sizes[d * runs_per_real + r]), b, 10))
    return out


def config_chain(n_seeds: int = 8, N: int = 4096, R0: int = 200_000) -> list[RunSpec]:
    """Open +-1 chain N = 4096, R0 = 200000, 401 betas 0..4, theta = 5, seeds 1..8
    (one disorder realisation per seed)."""
    b = linear_schedule(4.0, 401)
    return [RunSpec(1, N, s - 1, s, R0, b, 5) for s in range(1, n_seeds + 1)]


def paper_schedule_3d(n_approach: int = 20) -> np.ndarray:
    """Sec. 4, 3D: the paper's 100 temperatures 1/beta evenly spaced from 2 down
    to 0.2, reached from beta = 0 (where -beta F~ = N ln 2 anchors the free
    energy) by n_approach equal steps in beta up to 0.5; a single jump from
    beta = 0 to 0.5 would reweight by exp(-0.5 E) over an energy spread of
    ~40 at L = 8 and collapse the population."""
    T = np.array([(2.0 * (99 - k) + 0.2 * k) / 99 for k in range(100)])
    approach = [0.5 * k / n_approach for k in range(n_approach)]
    return np.concatenate([approach, 1.0 / T])


def paper_schedule_1d() -> np.ndarray:
    """Sec. 4, 1D: 19 steps evenly spaced in beta from 0 to 0.5, then 80
    evenly spaced in temperature from 2 down to 0.2 (100 betas, 99 steps)."""
    b = [0.5 * k / 19 for k in range(20)]
    b += [1.0 / ((2.0 * (80 - k) + 0.2 * k) / 80) for k in range(1, 81)]
    return np.array(b)


def config_gauss_3d(n_real: int = 25, runs_per_real: int = 50, R0: int = 2000,
                    theta: int = 100) -> list[RunSpec]:
    """The paper's 3D study (Sec. 4): L=8 periodic, Gaussian couplings, R=2000,
    the 3D temperature set, theta=100; 25 realisations x 50 independent runs
    (PA seed (d << 8 | r))."""
    b = paper_schedule_3d()
    return [RunSpec(3, 8, d, (d << 8) | r, R0, b, theta, gaussian=True)
            for d in range(n_real) for r in range(runs_per_real)]


def config_gauss_1d(n_real: int = 18, runs_per_real: int = 200, R0: int = 1000,
                    theta: int = 50) -> list[RunSpec]:
    """The paper's 1D study (Sec. 4): periodic chain N=256, Gaussian couplings,
    R=1000, the 1D temperature set, theta=50; 18 realisations x 200 runs."""
    b = paper_schedule_1d()
    return [RunSpec(1, 256, d, (d << 8) | r, R0, b, theta, gaussian=True, open_chain=False)
            for d in range(n_real) for r in range(runs_per_real)]


@dataclass
class Request:
    arrival_s: float
    spec: RunSpec


def serving_requests(n: int = 2000, rate_per_s: float = 10.0, seed: int = 5,
                     Ls=(4, 6, 8, 10, 12), r_lo: int = 10_000, r_hi: int = 200_000,
                     steps_lo: int = 51, steps_hi: int = 201, theta: int = 10) -> list[Request]:
    """Poisson stream of annealing requests: exponential inter-arrival gaps at
    the given rate, L uniform over Ls, R0 uniform in [r_lo, r_hi], number of
    betas uniform in [steps_lo, steps_hi], beta 0..5 linear."""
    u = (splitmix64(seed, n, stream=1) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    gaps = -np.log1p(-u) / rate_per_s
    t = np.cumsum(gaps)
    Lsel = uniform_ints(n, 0, len(Ls) - 1, seed, stream=2)
    R0s = uniform_ints(n, r_lo, r_hi, seed, stream=3)
    nb = uniform_ints(n, steps_lo, steps_hi, seed, stream=4)
    reqs = []
    for k in range(n):
        L = int(Ls[Lsel[k]])
        spec = RunSpec(3, L, k % 7, 10_000 + k, int(R0s[k]),
                       linear_schedule(5.0, int(nb[k])), theta)
        reqs.append(Request(float(t[k]), spec))
    return reqs
