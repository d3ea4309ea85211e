"""Exact enumeration of tiny Ising spin glasses, written independently of the
oracle: the bond list is rebuilt from the coupling layout here and energies
are evaluated for all 2^N states at once with numpy."""
from __future__ import annotations

import numpy as np


def bonds_3d(J: np.ndarray, Lx: int, Ly: int, Lz: int, periodic_mask: int):
    """(i, j, J) for every stored nonzero bond of a box with the [3][N] layout."""
    N = Lx * Ly * Lz
    out = []
    ext = (Lx, Ly, Lz)
    for z in range(Lz):
        for y in range(Ly):
            for x in range(Lx):
                i = x + Lx * (y + Ly * z)
                c = [x, y, z]
                for d in range(3):
                    if c[d] == ext[d] - 1 and not (periodic_mask >> d) & 1:
                        continue
                    n = list(c)
                    n[d] = (c[d] + 1) % ext[d]
                    j = n[0] + Lx * (n[1] + Ly * n[2])
                    val = int(J.reshape(-1)[d * N + i])
                    if val != 0:
                        out.append((i, j, val))
    return out


def bonds_chain(J: np.ndarray):
    N = len(J)
    return [(i, (i + 1) % N, int(J[i])) for i in range(N) if J[i] != 0]


def all_states(N: int) -> np.ndarray:
    """sigma[s, i] = +1/-1 for s in 0 .. 2^N - 1 (bit i of s set means -1)."""
    s = np.arange(2 ** N, dtype=np.int64)[:, None]
    bits = (s >> np.arange(N)[None, :]) & 1
    return (1 - 2 * bits).astype(np.int64)


def energies(bonds, N: int) -> np.ndarray:
    sig = all_states(N)
    E = np.zeros(sig.shape[0], dtype=np.int64)
    for i, j, Jb in bonds:
        E += Jb * sig[:, i] * sig[:, j]
    return E


def exact(E: np.ndarray, beta: float):
    """(ln Z, <E>, Var E) at inverse temperature beta from the state energies."""
    x = -beta * E.astype(np.float64)
    m = x.max()
    w = np.exp(x - m)
    Z = w.sum()
    p = w / Z
    Em = float((p * E).sum())
    return float(m + np.log(Z)), Em, float((p * (E - Em) ** 2).sum())
