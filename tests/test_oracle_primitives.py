"""Pins for the oracle's primitives (CPU only).

Each primitive is checked against something other than itself: Philox
against Triton's independent Philox4x32-10 (run on the CPU interpreter),
pexp and the Metropolis thresholds against mpmath at 120-bit precision, the
Poisson inverse-CDF walk against scipy's pmf on a stratified grid."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as o

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def _k(out, c0p, c1p, c2p, c3p, seed, n, BLOCK: tl.constexpr):
    offs = tl.arange(0, BLOCK)
    m = offs < n
    c0 = tl.load(c0p + offs, mask=m)
    c1 = tl.load(c1p + offs, mask=m)
    c2 = tl.load(c2p + offs, mask=m)
    c3 = tl.load(c3p + offs, mask=m)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out + offs * 4 + 0, a, mask=m)
    tl.store(out + offs * 4 + 1, b, mask=m)
    tl.store(out + offs * 4 + 2, c, mask=m)
    tl.store(out + offs * 4 + 3, d, mask=m)

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    n = len(ctrs)
    B = 1
    while B < n:
        B *= 2
    cols = [torch.tensor([c[j] for c in ctrs] + [0] * (B - n), dtype=torch.int64).to(torch.uint32) for j in range(4)]
    out = torch.zeros(4 * B, dtype=torch.uint32)
    _k[(1,)](out, *cols, seed, n, BLOCK=B)
    v = out.to(torch.int64) & 0xFFFFFFFF
    res.append([[int(v[4 * i + j]) for j in range(4)] for i in range(n)])
print(json.dumps(res))
"""


def test_philox_matches_triton_reference():
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    seeds = [0, 1, 0xFFFFFFFFFFFFFFFF, 0x243F6A8885A308D3, int(rng.integers(0, 2**63))]
    cases = []
    for s in seeds:
        ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 0x3C000001]]
        ctrs += [[int(v) for v in rng.integers(0, 2**32, size=4, dtype=np.uint64)] for _ in range(13)]
        cases.append([s, ctrs])
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    ref = json.loads(p.stdout.strip().splitlines()[-1])
    for (s, ctrs), outs in zip(cases, ref):
        key = (s & 0xFFFFFFFF, s >> 32)
        for c, expect in zip(ctrs, outs):
            assert list(o.philox(c, key)) == expect, (hex(s), c)


def test_philox_avalanche():
    # one flipped counter bit changes about half of the 128 output bits
    base = o.philox((5, 6, 7, 8), (9, 10))
    flips = []
    for w in range(4):
        for b in range(0, 32, 7):
            c = [5, 6, 7, 8]
            c[w] ^= 1 << b
            out = o.philox(c, (9, 10))
            flips.append(sum(bin(x ^ y).count("1") for x, y in zip(base, out)))
    assert 50 < np.mean(flips) < 78


def _ulp_err(got: float, want) -> float:
    import mpmath as mp
    w = float(want)
    if w == 0.0:
        return abs(got) / 5e-324
    return float(abs(mp.mpf(got) - want) / np.spacing(w))


def test_pexp_within_two_ulp_of_exact():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(11)
    xs = list(-rng.uniform(0, 1, 3000)) + list(-rng.uniform(0, 40, 3000)) + \
        list(-rng.uniform(0, 708, 3000)) + [-0.0, -1e-300, -1e-17, -0.5 * math.log(2),
                                            -math.log(2), -1.0, -10.0, -700.0, -708.39]
    worst = 0.0
    for x in xs:
        got = o.pexp(x)
        worst = max(worst, _ulp_err(got, mp.exp(mp.mpf(x))))
    assert worst <= 2.0, worst


def test_pexp_subnormal_range_and_limits():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    assert o.pexp(0.0) == 1.0 and o.pexp(-0.0) == 1.0
    assert o.pexp(-1e6) == 0.0 and o.pexp(float("-inf")) == 0.0
    for x in np.linspace(-745.0, -708.5, 200):
        want = float(mp.exp(mp.mpf(x)))
        got = o.pexp(float(x))
        assert abs(got - want) <= 2 * 5e-324 + 4 * np.spacing(want), x
    prev = 2.0
    for x in np.linspace(0.0, -3.0, 20001):  # monotone on a fine grid
        v = o.pexp(float(x))
        assert v <= prev
        prev = v


def test_pexp_functional_equation():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        # multiples of 2^-10 so that a + b is exact
        a = -float(rng.integers(0, 300 * 1024)) / 1024.0
        b = -float(rng.integers(0, 300 * 1024)) / 1024.0
        lhs = o.pexp(a) * o.pexp(b)
        rhs = o.pexp(a + b)
        assert abs(lhs - rhs) <= 8 * np.spacing(rhs) + 1e-300


def test_metropolis_threshold_is_floor_of_scaled_boltzmann_factor():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    for beta in np.linspace(0.0, 5.0, 101):
        for dE in range(2, 13, 2):
            t = o.threshold(float(beta), dE)
            exact = mp.exp(-mp.mpf(float(beta) * dE)) * 2 ** 32  # product rounded as specified
            fl = int(mp.floor(exact))
            if fl >= 2 ** 32:
                assert t == 2 ** 32 - 1
                continue
            if abs(exact - fl) > 1e-5 and abs(exact - fl - 1) > 1e-5:
                assert t == fl, (beta, dE, t, fl)
            else:
                assert abs(t - fl) <= 1
    assert o.threshold(0.0, 4) == 2 ** 32 - 1


def test_u53():
    assert o.u53(0, 0) == 0.0
    assert o.u53(0x80000000, 0) == 0.5
    assert o.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert o.u53(0, 0x800) == 2.0 ** -53


@pytest.mark.parametrize("am", [1e-3, 0.5, 1.0, 2.7, 10.0, 31.99])
def test_poisson_piece_matches_pmf_on_stratified_grid(am):
    st = pytest.importorskip("scipy.stats")
    n = 40000
    p0 = o.pexp(-am)
    ks = np.array([o.poisson_piece((i + 0.5) / n, am, p0) for i in range(n)])
    counts = np.bincount(ks, minlength=int(am * 4 + 30))
    pmf = st.poisson.pmf(np.arange(len(counts)), am)
    # stratified u: count_k = n * pmf_k up to one grid cell at each end
    assert np.max(np.abs(counts - n * pmf)) <= 2.0 + 1e-9 * n


def test_poisson_piece_degenerate_inputs():
    assert o.poisson_piece(0.0, 0.0, 1.0) == 0
    assert o.poisson_piece(0.999999, 0.0, 1.0) == 0
    assert o.poisson_piece(1.0 - 2.0 ** -53, 30.0, o.pexp(-30.0)) <= 512


def test_weighted_average_closed_forms():
    # equal free energies: plain mean (Eq. (5) with equal Eq. (6) weights)
    m, f = o.weighted_average([2.0, 2.0, 2.0], [1.0, 2.0, 6.0])
    assert abs(m - 3.0) < 1e-15 and abs(f - 2.0) < 1e-15
    # e^x ratio 1:3 -> weights 1/4, 3/4
    m, f = o.weighted_average([0.0, math.log(3.0)], [4.0, 8.0])
    assert abs(m - 7.0) < 1e-14
    assert abs(f - math.log(2.0)) < 1e-15  # ln[(1 + 3)/2], Eq. (7)
    # R^(r) factor of Sec. 3 cancels the 1:3 free-energy ratio
    m, _ = o.weighted_average([0.0, math.log(3.0)], [4.0, 8.0], R=[3.0, 1.0])
    assert abs(m - 6.0) < 1e-14
    # large arguments do not overflow
    m, f = o.weighted_average([1e4, 1e4 + math.log(3.0)], [4.0, 8.0])
    assert abs(m - 7.0) < 1e-12 and abs(f - (1e4 + math.log(2.0))) < 1e-9


def test_weighted_average_against_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    rng = np.random.default_rng(5)
    x = rng.normal(3000.0, 0.8, 64)
    A = rng.normal(-800.0, 3.0, 64)
    R = rng.integers(20000, 80000, 64).astype(float)
    m, f = o.weighted_average(x, A, R)
    ex = [mp.mpf(float(v)) for v in x]
    w = [mp.mpf(float(r)) * mp.exp(v) for v, r in zip(ex, R)]
    want_m = sum(wi * mp.mpf(float(a)) for wi, a in zip(w, A)) / sum(w)
    want_f = mp.log(sum(mp.exp(v) for v in ex) / len(ex))
    assert abs(m - float(want_m)) <= 1e-12 * abs(float(want_m))
    assert abs(f - float(want_f)) <= 1e-12 * abs(float(want_f))


def test_pair_weighted_average_closed_forms():
    """Sec. 4, Eq. (11): a pair's weight is e^{x1 + x2}, both runs' free energies."""
    # the second run alone sets a 1:3 ratio -> weights 1/4, 3/4
    m, f = o.weighted_average_pairs([0.0, 0.0], [0.0, math.log(3.0)], [4.0, 8.0])
    assert abs(m - 7.0) < 1e-14 and abs(f - math.log(2.0)) < 1e-15
    # the first run alone sets it (the order of the two runs does not matter)
    m, _ = o.weighted_average_pairs([0.0, math.log(3.0)], [0.0, 0.0], [4.0, 8.0])
    assert abs(m - 7.0) < 1e-14
    # the two runs cancel: equal pair weights, plain mean
    m, f = o.weighted_average_pairs([math.log(3.0), 0.0], [0.0, math.log(3.0)], [4.0, 8.0])
    assert abs(m - 6.0) < 1e-14 and abs(f - math.log(3.0)) < 1e-15
    # population factors R1 R2 of Sec. 3: 2:6 = 1:3
    m, _ = o.weighted_average_pairs([0.0, 0.0], [0.0, 0.0], [4.0, 8.0], R1=[2.0, 1.0], R2=[1.0, 6.0])
    assert abs(m - 7.0) < 1e-14
    # x2 = 0 everywhere: the single-run estimator of Eqs. (5)-(7)
    rng = np.random.default_rng(3)
    x = rng.normal(1500.0, 0.7, 33)
    A = rng.normal(-200.0, 2.0, 33)
    m, f = o.weighted_average_pairs(x, np.zeros(33), A)
    m1, f1 = o.weighted_average(x, A)
    assert abs(m - m1) <= 1e-13 * abs(m1) and abs(f - f1) <= 1e-13 * abs(f1)


def test_pair_weighted_average_against_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    rng = np.random.default_rng(8)
    M = 50
    x1 = rng.normal(2800.0, 0.6, M)
    x2 = rng.normal(2800.0, 0.6, M)
    G = rng.uniform(0.0, 0.3, M)
    R1 = rng.integers(1000, 3000, M).astype(float)
    R2 = rng.integers(1000, 3000, M).astype(float)
    m, f = o.weighted_average_pairs(x1, x2, G, R1, R2)
    e = [mp.exp(mp.mpf(float(a)) + mp.mpf(float(b))) for a, b in zip(x1, x2)]
    w = [mp.mpf(float(r1)) * mp.mpf(float(r2)) * ei for r1, r2, ei in zip(R1, R2, e)]
    want_m = sum(wi * mp.mpf(float(g)) for wi, g in zip(w, G)) / sum(w)
    want_f = mp.log(sum(e) / M)
    assert abs(m - float(want_m)) <= 1e-12 * abs(float(want_m))
    assert abs(f - float(want_f)) <= 1e-12 * abs(float(want_f))


def test_variance_and_bootstrap():
    assert abs(o.variance([1.0, 2.0, 3.0, 4.0]) - 5.0 / 3.0) < 1e-15
    sm, sf = o.bootstrap([1.0] * 10, [5.0] * 10, B=50, seed=1)
    assert sm == 0.0 and sf == 0.0
    rng = np.random.default_rng(9)
    A = rng.normal(0, 1, 400)
    sm, _ = o.bootstrap(np.zeros(400), A, B=200, seed=2)
    # equal weights: bootstrap std of the mean ~ std(A)/sqrt(M)
    assert abs(sm - A.std(ddof=1) / 20.0) < 0.25 * A.std(ddof=1) / 20.0
