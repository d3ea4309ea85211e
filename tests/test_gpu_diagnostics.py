"""On-device Sec. 3 estimators over groups of independent runs of a batch
(pa_batch_diagnostics, pa_batch_bootstrap) against the oracle's weighted average and variance on
the same per-step records: R-weighted E_bar and -beta F_bar within 1e-12
relative (log/exp of two math libraries), Var(-beta F~) within 1e-9 relative
(two-pass sums in different orders over values ~1e2..1e4 with variances
~1e-2..1e1)."""
import numpy as np
import pytest

from oracle import oracle as o
from paper_1006_0252_gb300 import inputs, pa

pytestmark = pytest.mark.gpu


def close(a, b, rtol):
    return abs(a - b) <= rtol * max(abs(a), abs(b), 1e-300)


def check_against_oracle(b, specs, M, count, target):
    diag = b.diagnostics(M, count)
    tr = b.trajectory(count)
    en = b.energy(count)
    G = len(specs) // M
    for g in range(G):
        sl = slice(g * M, (g + 1) * M)
        for k in range(count):
            Rw = np.array([s.R0 if k == 0 else target[r] for r, s in enumerate(specs)][sl], dtype=np.float64)
            m, f = o.weighted_average(tr["minus_beta_F"][sl, k], en["E_mean"][sl, k], Rw)
            v = o.variance(tr["minus_beta_F"][sl, k])
            assert close(diag["E_bar"][g, k], m, 1e-12), (g, k, diag["E_bar"][g, k], m)
            assert close(diag["minus_beta_F_bar"][g, k], f, 1e-12), (g, k)
            assert close(diag["var_minus_beta_F"][g, k], v, 1e-9) or abs(diag["var_minus_beta_F"][g, k] - v) < 1e-12


def check_bootstrap_against_oracle(b, specs, M, count, target, B, seed):
    """pa_batch_bootstrap against the oracle's bootstrap on the same records:
    the resample values agree to ~1e-13 relative, and their standard
    deviation (spread ~1e-3 of values ~1e3 for -beta F~) loses up to about
    four digits to cancellation, hence 1e-8."""
    boot = b.bootstrap(M, count, B=B, seed=seed)
    tr = b.trajectory(count)
    en = b.energy(count)
    for g in range(len(specs) // M):
        sl = slice(g * M, (g + 1) * M)
        for k in range(count):
            Rw = np.array([s.R0 if k == 0 else target[r] for r, s in enumerate(specs)][sl], dtype=np.float64)
            sm, sf = o.bootstrap(tr["minus_beta_F"][sl, k], en["E_mean"][sl, k], Rw, B=B, seed=seed)
            assert close(boot["sd_E_bar"][g, k], sm, 1e-8) or abs(boot["sd_E_bar"][g, k] - sm) < 1e-12, (g, k)
            assert close(boot["sd_minus_beta_F_bar"][g, k], sf, 1e-8) or \
                abs(boot["sd_minus_beta_F_bar"][g, k] - sf) < 1e-12, (g, k)


def test_pm_batch_groups_with_mixed_population_sizes():
    # 2 realisations x 5 runs, R0 differing inside each group (the R factor of Eq. (6))
    b5 = inputs.linear_schedule(5.0, 11)
    specs = [inputs.RunSpec(3, 6, d, (d << 8) | r, 400 + 150 * r, b5, 3) for d in range(2) for r in range(5)]
    b = pa.Batch(specs)
    b.run(b5[1:], thetas=3, use_graph=True)
    assert not b.sync().any()
    check_against_oracle(b, specs, 5, 11, [s.R0 for s in specs])
    check_bootstrap_against_oracle(b, specs, 5, 11, [s.R0 for s in specs], 64, 3)
    b.close()


def test_gaussian_batch_and_argument_errors():
    specs = inputs.config_gauss_1d(n_real=3, runs_per_real=4, R0=300, theta=2)
    betas = specs[0].betas[:9]
    b = pa.Batch(specs)
    b.run(betas[1:], thetas=2, use_graph=False)
    assert not b.sync().any()
    check_against_oracle(b, specs, 4, 9, [s.R0 for s in specs])
    check_bootstrap_against_oracle(b, specs, 4, 9, [s.R0 for s in specs], 37, 11)
    with pytest.raises(pa.PAError):
        b.diagnostics(5, 9)  # 12 runs do not split into groups of 5
    with pytest.raises(pa.PAError):
        b.diagnostics(4, 10)  # only 9 records
    with pytest.raises(pa.PAError):
        b.bootstrap(4, 10)  # only 9 records
    with pytest.raises(pa.PAError):
        b.bootstrap(4, 9, B=1)  # one resample has no spread
    b.close()


def test_batch_overlap_pairs_match_the_definition():
    """pa_batch_overlap against q = (1/N) sum s s' evaluated with numpy on the
    batch's own spins (replica k with replica k), for several pairs at once,
    +-1 and Gaussian runs."""
    for gaussian in (False, True):
        J = inputs.gaussian_couplings_3d(4, 0, 1) if gaussian else inputs.couplings_3d(4, 0, 1)
        b5 = inputs.linear_schedule(5.0, 9)
        specs = [inputs.RunSpec(3, 4, 0, s, 500 + 60 * s, b5, 3, gaussian=gaussian) for s in range(4)]
        assert all(np.array_equal(s.couplings(), J) for s in specs)  # one realisation
        b = pa.Batch(specs)
        b.run(b5[1:], thetas=3, use_graph=True)
        assert not b.sync().any()
        ra, rb = [0, 2, 0, 1], [1, 3, 3, 1]
        gamma, npairs = b.overlap(ra, rb, 0.2)
        for p in range(len(ra)):
            sa, sb = b.spins(ra[p], 4000), b.spins(rb[p], 4000)
            n = min(len(sa), len(sb))
            dot = (sa[:n].astype(np.int64) * sb[:n].astype(np.int64)).sum(axis=1)
            assert npairs[p] == n
            assert gamma[p] == np.count_nonzero(np.abs(dot.astype(np.float64)) < 0.2 * 64) / n
        assert gamma[3] == 0.0  # a run against itself: q = 1
        with pytest.raises(pa.PAError):
            b.overlap([0], [7])
        b.close()


def test_batch_overlap_histograms_match_the_definition():
    """pa_batch_overlap_hist against counts of (N q + N) / 2 evaluated with
    numpy on the batch's own spins, +-1 and Gaussian runs; the histogram's
    |q| < 0.2 part is the Gamma of pa_batch_overlap."""
    for gaussian in (False, True):
        b5 = inputs.linear_schedule(4.0, 7)
        specs = [inputs.RunSpec(3, 4, 0, s, 400 + 70 * s, b5, 3, gaussian=gaussian) for s in range(4)]
        b = pa.Batch(specs)
        b.run(b5[1:], thetas=3, use_graph=True)
        assert not b.sync().any()
        ra, rb = [0, 1, 2, 3], [1, 2, 3, 3]
        h = b.overlap_hist(ra, rb)
        gamma, npairs = b.overlap(ra, rb, 0.2)
        N = 64
        for p in range(len(ra)):
            sa, sb = b.spins(ra[p], 4000), b.spins(rb[p], 4000)
            n = min(len(sa), len(sb))
            dot = (sa[:n].astype(np.int64) * sb[:n].astype(np.int64)).sum(axis=1)
            want = np.bincount((N + dot) // 2, minlength=N + 1)
            assert np.array_equal(h[p], want), p
            q = (2 * np.arange(N + 1) - N) / N
            assert h[p][np.abs(q) < 0.2].sum() == round(gamma[p] * npairs[p])
        assert h[3][N] == npairs[3]  # a run against itself: q = 1 only
        with pytest.raises(pa.PAError):
            b.overlap_hist([0], [9])
        b.close()
