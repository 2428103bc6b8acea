"""Host analysis of Sec. 4 (autocorrelation, correlated error, optimal m), pinned to closed forms:
an AR(1) chain A_{i+1} = phi A_i + noise has R(k) = phi^k and m_c = phi / (1 - phi); the optimal m
and the penalty ratios are checked against a brute-force minimisation of the time to error."""
import math

import numpy as np
import pytest

from paper_1312_1282_gb300 import analysis as an


def _ar1(phi, W, S, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((W, S))
    a = np.empty((W, S))
    a[:, 0] = e[:, 0] / math.sqrt(1 - phi * phi)  # stationary start
    for i in range(1, S):
        a[:, i] = phi * a[:, i - 1] + e[:, i]
    return a


@pytest.mark.parametrize("phi", [0.0, 0.5, 0.8])
def test_ar1_autocorrelation_and_time(phi):
    a = _ar1(phi, 64, 4096, 7)
    r = an.autocorrelation(a, 8)
    assert r[0] == pytest.approx(1.0)
    np.testing.assert_allclose(r[:6], phi ** np.arange(6), atol=0.01)
    assert an.autocorr_time(a) == pytest.approx(phi / (1 - phi), abs=0.05 + 0.03 * phi / (1 - phi))


def test_autocorrelation_matches_direct_sum():
    a = np.random.default_rng(3).standard_normal((3, 50)).cumsum(axis=1)
    d = a - a.mean(axis=1, keepdims=True)
    den = (d * d).sum()
    direct = [sum((d[w, :50 - k] * d[w, k:]).sum() for w in range(3)) / den for k in range(10)]
    np.testing.assert_allclose(an.autocorrelation(a, 9), direct, rtol=1e-12, atol=1e-14)


def test_reblocking_plateau_is_one_plus_two_mc():
    phi = 0.6
    a = _ar1(phi, 32, 8192, 11)
    blocks = dict(an.reblocking(a))
    assert blocks[1] == pytest.approx(1.0, abs=1e-12)
    assert blocks[64] == pytest.approx((1 + phi) / (1 - phi), rel=0.08)


def test_correlated_error_matches_sampled_spread():
    """Eq. CorrelatedError: std of chain means of S/m samples taken every m steps."""
    phi, W, S, m = 0.7, 400, 4096, 4
    a = _ar1(phi, W, S, 5)
    sub = a[:, ::m]
    sigma0 = 1 / math.sqrt(1 - phi * phi)
    mc = phi / (1 - phi)
    pred = an.correlated_error(sigma0, sub.shape[1], mc, m)
    got = sub.mean(axis=1).std(ddof=1)
    assert got == pytest.approx(pred, rel=0.1)


@pytest.mark.parametrize("mc,alpha", [(0.5, 0.3), (3.0, 0.5), (20.0, 2.0), (1.0, 10.0)])
def test_optimal_m_and_penalties_by_brute_force(mc, alpha):
    tG, tA = 1.0, alpha
    ms = np.linspace(0.01, 200, 400001)
    t_seq = (1 + 2 * mc / ms) * (tA + ms * tG)
    m_star = ms[np.argmin(t_seq)]
    assert an.optimal_m_sequential(mc, alpha) == pytest.approx(m_star, abs=2e-3)
    assert an.penalty_seq_m1(mc, alpha) == pytest.approx(
        an.time_per_error(1, mc, tG, tA) / t_seq.min(), rel=1e-6)
    t_mask = (1 + 2 * mc / ms) * np.maximum(ms * tG, tA)
    assert an.optimal_m_masked(alpha) == pytest.approx(ms[np.argmin(t_mask)], abs=2e-3)
    if alpha >= 1:
        assert an.penalty_mask_m1(mc, alpha) == pytest.approx(
            an.time_per_error(1, mc, tG, tA, masked=True) / t_mask.min(), rel=1e-4)  # kink at m = alpha
    m_int = an.integer_m(an.optimal_m_sequential(mc, alpha), mc, tG, tA)
    best = min(range(1, 400), key=lambda m: an.time_per_error(m, mc, tG, tA))
    assert m_int == best


def test_penalty_limits():
    """Strong autocorrelation: P_seq(m=1) -> alpha + 1.  The bounds of Sec. 4.2 on P_seq(m) and
    P_mask(m) hold against the best m >= 1 (an analysis cannot come more often than every
    macroupdate, so a real-valued optimum below 1 is read as m = 1)."""
    assert an.penalty_seq_m1(1e9, 3.0) == pytest.approx(4.0, rel=1e-3)
    for mc in (0.1, 1.0, 10.0):
        for alpha in (0.5, 2.0, 8.0):
            best_seq = an.time_per_error(max(1.0, an.optimal_m_sequential(mc, alpha)), mc, 1, alpha)
            best_mask = an.time_per_error(max(1.0, an.optimal_m_masked(alpha)), mc, 1, alpha, masked=True)
            for m in (1, 2, 5, 13):
                p = an.time_per_error(m, mc, 1, alpha) / best_seq
                assert 1 - 1e-12 <= p < 1 + max(alpha / m, (m - 1) / (alpha + 1))
                if alpha >= 1:
                    p = an.time_per_error(m, mc, 1, alpha, masked=True) / best_mask
                    assert 1 - 1e-12 <= p <= max(alpha / m, m / alpha)


def test_pair_correlation_of_an_ideal_gas_is_one():
    """pair_correlation's normalisation: uniformly random points (an ideal gas) have g(r) = 1; the
    counts come from the oracle's brute-force histogram."""
    import oracle
    from paper_1312_1282_gb300 import pair_correlation
    n, L, nbins, samples = 200, 20.0, 10, 40
    rng = np.random.default_rng(12)
    counts = np.zeros(nbins)
    for _ in range(samples):
        counts += oracle.pair_hist(rng.uniform(0, L, size=(3, n)), L, nbins, L / 2)
    r, g = pair_correlation(counts, n, L, L / 2, samples)
    assert np.allclose(r, (np.arange(nbins) + 0.5) * L / 2 / nbins)
    # Poisson error of each bin's count, relative: 1/sqrt(count)
    err = 1 / np.sqrt(np.maximum(counts, 1))
    assert np.all(np.abs(g[1:] - 1) < 4 * err[1:] + 0.01), g
