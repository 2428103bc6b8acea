"""Host-side analysis of sampled observables: autocorrelation, the error of a correlated mean and
the choice of the number m of macroupdates between analyses (Sec. 4 of the paper, "Load
masking, optimal execution and the modified Amdahl law").

A macroupdate is N single-particle moves (one qmc_sweep sweep).  t_G is the time of one
macroupdate, t_A the time of one analysis (here the on-GPU local energy of every walker) and
alpha = t_A / t_G.  Everything here is plain numpy on small host arrays (a few thousand samples
per walker); the samples themselves come from the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np


def autocorrelation(series: np.ndarray, kmax: int | None = None) -> np.ndarray:
    """R(k), k = 0..kmax, of Sec. 4.1: sum_i (A_i - <A>)(A_{i+k} - <A>) / sum_i (A_i - <A>)^2.

    series: [S] or [W, S] (W independent chains of S samples); with several chains the numerator
    and denominator are summed over chains, each chain about its own mean."""
    a = np.atleast_2d(np.asarray(series, dtype=np.float64))
    S = a.shape[1]
    if S < 2:
        raise ValueError("need at least two samples per chain")
    kmax = S - 1 if kmax is None else min(int(kmax), S - 1)
    d = a - a.mean(axis=1, keepdims=True)
    den = float((d * d).sum())
    if den == 0.0:
        r = np.zeros(kmax + 1)
        r[0] = 1.0
        return r
    # all lags at once through a zero-padded FFT of each chain
    nfft = 1 << (2 * S - 1).bit_length()
    f = np.fft.rfft(d, n=nfft, axis=1)
    acf = np.fft.irfft(f * np.conj(f), n=nfft, axis=1)[:, :kmax + 1].sum(axis=0)
    return acf / den


def autocorr_time(series: np.ndarray, c: float = 6.0) -> float:
    """m_c = sum_{k>=1} R(k) (Sec. 4.1), the sum cut at the first lag M >= c (1 + 2 m_c(M))
    (Sokal's self-consistent window; the tail past a few autocorrelation times is noise)."""
    a = np.atleast_2d(np.asarray(series, dtype=np.float64))
    r = autocorrelation(a)
    partial = np.cumsum(r[1:])  # partial[M-1] = sum_{k=1..M} R(k)
    for M in range(1, len(r)):
        if M >= c * (1.0 + 2.0 * partial[M - 1]):
            return float(partial[M - 1])
    return float(partial[-1])


def reblocking(series: np.ndarray) -> list[tuple[int, float]]:
    """Blocking analysis (Flyvbjerg and Petersen): for block sizes B = 1, 2, 4, ... with at least
    8 blocks per chain, the ratio B var(block means) / var(samples).  Its plateau is
    1 + 2 m_c, the inflation of the squared error of the mean (Eq. CorrelatedError with m = 1)."""
    a = np.atleast_2d(np.asarray(series, dtype=np.float64))
    W, S = a.shape
    v0 = float(a.var(axis=1, ddof=1).mean())
    out = []
    B = 1
    while S // B >= 8:
        nb = S // B
        blocks = a[:, :nb * B].reshape(W, nb, B).mean(axis=2)
        out.append((B, B * float(blocks.var(axis=1, ddof=1).mean()) / v0 if v0 > 0 else 1.0))
        B *= 2
    return out


def correlated_error(sigma0: float, n_samples: float, m_c: float, m: float) -> float:
    """Eq. CorrelatedError: error of the mean of n_samples analyses taken every m macroupdates
    (any number of independent chains)."""
    return sigma0 / math.sqrt(n_samples) * math.sqrt(1.0 + 2.0 * m_c / m)


def optimal_m_sequential(m_c: float, alpha: float) -> float:
    """Eq. optimalCPU: m = sqrt(2 m_c alpha) when generation and analysis share one unit
    (t_step = t_A + m t_G, Eq. serialtime)."""
    return math.sqrt(2.0 * m_c * alpha)


def optimal_m_masked(alpha: float) -> float:
    """Eq. optimalGPU: m = alpha when the analysis overlaps generation
    (t_step = max(m t_G, t_A), Eq. maskedtime)."""
    return float(alpha)


def time_per_error(m: float, m_c: float, t_G: float, t_A: float, masked: bool = False) -> float:
    """Time to reach unit error for unit sigma0: (1 + 2 m_c / m) t_step, with t_step from
    Eq. serialtime or Eq. maskedtime."""
    t_step = max(m * t_G, t_A) if masked else t_A + m * t_G
    return (1.0 + 2.0 * m_c / m) * t_step


def penalty_seq_m1(m_c: float, alpha: float) -> float:
    """Eq. penaltyseq: t_seq(m = 1) / t_seq(optimal m)."""
    return (alpha + 1.0) * (1.0 + 2.0 * m_c) / (alpha * (1.0 + math.sqrt(2.0 * m_c / alpha)) ** 2)


def penalty_mask_m1(m_c: float, alpha: float) -> float:
    """The masked counterpart of Eq. penaltyseq: t_mask(m = 1) / t_mask(m = alpha), alpha >= 1."""
    return alpha * (1.0 + 2.0 * m_c) / (alpha + 2.0 * m_c)


def integer_m(m_real: float, m_c: float, t_G: float, t_A: float, masked: bool = False) -> int:
    """The better of the two integers around a real-valued optimum (at least 1)."""
    lo = max(1, int(math.floor(m_real)))
    cands = {lo, lo + 1}
    return min(cands, key=lambda m: time_per_error(m, m_c, t_G, t_A, masked))
