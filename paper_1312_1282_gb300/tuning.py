"""Trial-step tuning to a target acceptance.

The paper's sample run (Sec. 7) uses an RMS trial step of 0.5 rho^(-1/3), quoted at about 40 %
acceptance; the benchmark workloads aim at 50 % with the cube proposal.  The acceptance of
single-particle moves falls monotonically as the step grows, so the step is found by bisection on
short probes of the chains themselves.  Each probe is a `qmc_sweep`
call (the moves run in the CUDA kernels); this module only reads the accepted counts and moves
the bracket.
"""
from __future__ import annotations

import torch

from . import qmc_sweep

__all__ = ["tune_step"]


def tune_step(descs_of, opt, pos, logpsi, sweep, seed, accum, target=0.5, lo=0.1, hi=3.0, step=0.8, probes=5,
              sweeps=4, stream=None):
    """Bisect the trial step of a walker batch to an acceptance near `target`.

    descs_of(step) returns the batch's descriptor array with that step for every walker.  Each of
    the `probes` probes zeroes `accum`, advances the chains by `sweeps` sweeps at the current step
    (so the probes are part of equilibration; ln psi and the sweep counters advance as in any
    sweep), and takes the acceptance as accepted moves / (sweeps x sum of n).  A probe above the
    target raises the lower end of the bracket [lo, hi], any other lowers the upper end, and the
    next step is the bracket's midpoint.  Returns (step, acceptances): the midpoint after the
    last probe, and the acceptance each probe measured.  `accum` holds the last probe's sums.
    """
    if not (0.0 < target < 1.0):
        raise ValueError("target acceptance must lie in (0, 1)")
    if not (0.0 < lo < hi):
        raise ValueError("the step bracket must satisfy 0 < lo < hi")
    if probes < 1 or sweeps < 1:
        raise ValueError("probes and sweeps must be >= 1")
    rates = []
    for _ in range(probes):
        d = descs_of(step)
        moves = sweeps * sum(int(d[w].n) for w in range(len(d)))
        accum.zero_()
        qmc_sweep(d, opt, pos, logpsi, sweep, seed, sweeps, 0, accum, stream)
        if stream is not None:  # the read below is ordered on torch's current stream only
            torch.cuda.synchronize()
        rate = accum[:, 7].sum().item() / moves
        rates.append(rate)
        if rate > target:
            lo = step
        else:
            hi = step
        step = 0.5 * (lo + hi)
    return step, rates
