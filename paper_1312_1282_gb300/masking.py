"""Load masking on one GPU: the analysis of configurations overlapped with the generation of the
next ones (the paper's Sec. 4.2, Eqs. (serialtime), (maskedtime), (optimalGPU), and its
demonstration in Sec. 7.1).

In the paper the GPU generates macroupdates while the CPU analyses earlier configurations.  Here
both run on the GPU: the generation (qmc_sweep) on one stream, the analysis (qmc_local_energy and
qmc_pair_hist, the local energy and the g(r) histogram of Sec. 5.4) on a second stream, on
snapshots of the configurations.  The analysis kernels occupy SMs the generation leaves idle --
few walkers use few SMs, one CTA per walker, or a cluster of CTAs per walker at large N -- so
one analysis every m macroupdates costs t_step = max(m t_G, t_A) instead of t_A + m t_G.

The schedule (this module only orders work on streams; every step runs in the library's kernels):
generation stream: sweep m macroupdates, wait until snapshot buffer k mod 2 is free, copy the
configuration into it, record "ready"; analysis stream: wait for "ready", run the analyses on
the snapshot, record "free".  Two snapshot buffers let the generation run one analysis ahead.
The chains, the energies and the histograms are those of the sequential schedule, bit for bit
(the same kernels on the same configurations).
"""
from __future__ import annotations

import torch

from . import qmc_local_energy, qmc_pair_hist, qmc_sweep

__all__ = ["run_schedule"]


def run_schedule(d, opt, pos, logpsi, sweeps, accum, seed, m, count, energies=None, hist=None, nbins=0, rmax=0.0,
                 masked=True, gen_stream=None, ana_stream=None):
    """count analyses, one after every m macroupdates of the walker batch `d`.

    energies: optional device [count, W, 5] float64 tensor, row k receives qmc_local_energy of
    the configuration after macroupdate (k + 1) m.  hist: optional device [W, nbins] int64
    tensor, qmc_pair_hist of every analysed configuration is added to it (bins of rmax / nbins).
    masked: analyses on a second stream, overlapped with the generation (else one stream, in
    order).  Returns after enqueueing; synchronise `gen_stream` and `ana_stream` (or the device)
    before reading the outputs."""
    gen = gen_stream or torch.cuda.current_stream()
    if not masked:
        for k in range(count):
            qmc_sweep(d, opt, pos, logpsi, sweeps, seed, m, 0, accum, gen)
            if energies is not None:
                qmc_local_energy(d, opt, pos, energies[k], gen)
            if hist is not None:
                qmc_pair_hist(d, opt, pos, nbins, rmax, hist, gen)
        return
    ana = ana_stream or torch.cuda.Stream()
    ana.wait_stream(gen)  # the outputs and the starting state are ordered before the first analysis
    with torch.cuda.stream(gen):  # the snapshot buffers belong to the generation stream
        snaps = [torch.empty_like(pos), torch.empty_like(pos)]
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    free = [torch.cuda.Event(), torch.cuda.Event()]
    for k in range(count):
        b = k % 2
        qmc_sweep(d, opt, pos, logpsi, sweeps, seed, m, 0, accum, gen)
        if k >= 2:
            gen.wait_event(free[b])  # the analysis of configuration k - 2 has read buffer b
        with torch.cuda.stream(gen):
            snaps[b].copy_(pos, non_blocking=True)
        ready[b].record(gen)
        ana.wait_event(ready[b])
        if energies is not None:
            qmc_local_energy(d, opt, snaps[b], energies[k], ana)
        if hist is not None:
            qmc_pair_hist(d, opt, snaps[b], nbins, rmax, hist, ana)
        free[b].record(ana)
    # the snapshot buffers stay alive until the analysis stream has used them
    for t in snaps:
        t.record_stream(ana)
    gen.wait_stream(ana)  # callers that synchronise the generation stream see every analysis
