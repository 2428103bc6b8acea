"""Walker sharding across processes (one process per GPU) and the host-side reduction of the
per-walker FP64 accumulators.

Walkers are independent Markov chains (the paper, Sec. 4.1: independent chains are as good as
one long one), so a multi-GPU run is a set of replicas: each rank advances its own walkers,
whose Philox walker ids are disjoint, and no data moves during sweeps.  The only exchange is
one sum of accumulator totals at the end of a block, done here on the host through
torch.distributed (gloo or nccl).
"""
from __future__ import annotations

import math

import torch
import torch.distributed as dist


def walker_ids(rank: int, world: int, per_rank: int) -> list[int]:
    """Global walker ids of one rank: a contiguous, disjoint range per rank."""
    if not (0 <= rank < world) or per_rank <= 0:
        raise ValueError("bad rank/world/per_rank")
    return list(range(rank * per_rank, (rank + 1) * per_rank))


def block_stats(accum: torch.Tensor, n_atoms: torch.Tensor | float, group=None) -> dict:
    """Energy per atom over all walkers of all ranks, with the standard error across walkers.

    accum: [W, >= 8] per-walker sums {E_L, E_L^2, V, T_L, T_PB, T_F, samples, accepted, ...} (this
    rank; the ln psi drift fields that follow are not used here).
    Each walker's time average is one independent estimate (Eq. CorrelatedError with independent
    chains); their spread gives the error bar.  With torch.distributed initialised, the sums
    over walkers are all-reduced (float64, on the host)."""
    a = accum.detach().double().cpu()
    n = torch.as_tensor(n_atoms, dtype=torch.float64).expand(a.shape[0])
    ns = a[:, 6].clamp(min=1)
    e = a[:, 0] / ns / n
    v = a[:, 2] / ns / n
    t = a[:, 3] / ns / n
    tpb = a[:, 4] / ns / n
    tf = a[:, 5] / ns / n
    moves = (a[:, 6] > 0).double()  # walkers with samples
    sums = torch.stack([moves.sum(), (e * moves).sum(), (e * e * moves).sum(), (v * moves).sum(), (t * moves).sum(),
                        (tpb * moves).sum(), (tf * moves).sum(), a[:, 7].sum()])
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "nccl":
            s = sums.cuda()
            dist.all_reduce(s, group=group)
            sums = s.cpu()
        else:
            dist.all_reduce(sums, group=group)
    W = sums[0].item()
    mean = sums[1].item() / W
    var = max(sums[2].item() / W - mean * mean, 0.0)
    return {
        "walkers": int(W),
        "E_per_atom": mean,
        "E_err": math.sqrt(var / max(W - 1, 1)),
        "V_per_atom": sums[3].item() / W,
        "T_per_atom": sums[4].item() / W,
        "TPB_per_atom": sums[5].item() / W,
        "TF_per_atom": sums[6].item() / W,
        "accepted": sums[7].item(),
    }
