"""An uneven batch in one persistent launch, captured in a CUDA graph and replayed.

qmc_sweep of a batch with more walkers than SMs launches the walker-queue initialisation and the
persistent sweep kernel (FP64: the queue kernel; FP32 with dominant walkers: the mixed kernel).
After one uncaptured call of the batch (which registers its walker table and queue), the call is
captured once with torch.cuda.graph and replayed k times.  The replays must advance the chains
exactly as k uncaptured calls do -- positions, ln psi, sweep counters and accumulators bit for
bit -- so the cached walker table and the queue stay valid across replays."""
import numpy as np
import pytest
import torch

import paper_1312_1282_gb300 as q
from tests._gpu import lattice_batch, zeros

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,mixed", [(q.QMC_FP64, False), (q.QMC_FP32, True)])
def test_graph_replays_equal_uncaptured_calls(prec, mixed):
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    if mixed:  # two dominant walkers: the mixed kernel (whole CTAs for them, the queue for the rest)
        ns = [600, 600] + [64, 130] * ((nsm + 30) // 2)
        opt = q.options(precision=prec, recompute_every=3, threads_per_walker=128)
    else:
        ns = ([64, 130, 600] * (nsm // 3 + 14))[:nsm + 40]
        opt = q.options(precision=prec, recompute_every=3)
    W = len(ns)
    A = lattice_batch(ns, prec, seed=95)
    B = lattice_batch(ns, prec, seed=95)
    la, sa, aa = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    lb, sb, ab = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(A.d, opt, A.pos, la)
    q.qmc_log_psi(B.d, opt, B.pos, lb)
    seed, nsw, every, k = 0x6A7, 2, 1, 3
    # A and B have the same descriptors, so they share the library's walker table and queue:
    # their calls must not overlap on the GPU
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # the uncaptured first call of the batch, on the capture stream
        q.qmc_sweep(A.d, opt, A.pos, la, sa, seed, nsw, every, aa)
    torch.cuda.synchronize()
    q.qmc_sweep(B.d, opt, B.pos, lb, sb, seed, nsw, every, ab)
    torch.cuda.synchronize()
    launches = q.qmc_launch_count()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        q.qmc_sweep(A.d, opt, A.pos, la, sa, seed, nsw, every, aa)
    captured = q.qmc_launch_count() - launches
    assert captured == 2  # queue initialisation and the persistent (or mixed) sweep
    for _ in range(k):
        g.replay()
    torch.cuda.synchronize()
    for _ in range(k):
        q.qmc_sweep(B.d, opt, B.pos, lb, sb, seed, nsw, every, ab)
    torch.cuda.synchronize()
    assert q.qmc_status(timeout_ms=120000) == 0
    assert torch.all(sa == nsw * (k + 1))
    assert torch.equal(A.pos, B.pos) and torch.equal(sa, sb)
    assert torch.equal(la, lb) and torch.equal(aa, ab)
    assert np.all(aa[:, 6].cpu().numpy() == nsw * (k + 1))
