"""Few walkers of large N run each walker on a thread-block cluster (slices of the walker in the
shared memory of C CTAs, partial sums exchanged through distributed shared memory).  Chains as
the oracle's decision by decision except at near ties, checked sweep by sweep (one sweep per
call; the oracle reruns each sweep from the GPU's state, and a sweep that differs must contain
a near tie); ln psi carried through the moves as a fresh recompute; ragged slices (N not a
multiple of 4 C) and both proposals."""
import numpy as np
import pytest
import torch

import paper_1312_1282_gb300 as q
import qmc_inputs as qi
from tests._gpu import fp32_sweeps_vs_oracle, zeros

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,W,proposal", [(4096, 3, q.QMC_CUBE), (4099, 2, q.QMC_GAUSS), (6001, 5, q.QMC_CUBE)])
def test_cluster_sweep_matches_oracle(n, W, proposal):
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)
    step = 0.8 if proposal == q.QMC_CUBE else 0.6
    d = q.descs([(n, pad, w * 3 * pad, w, L, 0.0, qi.B_HE, 5.0, step) for w in range(W)])
    opt = q.options(precision=q.QMC_FP32, proposal=proposal, recompute_every=0)
    pos = torch.empty(W * 3 * pad, dtype=torch.float32, device="cuda")
    q.qmc_init_walkers(d, 0xC1, 0.1, opt, pos)
    start = pos.cpu().numpy()
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(d, opt, pos, lp)
    states, accepted, prev = [start], [], np.zeros(W)
    for _ in range(2):  # one sweep per call
        launches = q.qmc_launch_count()
        q.qmc_sweep(d, opt, pos, lp, sw, 0xC1, 1, 0, acc)
        assert q.qmc_launch_count() - launches == 1  # one cluster launch, no queue
        states.append(pos.cpu().numpy())
        a = acc[:, 7].cpu().numpy()
        accepted.append(a - prev)
        prev = a
    fresh = zeros(W)
    q.qmc_log_psi(d, opt, pos, fresh)
    assert q.qmc_status(timeout_ms=120000) == 0
    assert torch.all(sw == 2)
    host, a = pos.cpu().numpy(), acc.cpu().numpy()
    # ln psi carried through the moves equals a recompute of the final configuration (FP32 sums
    # of ~N^2/2 terms: relative 1e-5 of the sum of |u|, bounded here by |ln psi|)
    np.testing.assert_allclose(lp.cpu().numpy(), fresh.cpu().numpy(), rtol=2e-5)
    agree = 0
    for w in range(W):
        blk = [st[w * 3 * pad:(w + 1) * 3 * pad].reshape(3, pad)[:, :n].astype(np.float64) for st in states]
        assert np.all(np.isfinite(blk[-1])) and np.all((blk[-1] >= 0) & (blk[-1] <= L))
        agree += fp32_sweeps_vs_oracle(blk, [acc_k[w] for acc_k in accepted], n, L, qi.B_HE, 5.0, step, 0xC1, w,
                                       proposal=proposal)[0]
    assert agree >= 2 * W - 1
