"""Few walkers of large N run each walker on a thread-block cluster (slices of the walker in the
shared memory of C CTAs, partial sums exchanged through distributed shared memory).  Chains as
the oracle's decision by decision except at near ties; ln psi carried through the moves as a
fresh recompute; ragged slices (N not a multiple of 4 C) and both proposals."""
import numpy as np
import pytest
import torch

import oracle
import paper_1312_1282_gb300 as q
import qmc_inputs as qi
from tests._gpu import H2M, zeros

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
    launches = q.qmc_launch_count()
    q.qmc_sweep(d, opt, pos, lp, sw, 0xC1, 2, 0, acc)
    assert q.qmc_launch_count() - launches == 1  # one cluster launch, no queue
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
        blk0 = start[w * 3 * pad:(w + 1) * 3 * pad].reshape(3, pad)[:, :n].astype(np.float64)
        blk1 = host[w * 3 * pad:(w + 1) * 3 * pad].reshape(3, pad)[:, :n].astype(np.float64)
        assert np.all(np.isfinite(blk1)) and np.all((blk1 >= 0) & (blk1 <= L))
        P = oracle.make_walker(n, L, qi.B_HE, 5.0, step, proposal=proposal, seed=0xC1, wid=w, hbar2_over_m=H2M)
        opos, _, _, oacc, mg = oracle.run_walker(P, blk0, oracle.log_psi(blk0, L, qi.B_HE), 0, 2, 0, margins=True)
        if a[w, 7] == oacc[7] and np.abs(blk1 - opos).max() < 1e-3:
            agree += 1
        else:
            assert np.abs(mg).min() < 1e-3, (w, np.abs(mg).min())
    assert agree >= W - 1
