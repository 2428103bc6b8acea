"""Load masking (the paper's Sec. 4.2, Eq. maskedtime): analyses on a second stream, overlapped with
the generation of the next macroupdates, give the results of the sequential schedule.

Thirteen walkers of N = 4096 (the few-walker shape of the paper's largest run, scaled down: each
walker's sweep runs on a thread-block cluster, leaving SMs idle for the analysis), an analysis
(local energy and pair histogram) every m = 2 macroupdates, three analyses.  The masked and the
sequential schedule start from the same state: chains, ln psi, sweep counters, accumulators,
every analysed energy and the summed histograms agree bit for bit, and the energies of the last
analysed configuration agree with the oracle's."""
import numpy as np
import pytest
import torch

import oracle
import paper_1312_1282_gb300 as q
import qmc_inputs as qi
from paper_1312_1282_gb300 import masking
from tests._gpu import H2M, energy_scale, zeros

pytestmark = pytest.mark.gpu


def test_masked_schedule_equals_sequential_and_oracle():
    n, W, m, count, nbins = 4096, 13, 2, 3, 64
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)
    d = q.descs([(n, pad, w * 3 * pad, w, L, 0.0, qi.B_HE, 5.0, 0.8) for w in range(W)])
    opt = q.options(precision=q.QMC_FP32, recompute_every=0)
    start = torch.empty(W * 3 * pad, dtype=torch.float32, device="cuda")
    q.qmc_init_walkers(d, 0x3A5C, 0.1, opt, start)
    runs = {}
    for masked in (False, True):
        pos = start.clone()
        lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
        q.qmc_log_psi(d, opt, pos, lp)
        en, hist = zeros((count, W, 5)), zeros((W, nbins), torch.int64)
        masking.run_schedule(d, opt, pos, lp, sw, acc, 0x3A5C, m, count, energies=en, hist=hist, nbins=nbins,
                             rmax=L / 2, masked=masked)
        torch.cuda.synchronize()
        assert q.qmc_status(timeout_ms=300000) == 0
        runs[masked] = (pos, lp, sw, acc, en, hist)
    for a, b in zip(runs[False], runs[True]):
        assert torch.equal(a, b)
    pos, _, sw, _, en, hist = runs[True]
    assert torch.all(sw == m * count)
    assert torch.all(hist.sum(dim=1) > 0)
    blk = pos.cpu().numpy()[:3 * pad].reshape(3, pad)[:, :n].astype(np.float64)
    want = oracle.local_energy(blk, L, qi.B_HE, 5.0, 1, H2M)
    assert np.all(np.abs(en[count - 1, 0].cpu().numpy() - want) <= 1e-5 * energy_scale(want))
