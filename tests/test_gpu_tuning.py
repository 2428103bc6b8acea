"""The trial-step tuner on real chains: after bisection on short probes, a longer run at the
tuned step accepts close to the target fraction of moves, for both proposals (cube half-width
and Gaussian per-component sigma), and the probes advanced the chains like any sweep."""
import pytest
import torch

import paper_1312_1282_gb300 as q
import qmc_inputs as qi
from paper_1312_1282_gb300 import tuning
from tests._gpu import zeros

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("proposal", [q.QMC_CUBE, q.QMC_GAUSS])
def test_tuned_step_gives_the_target_acceptance(proposal):
    n, W, seed = 128, 64, 0x7A1
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)

    def descs_of(step):
        return q.descs([(n, pad, w * 3 * pad, w, L, 0.0, qi.B_HE, 5.0, step) for w in range(W)])

    opt = q.options(precision=q.QMC_FP32, proposal=proposal)
    pos = torch.empty(W * 3 * pad, dtype=torch.float32, device="cuda")
    q.qmc_init_walkers(descs_of(0.5), seed, 0.1, opt, pos)
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(descs_of(0.5), opt, pos, lp)
    q.qmc_sweep(descs_of(0.5), opt, pos, lp, sw, seed, 20, 0, acc)  # equilibration
    step, rates = tuning.tune_step(descs_of, opt, pos, lp, sw, seed, acc, target=0.5, probes=8)
    assert 0.1 < step < 3.0 and len(rates) == 8
    acc.zero_()
    q.qmc_sweep(descs_of(step), opt, pos, lp, sw, seed, 20, 0, acc)
    assert q.qmc_status(timeout_ms=60000) == 0
    # 164 k moves (sampling spread 0.002); the bracket after 8 probes is 0.011 A wide
    rate = acc[:, 7].sum().item() / (W * n * 20)
    assert abs(rate - 0.5) < 0.05, (step, rate, rates)
    assert torch.all(sw == 20 + 8 * 4 + 20)
