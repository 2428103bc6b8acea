"""The tiled local-energy pass with its drift arrays in global scratch instead of shared memory
(chosen when the arrays in shared memory would leave fewer walkers resident per SM).

Checked two ways: the fixed-configuration and chain parity suites are rerun in a child process
with QMC_TILE_GLOBAL=1 (every tiled sweep then uses the scratch), and walkers of 3000 atoms at
128 threads per walker -- which select the scratch on their own -- sample the energy inside the
sweep, compared with the stand-alone local-energy pass on the final configurations."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import paper_1312_1282_gb300 as q
import qmc_inputs as qi
from tests._gpu import energy_scale, zeros

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suites_pass_with_drift_scratch():
    env = dict(os.environ, QMC_TILE_GLOBAL="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        "tests/test_gpu_fixed.py", "tests/test_gpu_chain.py"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


def test_sweep_energy_with_drift_scratch_matches_the_pass():
    n = 3000
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    W = nsm + 8  # persistent mode
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)
    d = q.descs([(n, pad, w * 3 * pad, w, L, 0.0, qi.B_HE, 5.0, 0.8) for w in range(W)])
    opt = q.options(precision=q.QMC_FP32, recompute_every=1, threads_per_walker=128)
    pos = torch.empty(W * 3 * pad, dtype=torch.float32, device="cuda")
    q.qmc_init_walkers(d, 12, 0.1, opt, pos)
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(d, opt, pos, lp)
    q.qmc_sweep(d, opt, pos, lp, sw, 12, 2, 2, acc)
    e = zeros((W, 5))
    q.qmc_local_energy(d, q.options(precision=q.QMC_FP32), pos, e)
    assert q.qmc_status(timeout_ms=300000) == 0
    a = acc.cpu().numpy()
    assert np.all(a[:, 6] == 1)
    # the sample of the sweep and the separate pass see the same final configuration (their
    # FP32 sums run in different orders: compared on the scale of the sums T_L and E_L cancel)
    en = e.cpu().numpy()
    for w in range(W):
        assert np.all(np.abs(a[w, [2, 3, 4, 5, 0]] - en[w]) <= 1e-5 * energy_scale(en[w])), w


def test_batches_on_two_streams_keep_their_own_drift_scratch():
    """Sweeps of two different batches may run at the same time on two streams.  Each batch's
    energy samples use that batch's own drift scratch, so overlapping calls give bit for bit
    the chains and sums of calls made one after the other."""
    n, W = 3000, 8  # 3000 atoms at 128 threads per walker select the scratch; 16 CTAs run together
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)
    opt = q.options(precision=q.QMC_FP32, recompute_every=0, threads_per_walker=128)
    batches = [q.descs([(n, pad, w * 3 * pad, first + w, L, 0.0, qi.B_HE, 5.0, 0.8) for w in range(W)])
               for first in (0, W)]
    starts = []
    for d in batches:
        p = torch.empty(W * 3 * pad, dtype=torch.float32, device="cuda")
        q.qmc_init_walkers(d, 21, 0.1, opt, p)
        starts.append(p)

    def state():
        return [(p.clone(), zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))) for p in starts]

    one_after_other = state()
    for d, (p, lp, sw, acc) in zip(batches, one_after_other):
        q.qmc_sweep(d, opt, p, lp, sw, 21, 2, 1, acc)
    assert q.qmc_status(timeout_ms=300000) == 0

    together = state()
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for d, (p, lp, sw, acc), st in zip(batches, together, streams):
        q.qmc_sweep(d, opt, p, lp, sw, 21, 2, 1, acc, st)
    torch.cuda.synchronize()
    assert q.qmc_status(timeout_ms=300000) == 0
    for a, b in zip(one_after_other, together):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    assert np.all(one_after_other[0][3].cpu().numpy()[:, 6] == 2)  # two energy samples per walker
