"""Walkers larger than one CTA's shared memory run in place from HBM.

The HBM path is the same kernels with the coordinates read and written in global memory.  It
is checked two ways: the whole fixed-configuration and chain parity suites are rerun in a child
process with QMC_GLOBAL_WALKERS=1 (which forces the HBM path for every batch), and a walker of
20 000 atoms -- beyond the FP32 shared-memory capacity -- is swept and sampled, its energy
checked against the oracle's."""
import math
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import paper_1312_1282_gb300 as q
import qmc_inputs as qi
import oracle
from tests._gpu import H2M, energy_scale, zeros

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suites_pass_on_the_hbm_path():
    env = dict(os.environ, QMC_GLOBAL_WALKERS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        "tests/test_gpu_fixed.py", "tests/test_gpu_chain.py"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


def test_walker_beyond_shared_memory():
    n = 20000
    assert n > q.qmc_capacity(q.QMC_FP32)
    W = 2
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)
    d = q.descs([(n, pad, w * 3 * pad, w, L, 0.0, qi.B_HE, 5.0, 0.8) for w in range(W)])
    opt = q.options(precision=q.QMC_FP32, recompute_every=1)
    pos = torch.empty(W * 3 * pad, dtype=torch.float32, device="cuda")
    q.qmc_init_walkers(d, 11, 0.1, opt, pos)
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(d, opt, pos, lp)
    lp0 = lp.clone()
    q.qmc_sweep(d, opt, pos, lp, sw, 11, 1, 1, acc)
    e = zeros((W, 5))
    q.qmc_local_energy(d, opt, pos, e)
    lpe = zeros(W)
    q.qmc_log_psi(d, opt, pos, lpe)
    assert q.qmc_status(timeout_ms=600000) == 0
    a = acc.cpu().numpy()
    rate = a[:, 7] / n
    assert np.all((rate > 0.2) & (rate < 0.9)), rate
    assert torch.all(sw == 1)
    # the energy sample of the sweep and a separate pass see the same final configuration
    np.testing.assert_allclose(a[:, [2, 3, 4, 5, 0]], e.cpu().numpy(), rtol=1e-6)
    # ln psi was recomputed after the sweep (recompute_every = 1): equal to a fresh pass
    np.testing.assert_allclose(lp.cpu().numpy(), lpe.cpu().numpy(), rtol=1e-6)
    assert not torch.equal(lp, lp0)
    # parity: the oracle's local energy of walker 0's final configuration (2 x 10^8 pairs)
    host = pos.cpu().numpy()
    blk = host[:3 * pad].reshape(3, pad)[:, :n].astype(np.float64)
    want = oracle.local_energy(blk, L, qi.B_HE, 5.0, 1, H2M)
    assert np.all(np.abs(e.cpu().numpy()[0] - want) <= 1e-5 * energy_scale(want)), (e[0], want)
