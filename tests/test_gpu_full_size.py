"""Parity at the full sizes of the benchmark workloads, in the launch configurations bench.py
times, on sampled walkers the oracle reruns move by move:

- the uneven batch (3968 walkers of N = 128 ... 4000, densities and b drawn per walker; the
  autotuned shape, i.e. the mixed kernel with the dominant N = 4000 walkers on whole CTAs),
- N = 10 000, one walker per SM (autotuned shape, energy pass with the drift scratch),
  including the (b, m) adjoint of one walker,
- N = 512, 1024 walkers in FP64 (bit for bit).

FP32 chains agree with the FP64 oracle decision by decision except at near ties; energies of the
final configurations agree within 1e-5 of the sums they are made of."""
import numpy as np
import pytest
import torch

import oracle
import paper_1312_1282_gb300 as q
import qmc_inputs as qi
from tests._gpu import H2M, energy_scale, fp32_sweeps_vs_oracle, grad_scales, report, zeros

pytestmark = pytest.mark.gpu


def _sampled(d, pos, start, acc, w, seed, nsweeps, energy_every, opt, tol_pos=1e-3):
    """Rerun walker w in the oracle; returns True if the chains agree, else asserts a near tie."""
    r = d[w]
    blk0 = start[r.offset:r.offset + 3 * r.pad_n].reshape(3, r.pad_n)[:, :r.n].astype(np.float64)
    blk1 = pos[r.offset:r.offset + 3 * r.pad_n].reshape(3, r.pad_n)[:, :r.n].astype(np.float64)
    P = oracle.make_walker(r.n, r.L, r.b, r.m_exp, r.step, sym=opt.sym, proposal=opt.proposal, seed=seed, wid=r.id,
                           hbar2_over_m=H2M, recompute_every=opt.recompute_every)
    opos, _, _, oacc, mg = oracle.run_walker(P, blk0, oracle.log_psi(blk0, r.L, r.b, r.m_exp, opt.sym), 0, nsweeps,
                                             energy_every, margins=True)
    e = oracle.local_energy(blk1, r.L, r.b, r.m_exp, opt.sym, H2M)
    assert np.all(np.abs(acc[w, [2, 3, 4, 5, 0]] - e) <= 1e-5 * energy_scale(e)), (w, acc[w], e)
    if acc[w, 7] == oacc[7] and np.abs(blk1 - opos).max() < tol_pos:
        return True
    assert np.abs(mg).min() < 1e-3, (w, np.abs(mg).min())
    return False


def test_uneven_batch_sampled_walkers():
    params = qi.uneven_params(qi.uneven_groups(), seed=0x5EED0004)
    rows, off = [], 0
    for w, (n, rho, b) in enumerate(params):
        pad = qi.pad4(n)
        rows.append((n, pad, off, w, qi.box_side(n, rho), 0.0, b, 5.0, 0.3 * rho ** (-1.0 / 3.0)))
        off += 3 * pad
    d = q.descs(rows)
    W = len(rows)
    opt = q.options(precision=q.QMC_FP32, recompute_every=50)
    pos = torch.empty(off, dtype=torch.float32, device="cuda")
    q.qmc_init_walkers(d, 0x5EED0004, 0.1, opt, pos)
    q.qmc_autotune(d, opt, pos)
    start = pos.cpu().numpy()
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(d, opt, pos, lp)
    q.qmc_sweep(d, opt, pos, lp, sw, 0x5EED0004, 1, 1, acc)
    assert q.qmc_status(timeout_ms=300000) == 0
    assert torch.all(sw == 1)
    host, a = pos.cpu().numpy(), acc.cpu().numpy()
    # the first N = 4000 walker (dominant), and one walker of every other size
    firsts = {}
    for w, r in enumerate(rows):
        firsts.setdefault(r[0], w)
    picks = [firsts[n] for n in (4000, 1952, 1000, 500, 128)] + [W - 1]
    agree = sum(_sampled(d, host, start, a, w, 0x5EED0004, 1, 1, opt) for w in picks)
    assert agree >= len(picks) - 1


def test_large_walkers_sampled_with_adjoint():
    n = 10000
    W = torch.cuda.get_device_properties(0).multi_processor_count
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)
    d = q.descs([(n, pad, w * 3 * pad, w, L, 0.0, qi.B_HE, 5.0, 0.8) for w in range(W)])
    opt = q.options(precision=q.QMC_FP32, recompute_every=50)
    pos = torch.empty(W * 3 * pad, dtype=torch.float32, device="cuda")
    q.qmc_init_walkers(d, 0x5EED0005, 0.1, opt, pos)
    q.qmc_autotune(d, opt, pos)
    start = pos.cpu().numpy()
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(d, opt, pos, lp)
    q.qmc_sweep(d, opt, pos, lp, sw, 0x5EED0005, 1, 1, acc)
    grad = zeros((W, 6))
    q.qmc_energy_grad(d, opt, pos, grad)
    assert q.qmc_status(timeout_ms=300000) == 0
    host, a, g = pos.cpu().numpy(), acc.cpu().numpy(), grad.cpu().numpy()
    _sampled(d, host, start, a, W - 1, 0x5EED0005, 1, 1, opt)
    blk = host[:3 * pad].reshape(3, pad)[:, :n].astype(np.float64)
    want = oracle.energy_grad(blk, L, qi.B_HE, 5.0, 1, H2M)
    # as in the fixed-configuration test: each output on the summed magnitudes of its pair terms
    # (row sums from 200 evenly spaced atoms), at the FP32 tolerance 1e-5
    scale = grad_scales(blk, L, qi.B_HE, 5.0, 1, H2M, rows=200)
    err = np.abs(g[0] - want) / scale
    report("energy_grad_N10000", err_on_term_scale=err, err_on_own_magnitude=np.abs(g[0] - want) / np.abs(want))
    assert np.all(err <= 1e-5), (g[0], want, err)


def test_fp64_batch_sampled_walkers_bit_for_bit():
    n, W = 512, 1024
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)
    d = q.descs([(n, pad, w * 3 * pad, w, L, 0.0, qi.B_HE, 5.0, 0.8) for w in range(W)])
    opt = q.options(precision=q.QMC_FP64, recompute_every=50)
    pos = torch.empty(W * 3 * pad, dtype=torch.float64, device="cuda")
    q.qmc_init_walkers(d, 0x5EED0002, 0.1, opt, pos)
    start = pos.cpu().numpy()
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(d, opt, pos, lp)
    q.qmc_sweep(d, opt, pos, lp, sw, 0x5EED0002, 3, 3, acc)
    assert q.qmc_status(timeout_ms=300000) == 0
    host, a = pos.cpu().numpy(), acc.cpu().numpy()
    for w in (0, 511, W - 1):
        r = d[w]
        blk0 = start[r.offset:r.offset + 3 * pad].reshape(3, pad)[:, :n]
        blk1 = host[r.offset:r.offset + 3 * pad].reshape(3, pad)[:, :n]
        P = oracle.make_walker(n, L, qi.B_HE, 5.0, 0.8, seed=0x5EED0002, wid=w, hbar2_over_m=H2M, recompute_every=50)
        opos, _, _, oacc, _ = oracle.run_walker(P, blk0, oracle.log_psi(blk0, L, qi.B_HE), 0, 3, 3)
        assert np.array_equal(blk1, opos)
        assert a[w, 7] == oacc[7] and a[w, 6] == oacc[6]
        np.testing.assert_allclose(a[w, :6], oacc[:6], rtol=1e-10, atol=1e-9)
