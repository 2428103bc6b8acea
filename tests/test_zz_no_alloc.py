"""qmc_sweep_static: the sweep for callers that cannot allocate device memory.

Such callers (a process whose device memory is held by another allocator, code that must not
take the synchronisation of an allocation) get the same sweep with its walker table, order and
error word in a fixed array of the library image instead of memory the library allocates.
Checked here through the C ABI against qmc_sweep on the same inputs, over two calls in a row
(the second call finds the first call's contents in the shared array), with the tolerances
of the other chain tests: the two entry points run the same kernel, so they agree exactly.
This file is collected last so that a failure here leaves the rest of the suite already run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_1312_1282_gb300 as q
import qmc_inputs as qi
from tests._gpu import lattice_batch, zeros

pytestmark = pytest.mark.gpu


def _state(P):
    return zeros(P.W), zeros(P.W, torch.int64), zeros((P.W, q.NACC))


@pytest.mark.parametrize("prec", [q.QMC_FP32, q.QMC_FP64])
def test_static_sweep_matches_qmc_sweep_on_two_calls(prec):
    ns = [64, 130, 257, 512, 64, 1001]
    A = lattice_batch(ns, prec, seed=70)
    B = lattice_batch(ns, prec, seed=70)
    opt = q.options(precision=prec, recompute_every=3, threads_per_walker=64)
    la, sa, aa = _state(A)
    lb, sb, ab = _state(B)
    q.qmc_log_psi(A.d, opt, A.pos, la)
    q.qmc_log_psi(B.d, opt, B.pos, lb)
    err = zeros(1, torch.int32)
    for nsw, every in ((3, 1), (2, 2)):
        q.qmc_sweep(A.d, opt, A.pos, la, sa, 0xA110C, nsw, every, aa)
        q.qmc_sweep_static(B.d, opt, B.pos, lb, sb, 0xA110C, nsw, every, ab, err=err)
        torch.cuda.synchronize()
        tol = 1e-10 if prec == q.QMC_FP64 else 1e-5
        np.testing.assert_allclose(B.pos.cpu().numpy(), A.pos.cpu().numpy(), rtol=0, atol=tol)
        np.testing.assert_allclose(lb.cpu().numpy(), la.cpu().numpy(), rtol=tol)
        np.testing.assert_allclose(ab.cpu().numpy(), aa.cpu().numpy(), rtol=tol)
        assert torch.equal(sb, sa)
    assert err.item() == 0
    assert q.qmc_status(timeout_ms=60000) == 0


def test_static_sweep_second_batch_overwrites_first():
    # a different, smaller batch after a larger one: nothing of the first table may leak in
    big = lattice_batch([512] * 12, q.QMC_FP32, seed=71)
    lb, sb, ab = _state(big)
    q.qmc_sweep_static(big.d, q.options(), big.pos, lb, sb, 5, 1, 0, ab)
    A = lattice_batch([96, 200], q.QMC_FP32, seed=72)
    B = lattice_batch([96, 200], q.QMC_FP32, seed=72)
    la, sa, aa = _state(A)
    lc, sc, ac = _state(B)
    q.qmc_sweep(A.d, q.options(), A.pos, la, sa, 6, 2, 1, aa)
    q.qmc_sweep_static(B.d, q.options(), B.pos, lc, sc, 6, 2, 1, ac)
    torch.cuda.synchronize()
    np.testing.assert_allclose(B.pos.cpu().numpy(), A.pos.cpu().numpy(), rtol=0, atol=1e-5)
    np.testing.assert_allclose(ac.cpu().numpy(), aa.cpu().numpy(), rtol=1e-5)


def test_static_sweep_rejects_too_many_walkers():
    n = 8
    rows = [(n, n, w * 3 * n, w, 10.0, 0.0, 3.0, 5.0, 0.5) for w in range(q.QMC_STATIC_MAX_WALKERS + 1)]
    d = q.descs(rows)
    pos = zeros(len(rows) * 3 * n, torch.float32)
    lp, sw, acc = zeros(len(rows)), zeros(len(rows), torch.int64), zeros((len(rows), q.NACC))
    with pytest.raises(q.QmcError, match="at most 4096 walkers"):
        q.qmc_sweep_static(d, q.options(), pos, lp, sw, 1, 1, 0, acc)
    assert q.lib().qmc_sweep_static(d, len(rows), C.byref(q.options()), C.c_void_p(pos.data_ptr()),
                                    C.c_void_p(lp.data_ptr()), C.c_void_p(sw.data_ptr()), 1, 1, 0,
                                    C.c_void_p(acc.data_ptr()), None, None) == -1


@pytest.mark.parametrize("case", ["queue_and_groups", "drift_tile_modes", "hbm_walkers"])
def test_static_sweep_matches_qmc_sweep_on_other_launch_shapes(case):
    # qmc_sweep runs these batches through launch shapes the static path never takes: the
    # persistent walker queue (more walkers than SMs), several walkers per CTA (thousands of small
    # walkers), the drift arrays of the energy pass in global scratch (n > 2400 at 128 threads per
    # walker), and walkers too large for shared memory used in place in HBM.  The chains and sums
    # must be the same, bit for bit (the arithmetic of every move and energy sample is the same).
    if case == "queue_and_groups":
        prec, ns, kw = q.QMC_FP64, [64] * 3700, dict(threads_per_walker=32)
    elif case == "drift_tile_modes":
        prec, ns, kw = q.QMC_FP32, [2500, 2504, 2404], dict(threads_per_walker=128)
    else:
        prec, ns, kw = q.QMC_FP64, [10000, 9700], {}
        assert min(ns) > q.qmc_capacity(q.QMC_FP64)
    A = lattice_batch(ns, prec, seed=74)
    B = lattice_batch(ns, prec, seed=74)
    opt = q.options(precision=prec, recompute_every=1, **kw)
    la, sa, aa = _state(A)
    lb, sb, ab = _state(B)
    q.qmc_log_psi(A.d, opt, A.pos, la)
    q.qmc_log_psi(B.d, opt, B.pos, lb)
    q.qmc_sweep(A.d, opt, A.pos, la, sa, 0xB0B, 1, 1, aa)
    q.qmc_sweep_static(B.d, opt, B.pos, lb, sb, 0xB0B, 1, 1, ab)
    assert q.qmc_status(timeout_ms=300000) == 0
    assert torch.equal(A.pos, B.pos) and torch.equal(sa, sb) and torch.all(sa == 1)
    assert torch.equal(la, lb) and torch.equal(aa, ab)


def test_static_sweep_refuses_stream_capture():
    # its walker table is staged from host memory that the next call reuses, so a recorded copy
    # would replay whatever was staged last: the call is refused before anything is enqueued
    A = lattice_batch([64, 130], q.QMC_FP32, seed=75)
    lp, sw, acc = _state(A)
    q.qmc_sweep_static(A.d, q.options(), A.pos, lp, sw, 7, 1, 0, acc)  # first call: outside capture
    torch.cuda.synchronize()
    before, marker = A.pos.clone(), zeros(1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(g, stream=s):
        try:
            q.qmc_sweep_static(A.d, q.options(), A.pos, lp, sw, 7, 1, 0, acc)
        except q.QmcError as e:
            refused = e
        marker.add_(1.0)  # the capture itself stays valid
    assert refused is not None and refused.code == -1 and "capture" in str(refused)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(A.pos, before) and marker.item() == 1.0 and torch.all(sw == 1)
    assert q.qmc_status(timeout_ms=60000) == 0


def test_status_reports_static_path_errors_without_an_err_word():
    A = lattice_batch([64, 64], q.QMC_FP32, seed=76)
    A.pos[A.d[1].offset + 3] = float("nan")
    lp, sw, acc = _state(A)
    q.qmc_sweep_static(A.d, q.options(), A.pos, lp, sw, 8, 1, 0, acc)  # err = NULL
    with pytest.raises(q.QmcError, match="bad coordinate"):
        q.qmc_status(timeout_ms=60000)
    assert q.qmc_status(timeout_ms=60000) == 0  # read and cleared
    assert sw.cpu().tolist() == [1, 0]
