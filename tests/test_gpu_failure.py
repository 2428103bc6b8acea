"""Failure detection on the GPU without a fault: a bounded device wait that runs out.

Every wait in the sweep kernels is bounded (the walker queue of the persistent sweep, the
partial-sum exchange of the cluster sweep); when the limit passes, the kernel sets
QMC_DEVERR_TIMEOUT in the device error word, stops waiting and returns, so the context stays
usable.  Each test runs in a child process with the limit shortened to 20 ms (QMC_WAIT_LIMIT_MS)
and one producer silenced for the first call of the process (QMC_TEST_DROP): in the queue case
one walker is never pushed back, so the pop that waits for it runs out; in the cluster case one
CTA of a walker's cluster never stores its partial sums nor arrives on its peers' barriers, so
every CTA of that cluster runs out at its first exchange.  The child checks that qmc_status
reports the timeout, that the call ended promptly, that the walker whose producer was silenced
was not written back where the path guarantees it, and that the next, normal call in the same
context runs to the oracle's chains."""
import ctypes as C
import json
import os
import subprocess
import sys
import time

import numpy as np
import pytest
import torch

import paper_1312_1282_gb300 as q
import qmc_inputs as qi
from tests._gpu import H2M, fp32_sweeps_vs_oracle, lattice_batch, zeros

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _status():
    bits = C.c_uint32(0)
    rc = q.lib().qmc_status(q._stream(None), 60000, C.byref(bits))
    return rc, bits.value


def _child_queue():
    import oracle
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    W = nsm + 5  # more walkers than SMs, not a multiple: the persistent sweep with its queue
    opt = q.options(precision=q.QMC_FP64, recompute_every=0)
    P = lattice_batch([64] * W, q.QMC_FP64, seed=91)
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(P.d, opt, P.pos, lp)
    torch.cuda.synchronize()
    t0 = time.time()
    q.qmc_sweep(P.d, opt, P.pos, lp, sw, 5, 4, 0, acc)  # one push withheld: a pop runs out
    rc, bits = _status()
    seconds = time.time() - t0
    # the next call in the same context runs normally
    Q = lattice_batch([64] * W, q.QMC_FP64, seed=92)
    lq, sq, aq = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(Q.d, opt, Q.pos, lq)
    q.qmc_sweep(Q.d, opt, Q.pos, lq, sq, 5, 4, 0, aq)
    rc2, bits2 = _status()
    same = []
    for w in (0, W - 1):
        Wk = oracle.make_walker(64, Q.Ls[w], Q.bs[w], 5.0, 0.8, seed=5, wid=Q.ids[w], hbar2_over_m=H2M)
        opos, _, _, oacc, _ = oracle.run_walker(Wk, Q.confs[w], 0.0, 0, 4, 0)
        same.append(bool(np.array_equal(Q.positions(w), opos) and aq[w, 7].item() == oacc[7]))
    print(json.dumps({"rc": rc, "bits": bits, "seconds": seconds, "sweeps_done": int((sw == 4).sum().item()),
                      "W": W, "rc2": rc2, "bits2": bits2, "all_advanced": bool(torch.all(sq == 4).item()),
                      "oracle_same": same}))


def _child_cluster():
    n, W = 4096, 2
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)
    d = q.descs([(n, pad, w * 3 * pad, w, L, 0.0, qi.B_HE, 5.0, 0.8) for w in range(W)])
    opt = q.options(precision=q.QMC_FP32, recompute_every=0)
    pos = torch.empty(W * 3 * pad, dtype=torch.float32, device="cuda")
    q.qmc_init_walkers(d, 0xC1, 0.1, opt, pos)
    start = pos.clone()
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(d, opt, pos, lp)
    torch.cuda.synchronize()
    t0 = time.time()
    launches = q.qmc_launch_count()
    q.qmc_sweep(d, opt, pos, lp, sw, 0xC1, 1, 0, acc)  # CTA 1 of walker 0's cluster stays silent
    one_launch = q.qmc_launch_count() - launches == 1
    rc, bits = _status()
    seconds = time.time() - t0
    untouched = bool(torch.equal(pos[:3 * pad], start[:3 * pad]) and sw[0].item() == 0)
    # the next call in the same context, from the same start, runs normally
    pos2 = start.clone()
    lp2, sw2, acc2 = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(d, opt, pos2, lp2)
    q.qmc_sweep(d, opt, pos2, lp2, sw2, 0xC1, 1, 0, acc2)
    rc2, bits2 = _status()
    h0, h1, a = start.cpu().numpy(), pos2.cpu().numpy(), acc2.cpu().numpy()
    agree = 0
    for w in range(W):
        blk = [h[w * 3 * pad:(w + 1) * 3 * pad].reshape(3, pad)[:, :n].astype(np.float64) for h in (h0, h1)]
        agree += fp32_sweeps_vs_oracle(blk, [a[w, 7]], n, L, qi.B_HE, 5.0, 0.8, 0xC1, w)[0]
    print(json.dumps({"rc": rc, "bits": bits, "seconds": seconds, "one_launch": one_launch, "untouched": untouched,
                      "rc2": rc2, "bits2": bits2, "all_advanced": bool(torch.all(sw2 == 1).item()),
                      "agree": agree, "W": W}))


def _run_child(fn, **env):
    e = dict(os.environ, QMC_WAIT_LIMIT_MS="20", **env)
    r = subprocess.run([sys.executable, "-c", f"import tests.test_gpu_failure as t; t.{fn}()"], cwd=ROOT, env=e,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_queue_wait_runs_out_and_the_context_stays_usable():
    out = _run_child("_child_queue", QMC_TEST_DROP="queue")
    assert out["rc"] == -4 and out["bits"] & 8, out  # QMC_ERR_DEVICE with QMC_DEVERR_TIMEOUT
    assert out["seconds"] < 30, out
    assert out["sweeps_done"] == out["W"] - 1, out  # every walker but the one never pushed back
    assert out["rc2"] == 0 and out["bits2"] == 0 and out["all_advanced"], out
    assert all(out["oracle_same"]), out


def test_cluster_exchange_wait_runs_out_and_the_context_stays_usable():
    out = _run_child("_child_cluster", QMC_TEST_DROP="cluster", QMC_CLUSTER="1")
    assert out["one_launch"], out
    assert out["rc"] == -4 and out["bits"] & 8, out
    assert out["seconds"] < 30, out
    assert out["untouched"], out  # no CTA of the failed cluster wrote the walker back
    assert out["rc2"] == 0 and out["bits2"] == 0 and out["all_advanced"], out
    assert out["agree"] >= out["W"] - 1, out
