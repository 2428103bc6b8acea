"""GPU Markov chains vs the oracle's, on the same Philox streams.

FP64: the chain is the oracle's move for move -- positions bit for bit (the moves use the same
words, the same uniform maps and a single rounding per coordinate update), ln psi and the
energy sums to 1e-10 relative, accepted-move counts exactly -- for every threads-per-walker
shape, both proposals, sequential order, the general exponent and the plain u.
FP32: the same decisions as the FP64 oracle except at near ties (a decision whose margin
2 Delta - ln xi is within FP32 rounding of zero may legitimately go either way).  The FP32
chains run one sweep per call (a run split at sweep boundaries is bit-identical), the oracle
reruns every sweep from the GPU's own state, and a sweep whose result differs must itself
contain a near tie -- a divergence is never excused by a tie elsewhere in the run.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1312_1282_gb300 as q
import qmc_inputs as qi
from tests._gpu import H2M, energy_scale, fp32_sweeps_vs_oracle, lattice_batch, report, zeros

pytestmark = pytest.mark.gpu


def _oracle_chain(P, w, seed, nsw, every, opt, k0=0, lp0=None, margins=False):
    W = oracle.make_walker(P.d[w].n, P.Ls[w], P.bs[w], P.ms[w], P.steps[w], sym=opt.sym, proposal=opt.proposal,
                           sequential=opt.sequential, hbar2_over_m=H2M, recompute_every=opt.recompute_every,
                           seed=seed, wid=P.ids[w])
    lp = oracle.log_psi(P.confs[w], P.Ls[w], P.bs[w], P.ms[w], opt.sym) if lp0 is None else lp0
    return oracle.run_walker(W, P.confs[w], lp, k0, nsw, every, margins=margins)


def _gpu_chain(P, seed, nsw, every, opt):
    lp = zeros(P.W)
    q.qmc_log_psi(P.d, opt, P.pos, lp)
    sw, acc = zeros(P.W, torch.int64), zeros((P.W, q.NACC))
    q.qmc_sweep(P.d, opt, P.pos, lp, sw, seed, nsw, every, acc)
    assert q.qmc_status(timeout_ms=120000) == 0
    return lp.cpu().numpy(), sw.cpu().numpy(), acc.cpu().numpy()


def _compare_fp64(P, seed, nsw, every, opt):
    lp, sw, acc = _gpu_chain(P, seed, nsw, every, opt)
    for w in range(P.W):
        pos, olp, ok, oacc, _ = _oracle_chain(P, w, seed, nsw, every, opt)
        g = P.positions(w)
        assert np.array_equal(g, pos) or np.abs(g - pos).max() < 1e-12, np.abs(g - pos).max()
        assert sw[w] == ok == nsw
        assert acc[w, 7] == oacc[7] and acc[w, 6] == oacc[6]
        np.testing.assert_allclose(acc[w, :6], oacc[:6], rtol=1e-10, atol=1e-9)
        assert abs(lp[w] - olp) <= 1e-10 * max(1.0, abs(olp))


@pytest.mark.parametrize("tpw", [32, 64, 128, 256])
def test_fp64_chain_matches_oracle_every_shape(tpw):
    P = lattice_batch([64, 130, 97, 257], q.QMC_FP64, seed=1, steps=0.8, ids=[0, 1, 2, 40000])
    opt = q.options(precision=q.QMC_FP64, recompute_every=7, threads_per_walker=tpw)
    _compare_fp64(P, 0xC0DE, 12, 3, opt)


def test_fp64_chain_ten_thousand_moves():
    P = lattice_batch([64, 64, 64], q.QMC_FP64, seed=2)
    opt = q.options(precision=q.QMC_FP64, recompute_every=50)
    _compare_fp64(P, 0x5EED0001, 160, 5, opt)


@pytest.mark.parametrize("variant", ["gauss", "sequential", "general_m", "plain_u", "large_tpw"])
def test_fp64_chain_variants(variant):
    kw = dict(precision=q.QMC_FP64, recompute_every=4)
    ms, steps = 5.0, 0.8
    if variant == "gauss":
        kw["proposal"] = q.QMC_GAUSS
        steps = 0.6
    elif variant == "sequential":
        kw["sequential"] = 1
    elif variant == "general_m":
        ms = 4.7
    elif variant == "plain_u":
        kw["sym"] = 0
    elif variant == "large_tpw":
        kw["threads_per_walker"] = 1024
    P = lattice_batch([64, 130, 2050], q.QMC_FP64, seed=3, ms=ms, steps=steps)
    opt = q.options(**kw)
    if variant == "gauss":
        lp, sw, acc = _gpu_chain(P, 9, 5, 1, opt)
        for w in range(P.W):
            pos, olp, _, oacc, _ = _oracle_chain(P, w, 9, 5, 1, opt)
            # Box-Muller goes through log/cos/sin of two different math libraries: equal
            # decisions, coordinates equal to rounding
            assert np.abs(P.positions(w) - pos).max() < 1e-9
            assert acc[w, 7] == oacc[7]
            np.testing.assert_allclose(acc[w, :6], oacc[:6], rtol=1e-9)
    else:
        _compare_fp64(P, 9, 4 if variant != "large_tpw" else 3, 2, opt)


def _gpu_sweeps(P, opt, seed, nsw, every=0, walkers=None):
    """nsw sweeps, one call each: the configuration of each listed walker before every sweep and
    after the last, and the moves it accepted in each sweep."""
    walkers = range(P.W) if walkers is None else walkers
    lp = zeros(P.W)
    q.qmc_log_psi(P.d, opt, P.pos, lp)
    sw, acc = zeros(P.W, torch.int64), zeros((P.W, q.NACC))
    states = {w: [P.positions(w)] for w in walkers}
    accepted = {w: [] for w in walkers}
    prev = np.zeros(P.W)
    for _ in range(nsw):
        q.qmc_sweep(P.d, opt, P.pos, lp, sw, seed, 1, every, acc)
        a = acc[:, 7].cpu().numpy()
        for w in walkers:
            states[w].append(P.positions(w))
            accepted[w].append(a[w] - prev[w])
        prev = a
    assert q.qmc_status(timeout_ms=120000) == 0
    return states, accepted, acc.cpu().numpy()


def test_fp32_chain_divergence_is_localised_to_a_near_tie():
    P = lattice_batch([64] * 12 + [130] * 4, q.QMC_FP32, seed=4)
    opt = q.options(precision=q.QMC_FP32, recompute_every=0)
    nsw = 20
    states, accepted, _ = _gpu_sweeps(P, opt, 77, nsw)
    agree, differ = 0, []
    for w in range(P.W):
        r = P.d[w]
        a, dif = fp32_sweeps_vs_oracle(states[w], accepted[w], r.n, P.Ls[w], P.bs[w], P.ms[w], P.steps[w], 77,
                                       P.ids[w])
        agree += a
        differ += dif
    report("fp32_chain_sweeps", sweeps=P.W * nsw, agree=agree, differ=len(differ),
           smallest_margin_of_differing=min([m for _, m in differ], default=0.0))
    assert agree >= P.W * nsw - 3


def test_resume_is_bitwise_identical():
    for prec in (q.QMC_FP32, q.QMC_FP64):
        A = lattice_batch([64, 130, 512], prec, seed=5)
        B = lattice_batch([64, 130, 512], prec, seed=5)
        opt = q.options(precision=prec, recompute_every=3)
        la, sa, aa = zeros(3), zeros(3, torch.int64), zeros((3, q.NACC))
        lb, sb, ab = zeros(3), zeros(3, torch.int64), zeros((3, q.NACC))
        q.qmc_sweep(A.d, opt, A.pos, la, sa, 11, 10, 2, aa)
        q.qmc_sweep(B.d, opt, B.pos, lb, sb, 11, 4, 2, ab)
        q.qmc_sweep(B.d, opt, B.pos, lb, sb, 11, 6, 2, ab)
        torch.cuda.synchronize()
        assert torch.equal(A.pos, B.pos) and torch.equal(la, lb) and torch.equal(sa, sb)
        assert torch.equal(aa[:, :8], ab[:, :8])
        # the ln psi drift (fields 8, 9) measures the rounding of the carried sum; a call boundary
        # collapses its compensated-float part into the stored double once more, which moves it by
        # the rounding of that FP32 sum (here the drift also holds the start's ln psi, left at 0)
        np.testing.assert_allclose(aa[:, 8:].cpu().numpy(), ab[:, 8:].cpu().numpy(), rtol=1e-6, atol=1e-9)


def test_autotune_keeps_the_chain():
    P = lattice_batch([512] * 8, q.QMC_FP32, seed=6)
    Q = lattice_batch([512] * 8, q.QMC_FP32, seed=6)
    opt = q.options(precision=q.QMC_FP32)
    t, g = q.qmc_autotune(P.d, opt, P.pos)
    assert t in (32, 64, 128, 256, 512, 1024) and g in (1, 2, 4, 8) and g * t <= max(256, t)
    torch.cuda.synchronize()
    assert torch.equal(P.pos, Q.pos)  # tuning runs on a scratch copy
    for shape in (t, 32):
        o = q.options(precision=q.QMC_FP32, threads_per_walker=shape)
        R = lattice_batch([512] * 8, q.QMC_FP32, seed=6)
        lp, sw, acc = zeros(8), zeros(8, torch.int64), zeros((8, q.NACC))
        q.qmc_sweep(R.d, o, R.pos, lp, sw, 3, 2, 0, acc)
        torch.cuda.synchronize()
        if shape == t:
            ref = (R.pos.clone(), acc[:, 7].clone())
        else:
            # another thread shape sums the partners in another order: same chain except at ties
            assert (acc[:, 7] == ref[1]).sum() >= 7


def test_full_size_sampled_walkers():
    """N = 1952, 528 walkers, FP32, in the benchmark's launch shape: one sweep from the fcc start,
    then three sampled walkers rerun by the oracle move by move, and their final configurations'
    energies checked against the oracle."""
    n, W = 1952, 528
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)
    d = q.descs([(n, pad, w * 3 * pad, w, L, 0.0, qi.B_HE, 5.0, 0.8) for w in range(W)])
    opt = q.options(precision=q.QMC_FP32, recompute_every=50)
    pos = torch.empty(W * 3 * pad, dtype=torch.float32, device="cuda")
    q.qmc_init_walkers(d, 0x5EED0003, 0.1, opt, pos)
    start = pos.cpu().numpy().astype(np.float64)
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(d, opt, pos, lp)
    q.qmc_sweep(d, opt, pos, lp, sw, 0x5EED0003, 1, 1, acc)
    assert q.qmc_status(timeout_ms=300000) == 0
    host = pos.cpu().numpy().astype(np.float64)
    a = acc.cpu().numpy()
    matched = 0
    for w in (0, 263, 527):
        blk0 = start[w * 3 * pad:(w + 1) * 3 * pad].reshape(3, pad)[:, :n]
        blk1 = host[w * 3 * pad:(w + 1) * 3 * pad].reshape(3, pad)[:, :n]
        Wk = oracle.make_walker(n, L, qi.B_HE, 5.0, 0.8, seed=0x5EED0003, wid=w, hbar2_over_m=H2M)
        opos, _, _, oacc, mg = oracle.run_walker(Wk, blk0, 0.0, 0, 1, 0, margins=True)
        if a[w, 7] == oacc[7] and np.abs(blk1 - opos).max() < 1e-3:
            matched += 1
        else:
            assert np.abs(mg).min() < 1e-3
        e = oracle.local_energy(blk1, L, qi.B_HE, 5.0, 1, H2M)
        assert np.all(np.abs(a[w, [2, 3, 4, 5, 0]] - e) <= 1e-5 * energy_scale(e))
    assert matched >= 2


def test_persistent_queue_mode_matches_oracle_and_static_path():
    """More walkers than SMs: qmc_sweep runs persistent CTAs that take walkers from a FIFO in
    chunks of moves.  The chains must be those of the oracle (FP64, bit for bit) and of the
    one-walker-per-group path of qmc_sweep_static, for an uneven batch."""
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    W = nsm + 37
    ns = [64, 130, 200, 97] * (W // 4) + [64] * (W % 4)
    A = lattice_batch(ns, q.QMC_FP64, seed=8)
    B = lattice_batch(ns, q.QMC_FP64, seed=8)
    opt = q.options(precision=q.QMC_FP64, recompute_every=3)
    la, sa, aa = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    lb, sb, ab = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(A.d, opt, A.pos, la)
    q.qmc_log_psi(B.d, opt, B.pos, lb)
    q.qmc_sweep(A.d, opt, A.pos, la, sa, 0xD1CE, 4, 2, aa)
    q.qmc_sweep(A.d, opt, A.pos, la, sa, 0xD1CE, 3, 2, aa)
    q.qmc_sweep_static(B.d, opt, B.pos, lb, sb, 0xD1CE, 7, 2, ab)
    assert q.qmc_status(timeout_ms=120000) == 0
    assert torch.equal(A.pos, B.pos) and torch.equal(sa, sb)
    np.testing.assert_allclose(la.cpu().numpy(), lb.cpu().numpy(), rtol=1e-12)
    np.testing.assert_allclose(aa.cpu().numpy(), ab.cpu().numpy(), rtol=1e-12)
    acc = aa.cpu().numpy()
    for w in (0, 1, 2, 3, W - 1):
        pos, olp, ok, oacc, _ = _oracle_chain(A, w, 0xD1CE, 7, 2, opt)
        assert np.array_equal(A.positions(w), pos)
        assert acc[w, 7] == oacc[7] and acc[w, 6] == oacc[6]
        np.testing.assert_allclose(acc[w, :6], oacc[:6], rtol=1e-10, atol=1e-9)


def test_uneven_batch_with_a_dominant_walker():
    """An uneven batch in which one walker's pair work dominates, in FP64 (the persistent queue;
    FP32 batches of this kind run the mixed kernel, tested below).  Chains as the oracle's (bit
    for bit) and as the one-walker-per-group path."""
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    ns = [600] + [64] * (nsm + 20)
    W = len(ns)
    A = lattice_batch(ns, q.QMC_FP64, seed=9)
    B = lattice_batch(ns, q.QMC_FP64, seed=9)
    opt = q.options(precision=q.QMC_FP64, recompute_every=2)
    la, sa, aa = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    lb, sb, ab = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_log_psi(A.d, opt, A.pos, la)
    q.qmc_log_psi(B.d, opt, B.pos, lb)
    q.qmc_sweep(A.d, opt, A.pos, la, sa, 0xB16, 3, 1, aa)
    q.qmc_sweep_static(B.d, opt, B.pos, lb, sb, 0xB16, 3, 1, ab)
    assert q.qmc_status(timeout_ms=120000) == 0
    assert torch.equal(A.pos, B.pos) and torch.equal(sa, sb)
    np.testing.assert_allclose(la.cpu().numpy(), lb.cpu().numpy(), rtol=1e-12)
    np.testing.assert_allclose(aa.cpu().numpy(), ab.cpu().numpy(), rtol=1e-12)
    acc = aa.cpu().numpy()
    for w in (0, 1, W - 1):
        pos, olp, ok, oacc, _ = _oracle_chain(A, w, 0xB16, 3, 1, opt)
        assert np.array_equal(A.positions(w), pos)
        assert acc[w, 7] == oacc[7] and acc[w, 6] == oacc[6]


@pytest.mark.parametrize("tpw", [64, 128])
def test_mixed_sweep_matches_oracle_and_energy_pass(tpw):
    """FP32 uneven batch with a dominant walker: the mixed kernel runs it on a whole CTA of 256
    threads and the other walkers on groups of tpw threads from the queue.  Chains as the oracle's
    decision by decision (except near ties), the energy samples as the stand-alone pass."""
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    ns = [600, 600] + [64] * (nsm + 30)
    W = len(ns)
    P = lattice_batch(ns, q.QMC_FP32, seed=10)
    opt = q.options(precision=q.QMC_FP32, recompute_every=0, threads_per_walker=tpw)
    picks = (0, 2, W - 1)
    # two sweeps, one per call, the energy sampled after the second
    states, accepted, a = _gpu_sweeps(P, opt, 0x313, 2, every=2, walkers=picks)
    e = zeros((W, 5))
    q.qmc_local_energy(P.d, q.options(precision=q.QMC_FP32), P.pos, e)
    assert q.qmc_status(timeout_ms=120000) == 0
    assert np.all(a[:, 6] == 1)
    en = e.cpu().numpy()
    for w in range(W):
        assert np.all(np.abs(a[w, [2, 3, 4, 5, 0]] - en[w]) <= 1e-5 * energy_scale(en[w])), w
    agree = 0
    for w in picks:
        r = P.d[w]
        agree += fp32_sweeps_vs_oracle(states[w], accepted[w], r.n, P.Ls[w], P.bs[w], P.ms[w], P.steps[w], 0x313,
                                       P.ids[w])[0]
    assert agree >= 2 * len(picks) - 1


def test_persistent_queue_mode_survives_a_faulted_walker():
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    W = nsm + 5
    P = lattice_batch([64] * W, q.QMC_FP32, seed=9)
    before = P.pos.clone()
    bad = P.d[3]
    P.pos[bad.offset + 7] = float("nan")
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_sweep(P.d, q.options(), P.pos, lp, sw, 4, 6, 3, acc)
    with pytest.raises(q.QmcError, match="bad coordinate"):
        q.qmc_status(timeout_ms=120000)
    s = sw.cpu().numpy()
    assert s[3] == 0 and np.all(np.delete(s, 3) == 6)
    host = P.pos.cpu()
    assert torch.equal(host[bad.offset + 8:bad.offset + 3 * 64], before[bad.offset + 8:bad.offset + 3 * 64].cpu())
