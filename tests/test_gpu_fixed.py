"""GPU vs oracle on fixed configurations: local energy, ln psi, (b, m) gradient, trial ratios
and start configurations, through the C ABI.  FP64: 1e-10 relative; FP32: 1e-5 relative
(the tolerances of the method's fixed-configuration parity), on batches whose sizes span
several partner chunks and thread groups with ragged tails.  Quantities that are differences
(T_L, E_L, the derivatives of E_L, a trial ratio) are compared on the sum of the magnitudes of
the terms they are made of, computed from the oracle's pair terms; the achieved errors, on that
scale and on each output's own magnitude, go to the QMC_PARITY_REPORT file when it is set."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1312_1282_gb300 as q
import qmc_inputs as qi
from tests._gpu import H2M, Packed, energy_scale, grad_scales, lattice_batch, report, trial_scale, zeros

pytestmark = pytest.mark.gpu

NS = [2, 3, 5, 17, 64, 130, 257, 512, 1001]
TOL = {q.QMC_FP64: 1e-10, q.QMC_FP32: 1e-5}
PREC = [q.QMC_FP64, q.QMC_FP32]


def _close(got, want, rel, scale=None):
    scale = np.maximum(np.abs(want), 1e-300) if scale is None else scale
    err = np.abs(np.asarray(got) - np.asarray(want)) / scale
    assert np.all(err <= rel), (err.max(), got, want)
    return err


@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("sym,m", [(1, 5.0), (1, 4.6), (0, 5.0)])
def test_local_energy(prec, sym, m):
    P = lattice_batch(NS, prec, seed=10, ms=m)
    opt = q.options(precision=prec, sym=sym)
    out = zeros((P.W, 5))
    q.qmc_local_energy(P.d, opt, P.pos, out)
    got = out.cpu().numpy()
    worst, worst_own = np.zeros(5), np.zeros(5)
    for w in range(P.W):
        want = oracle.local_energy(P.confs[w], P.Ls[w], P.bs[w], m, sym, H2M)
        # T_L and E_L are differences: compared on the scale of the sums they are built from
        err = _close(got[w], want, TOL[prec], energy_scale(want))
        worst = np.maximum(worst, err)
        if P.confs[w].shape[1] >= 17:  # below that E_L can pass through zero
            worst_own = np.maximum(worst_own, np.abs(got[w] - want) / np.maximum(np.abs(want), 1e-300))
    # the achieved error on each output's own magnitude (E_L and T_L included), for the record
    report("local_energy", prec=prec, sym=sym, m=m, fields="V,T_L,T_PB,T_F,E_L", err_on_summed_scale=worst,
           err_on_own_magnitude=worst_own)


@pytest.mark.parametrize("prec", PREC)
def test_log_psi(prec):
    P = lattice_batch(NS, prec, seed=20)
    out = zeros(P.W)
    q.qmc_log_psi(P.d, q.options(precision=prec), P.pos, out)
    want = [oracle.log_psi(P.confs[w], P.Ls[w], P.bs[w]) for w in range(P.W)]
    _close(out.cpu().numpy(), want, TOL[prec])


@pytest.mark.parametrize("prec", PREC)
def test_energy_grad(prec):
    ns = [2, 17, 64, 130, 512]
    P = lattice_batch(ns, prec, seed=30, bs=[2.95, 3.0, 3.07, 3.1, 3.2])
    out = zeros((P.W, 6))
    q.qmc_energy_grad(P.d, q.options(precision=prec), P.pos, out)
    got = out.cpu().numpy()
    worst, worst_own = np.zeros(6), np.zeros(6)
    for w in range(P.W):
        want = oracle.energy_grad(P.confs[w], P.Ls[w], P.bs[w], 5.0, 1, H2M)
        # each output on the sum of the magnitudes of the pair terms it is made of (the
        # derivatives of E_L are sums of kinetic terms of both signs)
        scale = grad_scales(P.confs[w], P.Ls[w], P.bs[w], 5.0, 1, H2M)
        err = _close(got[w], want, TOL[prec], np.maximum(scale, 1e-12))
        worst = np.maximum(worst, err)
        worst_own = np.maximum(worst_own, np.abs(got[w] - want) / np.maximum(np.abs(want), 1e-300))
    report("energy_grad", prec=prec, fields="lnpsi,E_L,dlnpsi_db,dlnpsi_dm,dEL_db,dEL_dm", err_on_term_scale=worst,
           err_on_own_magnitude=worst_own)


@pytest.mark.parametrize("prec", PREC)
def test_trial_delta(prec):
    ns = [3, 17, 64, 130, 512, 1001]
    P = lattice_batch(ns, prec, seed=40)
    M = 24
    rng = np.random.default_rng(5)
    s = np.stack([rng.integers(0, n, size=M) for n in ns]).astype(np.int32)
    delta = rng.uniform(-1.5, 1.5, size=(P.W, M, 3))
    out = zeros((P.W, M))
    q.qmc_trial_delta(P.d, q.options(precision=prec), P.pos, torch.tensor(s, device="cuda"),
                      torch.tensor(delta, device="cuda"), M, out)
    got = out.cpu().numpy()
    worst = 0.0
    for w in range(P.W):
        for k in range(M):
            d = delta[w, k]
            if prec == q.QMC_FP32:
                d = d.astype(np.float32).astype(np.float64)
            want, new = oracle.trial_delta(P.confs[w], P.Ls[w], P.bs[w], 5.0, 1, s[w, k], d)
            # Delta -> 0 cancels: absolute error on sum_j (|u| + |u'|) at the old and new distances
            scale = trial_scale(P.confs[w], P.Ls[w], P.bs[w], 5.0, 1, s[w, k], new) + 1e-300
            err = abs(got[w, k] - want) / scale
            assert err <= TOL[prec], (w, k, got[w, k], want, scale)
            worst = max(worst, err)
    report("trial_delta", prec=prec, err_on_term_scale=worst)


@pytest.mark.parametrize("prec", PREC)
def test_init_walkers_match_oracle(prec):
    ns = [2, 64, 130, 500, 1952]
    rows, off = [], 0
    for i, n in enumerate(ns):
        pad = qi.pad4(n)
        rows.append((n, pad, off, 7 + i, 0.0, qi.RHO_HE, 3.07, 5.0, 0.8))
        off += 3 * pad
    d = q.descs(rows)
    dt = torch.float64 if prec == q.QMC_FP64 else torch.float32
    pos = torch.full((off,), -1.0, dtype=dt, device="cuda")
    q.qmc_init_walkers(d, 0x5EED0002, 0.1, q.options(precision=prec), pos)
    host = pos.cpu().numpy().astype(np.float64)
    for i, n in enumerate(ns):
        L = (n / qi.RHO_HE) ** (1 / 3)
        r = rows[i]
        blk = host[r[2]:r[2] + 3 * r[1]].reshape(3, r[1])
        want = oracle.init_walker(n, L, 0x5EED0002, 7 + i, 0.1)
        atol = 1e-12 * L if prec == q.QMC_FP64 else 2 * np.spacing(np.float32(L))
        assert np.allclose(blk[:, :n], want, rtol=0, atol=atol)
        assert np.all(blk[:, n:] == 0.0)


def test_padding_is_ignored_and_left_alone():
    P = lattice_batch([5, 130], q.QMC_FP32, seed=50, junk=float("nan"))
    out = zeros((P.W, 5))
    q.qmc_local_energy(P.d, q.options(), P.pos, out)
    assert torch.isfinite(out).all()
    lp, sw, acc = zeros(P.W), zeros(P.W, torch.int64), zeros((P.W, q.NACC))
    q.qmc_sweep(P.d, q.options(), P.pos, lp, sw, 1, 2, 1, acc)
    assert q.qmc_status(timeout_ms=60000) == 0
    assert np.all(np.isnan(P.padding(0))) and np.all(np.isnan(P.padding(1)))


def test_capacity_and_argument_errors():
    big = lattice_batch([2], q.QMC_FP32)
    # start lattices beyond one CTA's shared memory are refused on the host, before any launch
    rows = [(60000, 60000, 0, 0, 140.0, 0, 3.07, 5.0, 0.8)]
    with pytest.raises(q.QmcError, match="CAPACITY"):
        q.qmc_init_walkers(q.descs(rows), 1, 0.1, q.options(), big.pos)
    for bad in [(1, 4, 0, 0, 10.0, 0, 3.0, 5.0, 0.8), (8, 6, 0, 0, 10.0, 0, 3.0, 5.0, 0.8),
                (8, 8, 2, 0, 10.0, 0, 3.0, 5.0, 0.8), (8, 8, 0, 0, 0.0, 0.0, 3.0, 5.0, 0.8),
                (8, 8, 0, 0, 10.0, 0, -1.0, 5.0, 0.8), (8, 8, 0, 0, 10.0, 0, 3.0, 5.0, 11.0),
                (8, 8, 0, 0, 10.0, 0, math.nan, 5.0, 0.8)]:
        with pytest.raises(q.QmcError, match="ARG"):
            q.qmc_local_energy(q.descs([bad]), q.options(), big.pos, zeros(5))


def test_gaussian_step_is_checked_on_a_batch_registered_by_a_cube_call():
    """The step check depends on the proposal: a Gaussian displacement reaches about 6.8 sigma,
    a cube one its half-width.  A batch first registered by a cube-proposal call (which caches its
    walker table) must still refuse a Gaussian call whose reach is a box side or more, before
    anything is enqueued, and must keep working for the cube proposal."""
    n = 64
    L = qi.box_side(n, qi.RHO_HE)  # 14.3 A: a 3 A step is fine for the cube, 6.8 x 3 A is not
    P = lattice_batch([n], q.QMC_FP32, seed=90, steps=3.0)
    lp, sw, acc = zeros(1), zeros(1, torch.int64), zeros((1, q.NACC))
    q.qmc_sweep(P.d, q.options(), P.pos, lp, sw, 5, 1, 0, acc)
    assert q.qmc_status(timeout_ms=60000) == 0
    before = P.pos.clone()
    with pytest.raises(q.QmcError, match="ARG.*step too large"):
        q.qmc_sweep(P.d, q.options(proposal=q.QMC_GAUSS), P.pos, lp, sw, 5, 1, 0, acc)
    assert torch.equal(P.pos, before) and sw.cpu().tolist() == [1]
    q.qmc_sweep(P.d, q.options(), P.pos, lp, sw, 5, 1, 0, acc)
    assert q.qmc_status(timeout_ms=60000) == 0 and sw.cpu().tolist() == [2]
    assert 3.0 < L < 6.8 * 3.0


def test_nonfinite_coordinates_are_flagged_not_faulted():
    P = lattice_batch([64, 64], q.QMC_FP32, seed=60)
    before = P.pos.clone()
    r = P.d[1]
    P.pos[r.offset + 5] = float("nan")
    lp, sw, acc = zeros(P.W), zeros(P.W, torch.int64), zeros((P.W, q.NACC))
    q.qmc_sweep(P.d, q.options(), P.pos, lp, sw, 3, 2, 0, acc)
    with pytest.raises(q.QmcError, match="DEVICE"):
        q.qmc_status(timeout_ms=60000)
    assert q.qmc_status(timeout_ms=60000) == 0  # the word is cleared by reading it
    host = P.pos.cpu()
    assert not torch.equal(host[:3 * 64], before[:3 * 64].cpu())       # walker 0 moved
    assert torch.equal(host[r.offset + 6:r.offset + 3 * 64], before[r.offset + 6:r.offset + 3 * 64].cpu())
    assert sw.cpu().tolist() == [2, 0]


@pytest.mark.parametrize("prec", PREC)
def test_pair_histogram(prec):
    ns = [2, 17, 64, 130, 512]
    P = lattice_batch(ns, prec, seed=80)
    nbins = 64
    hist = zeros((P.W, nbins), torch.int64)
    rmax = [L / 2 for L in P.Ls]
    # one call per walker because rmax differs; the second call on the same rows adds
    for w in range(P.W):
        one = q.descs([tuple(getattr(P.d[w], f) for f, _ in q.WalkerDesc._fields_)])
        one[0].offset = 0
        r = P.d[w]
        sub = P.pos[r.offset:r.offset + 3 * r.pad_n].contiguous()
        q.qmc_pair_hist(one, q.options(precision=prec), sub, nbins, rmax[w], hist[w])
        q.qmc_pair_hist(one, q.options(precision=prec), sub, nbins, rmax[w], hist[w])
    got = hist.cpu().numpy()
    for w in range(P.W):
        want = 2 * oracle.pair_hist(P.confs[w], P.Ls[w], nbins, rmax[w]).astype(np.int64)
        if prec == q.QMC_FP64:
            assert np.array_equal(got[w], want)
        else:
            # FP32 distances may move a pair whose r lies within 1e-5 (relative) of a bin edge or
            # of r_max into the neighbouring bin, and no other pair
            c = P.confs[w]
            d = c[:, :, None] - c[:, None, :]
            d -= P.Ls[w] * np.rint(d / P.Ls[w])
            iu = np.triu_indices(c.shape[1], 1)
            x = np.sqrt((d ** 2).sum(axis=0))[iu] * nbins / rmax[w]
            near = np.abs(x - np.rint(x)) < 1e-5 * np.maximum(x, 1.0)
            edge = near & (np.rint(x) == nbins)
            diff = got[w] - want
            assert abs(int(diff.sum())) <= 2 * int(edge.sum())
            assert int(np.abs(diff).sum()) <= 4 * int(near.sum())
            # a bin may change only by pairs near one of its two edges
            k = np.rint(x[near]).astype(int)
            allow = np.zeros(nbins + 1, dtype=np.int64)
            np.add.at(allow, np.clip(k, 0, nbins), 1)
            per_bin = 2 * (allow[:-1] + allow[1:])
            assert np.all(np.abs(diff) <= per_bin)


def test_pair_correlation_of_a_liquid():
    n, W = 512, 64
    L = qi.box_side(n, qi.RHO_HE)
    pad = qi.pad4(n)
    d = q.descs([(n, pad, w * 3 * pad, w, L, 0.0, qi.B_HE, 5.0, 0.8) for w in range(W)])
    opt = q.options()
    pos = torch.empty(W * 3 * pad, dtype=torch.float32, device="cuda")
    q.qmc_init_walkers(d, 21, 0.1, opt, pos)
    lp, sw, acc = zeros(W), zeros(W, torch.int64), zeros((W, q.NACC))
    q.qmc_sweep(d, opt, pos, lp, sw, 21, 300, 0, acc)
    nbins, rmax = 70, L / 2
    hist = zeros((W, nbins), torch.int64)
    for _ in range(10):
        q.qmc_sweep(d, opt, pos, lp, sw, 21, 5, 0, acc)
        q.qmc_pair_hist(d, opt, pos, nbins, rmax, hist)
    r, g = q.pair_correlation(hist.sum(0).cpu().numpy(), n, L, rmax, 10 * W)
    assert np.all(g[r < 1.8] == 0.0)           # hard core of the Jastrow factor
    assert 1.2 < g.max() < 1.8 and 3.0 < r[np.argmax(g)] < 4.0   # first shell of liquid 4He
    assert abs(g[(r > 9) & (r < 12)].mean() - 1.0) < 0.05


def test_split_passes_match_oracle():
    # Two walkers of N = 2048 in FP64: with far fewer walkers than SMs every row-wise pass splits
    # each walker's rows over several CTAs, whose shares the last CTA of the walker adds up (ln psi,
    # local energy, adjoint) or which add their counts atomically (histogram).
    P = lattice_batch([2048, 2044], q.QMC_FP64, seed=90)
    opt = q.options(precision=q.QMC_FP64)
    lp, e, g = zeros(P.W), zeros((P.W, 5)), zeros((P.W, 6))
    nbins = 50
    hist = zeros((P.W, nbins), torch.int64)
    for _ in range(2):  # the second call of each pass finds the counters reset by the first
        q.qmc_log_psi(P.d, opt, P.pos, lp)
        q.qmc_local_energy(P.d, opt, P.pos, e)
        q.qmc_energy_grad(P.d, opt, P.pos, g)
    rmax = min(P.Ls) / 2
    q.qmc_pair_hist(P.d, opt, P.pos, nbins, rmax, hist)
    assert q.qmc_status(timeout_ms=120000) == 0
    for w in range(P.W):
        c, L, b = P.confs[w], P.Ls[w], P.bs[w]
        _close(lp.cpu().numpy()[w], oracle.log_psi(c, L, b), 1e-10)
        want = oracle.local_energy(c, L, b, 5.0, 1, H2M)
        _close(e.cpu().numpy()[w], want, 1e-10, energy_scale(want))
        wg = oracle.energy_grad(c, L, b, 5.0, 1, H2M)
        _close(g.cpu().numpy()[w], wg, 1e-10, grad_scales(c, L, b, 5.0, 1, H2M, rows=64))
        assert np.array_equal(hist.cpu().numpy()[w], oracle.pair_hist(c, L, nbins, rmax).astype(np.int64))
