"""Pins of the FP64 oracle to facts fixed outside it (CPU only).

Each test checks one oracle routine against something the oracle does not compute itself:
a published known-answer vector, the physical constants of the potential, a closed form,
an invariance of the many-body wavefunction, a finite difference, or a brute-force
re-evaluation on a tiny input.  A dropped term, a wrong sign, a wrong power or a wrong image
convention in the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import qmc_inputs as qi

GOLD = os.path.join(os.path.dirname(__file__), "golden")
H2M = qi.HBAR2_OVER_M


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------------------------

def test_philox_known_answers():
    for row in _golden_rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_move_randoms_distributions():
    n, step = 37, 0.8
    S, D, X = [], [], []
    for k in range(40):
        for t in range(n):
            s, d, xi = oracle.move_randoms(0x1234, 7, 0, 0, n, t, k, step)
            S.append(s); D.append(d); X.append(xi)
    S, D, X = np.array(S), np.array(D), np.array(X)
    assert S.min() >= 0 and S.max() < n
    counts = np.bincount(S, minlength=n)
    chi2 = ((counts - len(S) / n) ** 2 / (len(S) / n)).sum()
    assert chi2 < n + 6 * math.sqrt(2 * n)
    assert np.all(np.abs(D) < step)
    assert abs(D.mean()) < 4 * step / math.sqrt(3 * D.size)
    assert abs(D.var() / (step ** 2 / 3) - 1) < 0.05
    assert np.all((X > 0) & (X < 1))
    assert abs(X.mean() - 0.5) < 4 * math.sqrt(1 / 12 / X.size)
    # sequential mode visits s = t
    assert [oracle.move_randoms(1, 2, 0, 1, 5, t, 0, step)[0] for t in range(5)] == list(range(5))


def test_gaussian_proposal_moments():
    step = 1.1
    D = np.array([oracle.move_randoms(99, 3, 1, 0, 10, t, k, step)[1] for k in range(300) for t in range(10)])
    assert abs(D.mean()) < 4 * step / math.sqrt(D.size)
    assert abs(D.var() / step ** 2 - 1) < 0.06
    # fourth moment of a normal: 3 sigma^4 (a uniform would give 1.8)
    assert abs((D ** 4).mean() / step ** 4 / 3 - 1) < 0.15


# --------------------------------------------------------------------------------------------
# pair potential
# --------------------------------------------------------------------------------------------

def test_aziz_minimum_and_depth():
    g = dict((r[0], float(r[1])) for r in _golden_rows("aziz_hfdb_he.txt"))
    eps, rm = g["epsilon_K"], g["r_m_A"]
    from scipy.optimize import minimize_scalar
    res = minimize_scalar(oracle.aziz, bounds=(2.5, 3.5), method="bounded", options={"xatol": 1e-10})
    assert abs(res.x - rm) < 1e-5
    assert abs(oracle.aziz(rm) + eps) < 1e-4 * eps
    h = 1e-5
    assert abs((oracle.aziz(rm + h) - oracle.aziz(rm - h)) / (2 * h)) < 1e-3
    # steep but finite repulsive wall, weak attractive tail
    assert 1e5 < oracle.aziz(0.5) < 1e7
    assert oracle.aziz(2.0) > 0 > oracle.aziz(2.7)
    assert -0.1 < oracle.aziz(8.0) < 0


# --------------------------------------------------------------------------------------------
# pair correlation exponent u(r)
# --------------------------------------------------------------------------------------------

def test_u_closed_form_values():
    L, b = 40.0, 3.07
    # plain Schiff-Verlet form: u(b) = -1/2, u(2b) = -1/2 * 2^-5 = -1/64, zero past L/2
    assert oracle.pair_u(b, L, b, 5.0, 0)[0] == pytest.approx(-0.5, rel=1e-14)
    assert oracle.pair_u(2 * b, L, b, 5.0, 0)[0] == pytest.approx(-1.0 / 64.0, rel=1e-14)
    assert oracle.pair_u(2 * b, L, b, 3.0, 0)[0] == pytest.approx(-1.0 / 16.0, rel=1e-14)
    for sym in (0, 1):
        assert np.all(oracle.pair_u(0.5 * L, L, b, 5.0, sym) == 0.0)
        assert np.all(oracle.pair_u(0.7 * L, L, b, 5.0, sym) == 0.0)
    # symmetrised u: sum of the two plain pieces at r and L - r, shifted to vanish at L/2
    r = 7.3
    plain = lambda rr: -0.5 * (b / rr) ** 5  # noqa: E731  (Eq. fifthPower)
    want = plain(r) + plain(L - r) - 2 * plain(L / 2)
    assert oracle.pair_u(r, L, b, 5.0, 1)[0] == pytest.approx(want, rel=1e-13)


def test_u_is_c1_at_half_box():
    L, b = 20.0, 3.07
    p = oracle.pair_u(0.5 * L - 1e-7, L, b, 5.0, 1)
    assert abs(p[0]) < 1e-12 and abs(p[1]) < 1e-9
    # the truncated form is not: it jumps at L/2
    assert abs(oracle.pair_u(0.5 * L - 1e-7, L, b, 5.0, 0)[0]) > 1e-6


@pytest.mark.parametrize("sym", [0, 1])
@pytest.mark.parametrize("r", [2.1, 2.9, 4.4, 8.0])
def test_u_derivatives_by_finite_differences(sym, r):
    L, b, m = 18.0, 3.07, 5.0
    p = oracle.pair_u(r, L, b, m, sym)
    h = 1e-5 * r
    up = oracle.pair_u(r + h, L, b, m, sym)
    um = oracle.pair_u(r - h, L, b, m, sym)
    assert p[1] == pytest.approx((up[0] - um[0]) / (2 * h), rel=1e-7, abs=1e-12)
    assert p[2] == pytest.approx((up[1] - um[1]) / (2 * h), rel=1e-7, abs=1e-12)
    hb = 1e-6 * b
    bp, bm = oracle.pair_u(r, L, b + hb, m, sym), oracle.pair_u(r, L, b - hb, m, sym)
    for i in range(3):
        assert p[3 + i] == pytest.approx((bp[i] - bm[i]) / (2 * hb), rel=1e-7, abs=1e-12)
    hm = 1e-6
    mp, mm = oracle.pair_u(r, L, b, m + hm, sym), oracle.pair_u(r, L, b, m - hm, sym)
    for i in range(3):
        assert p[6 + i] == pytest.approx((mp[i] - mm[i]) / (2 * hm), rel=1e-6, abs=1e-12)


# --------------------------------------------------------------------------------------------
# many-body quantities
# --------------------------------------------------------------------------------------------

def _brute_pairs(pos, L):
    """All pairs i<j with their minimum-image distance, found by enumerating the 27 images."""
    n = pos.shape[1]
    shifts = np.array(list(itertools.product((-1, 0, 1), repeat=3)), dtype=float) * L
    out = []
    for i in range(n):
        for j in range(i + 1, n):
            d = pos[:, i] - pos[:, j]
            out.append((i, j, np.min(np.linalg.norm(d[None, :] + shifts, axis=1))))
    return out


def test_log_psi_and_potential_by_brute_force_images():
    n, L, b = 9, 7.5, 3.07
    pos = qi.uniform_positions(n, L, 3)
    for sym in (0, 1):
        lp = sum(oracle.pair_u(r, L, b, 5.0, sym)[0] for _, _, r in _brute_pairs(pos, L))
        assert oracle.log_psi(pos, L, b, 5.0, sym) == pytest.approx(lp, rel=1e-12)
    V = sum(oracle.aziz(r) for _, _, r in _brute_pairs(pos, L) if r < L / 2)
    assert oracle.local_energy(pos, L, b)[0] == pytest.approx(V, rel=1e-12)


def _all_outputs(pos, L, b, m=5.0):
    return np.concatenate([[oracle.log_psi(pos, L, b, m)], oracle.local_energy(pos, L, b, m),
                           oracle.energy_grad(pos, L, b, m)])


def test_translation_permutation_image_invariance():
    n = 40
    L = qi.box_side(n, qi.RHO_HE)
    pos = qi.jittered_lattice(n, L, 11)
    ref = _all_outputs(pos, L, 3.07)
    rng = np.random.default_rng(0)
    shifted = np.mod(pos + rng.uniform(-L, L, size=(3, 1)), L)
    perm = pos[:, rng.permutation(n)]
    images = pos + L * rng.integers(-2, 3, size=pos.shape)
    for alt in (shifted, perm, images):
        assert np.allclose(_all_outputs(alt, L, 3.07), ref, rtol=1e-11, atol=0)


def test_incremental_ratio_equals_full_recompute():
    n = 30
    L = qi.box_side(n, qi.RHO_HE)
    pos = qi.jittered_lattice(n, L, 5)
    base = oracle.log_psi(pos, L, 3.07)
    scale = sum(abs(oracle.pair_u(r, L, 3.07)[0]) for _, _, r in _brute_pairs(pos, L))
    rng = np.random.default_rng(1)
    for _ in range(25):
        s = int(rng.integers(n))
        # large steps so that some moves cross the box faces and get wrapped
        delta = rng.uniform(-2.5, 2.5, size=3)
        D, npos = oracle.trial_delta(pos, L, 3.07, 5.0, 1, s, delta)
        assert np.all((npos >= 0) & (npos <= L))
        moved = pos.copy()
        moved[:, s] = npos
        assert abs(D - (oracle.log_psi(moved, L, 3.07) - base)) < 1e-12 * scale


def test_drift_and_laplacian_by_finite_differences():
    n = 12
    L = qi.box_side(n, qi.RHO_HE)
    pos = qi.jittered_lattice(n, L, 2)
    b = 3.07
    lap, F = oracle.local_terms(pos, L, b)
    lp0 = oracle.log_psi(pos, L, b)
    h1, h2 = 1e-5, 1e-4
    for i in range(n):
        for c in range(3):
            p, m = pos.copy(), pos.copy()
            p[c, i] += h1
            m[c, i] -= h1
            fd = (oracle.log_psi(p, L, b) - oracle.log_psi(m, L, b)) / (2 * h1)
            assert F[i, c] == pytest.approx(fd, rel=1e-6, abs=1e-8)
        acc = 0.0
        for c in range(3):
            p, m = pos.copy(), pos.copy()
            p[c, i] += h2
            m[c, i] -= h2
            acc += (oracle.log_psi(p, L, b) - 2 * lp0 + oracle.log_psi(m, L, b)) / h2 ** 2
        assert lap[i] == pytest.approx(acc, rel=1e-5, abs=1e-6)


def test_local_kinetic_energy_is_laplacian_of_psi():
    """T_L = -(hbar^2/2m) sum_i nabla_i^2 psi / psi, with psi itself differentiated."""
    n = 10
    L = qi.box_side(n, qi.RHO_HE)
    pos = qi.jittered_lattice(n, L, 4)
    b = 3.07
    V, TL, TPB, TF, EL = oracle.local_energy(pos, L, b)
    lp0 = oracle.log_psi(pos, L, b)
    h = 1e-4
    s = 0.0
    for i in range(n):
        for c in range(3):
            p, m = pos.copy(), pos.copy()
            p[c, i] += h
            m[c, i] -= h
            s += (math.exp(oracle.log_psi(p, L, b) - lp0) + math.exp(oracle.log_psi(m, L, b) - lp0) - 2.0) / h ** 2
    assert TL == pytest.approx(-0.5 * H2M * s, rel=1e-5)
    assert EL == pytest.approx(V + TL, rel=1e-14)
    lap, F = oracle.local_terms(pos, L, b)
    assert TPB == pytest.approx(-0.25 * H2M * lap.sum(), rel=1e-13)
    assert TF == pytest.approx(0.5 * H2M * (F ** 2).sum(), rel=1e-13)


def test_zero_kinetic_energy_without_correlation():
    n = 20
    L = qi.box_side(n, qi.RHO_HE)
    pos = qi.uniform_positions(n, L, 8)
    V, TL, TPB, TF, EL = oracle.local_energy(pos, L, 0.0)
    assert TL == 0.0 and TPB == 0.0 and TF == 0.0 and EL == V
    assert oracle.log_psi(pos, L, 0.0) == 0.0


def test_parameter_gradients_closed_forms_and_fd():
    n = 16
    L = qi.box_side(n, qi.RHO_HE)
    pos = qi.jittered_lattice(n, L, 9)
    b, m = 3.07, 5.0
    lp, EL, lpb, lpm, Eb, Em = oracle.energy_grad(pos, L, b, m)
    # u is linear in b^m: d ln psi/db = (m/b) ln psi, and the kinetic b-derivative has a closed form
    assert lpb == pytest.approx(m / b * lp, rel=1e-12)
    lap, F = oracle.local_terms(pos, L, b, m)
    assert Eb == pytest.approx(-0.5 * H2M * (m / b) * (lap.sum() + 2 * (F ** 2).sum()), rel=1e-11)
    def fd(fun, x0, h=1e-4):
        # central difference, Richardson-extrapolated from steps 2h and h (error O(h^4))
        c = lambda hh: (fun(x0 + hh) - fun(x0 - hh)) / (2 * hh)  # noqa: E731
        return (4 * c(h) - c(2 * h)) / 3

    assert lpb == pytest.approx(fd(lambda x: oracle.log_psi(pos, L, x, m), b), rel=1e-8)
    assert lpm == pytest.approx(fd(lambda x: oracle.log_psi(pos, L, b, x), m), rel=1e-8)
    assert Eb == pytest.approx(fd(lambda x: oracle.local_energy(pos, L, x, m)[4], b), rel=1e-7)
    assert Em == pytest.approx(fd(lambda x: oracle.local_energy(pos, L, b, x)[4], m), rel=1e-7)
    assert lp == pytest.approx(oracle.log_psi(pos, L, b, m), rel=1e-13)
    assert EL == pytest.approx(oracle.local_energy(pos, L, b, m)[4], rel=1e-13)


# --------------------------------------------------------------------------------------------
# Markov chain
# --------------------------------------------------------------------------------------------

def test_chain_replayed_by_full_recompute():
    """Replay the oracle chain move by move with full ln psi recomputation and the Metropolis
    rule |psi'|^2/|psi|^2 > xi (Eq. Decision) evaluated from scratch."""
    n = 8
    L = qi.box_side(n, qi.RHO_HE)
    pos0 = qi.jittered_lattice(n, L, 21)
    P = oracle.make_walker(n, L, 3.07, step=0.9, seed=0xABCDEF, wid=3)
    nsw = 6
    pos, lp, k, acc, _ = oracle.run_walker(P, pos0, oracle.log_psi(pos0, L, 3.07), 0, nsw, 0)
    cur = pos0.copy()
    accepted = 0
    for kk in range(nsw):
        for t in range(n):
            s, d, xi = oracle.move_randoms(P.seed, P.wid, 0, 0, n, t, kk, P.step)
            trial = cur.copy()
            trial[:, s] = np.mod(cur[:, s] + d, L)
            ratio = math.exp(2 * (oracle.log_psi(trial, L, 3.07) - oracle.log_psi(cur, L, 3.07)))
            if ratio > xi:
                cur = trial
                accepted += 1
    assert k == nsw and acc[7] == accepted
    assert np.allclose(pos, cur, rtol=0, atol=1e-12)
    assert lp == pytest.approx(oracle.log_psi(pos, L, 3.07), rel=1e-10)


def test_resume_is_bitwise_identical():
    n = 24
    L = qi.box_side(n, qi.RHO_HE)
    pos0 = qi.jittered_lattice(n, L, 6)
    P = oracle.make_walker(n, L, 3.07, step=0.8, seed=77, wid=1, recompute_every=3)
    a = oracle.run_walker(P, pos0, 0.0, 0, 10, 2)
    b1 = oracle.run_walker(P, pos0, 0.0, 0, 4, 2)
    b2 = oracle.run_walker(P, b1[0], b1[1], b1[2], 6, 2, accum=b1[3])
    assert np.array_equal(a[0], b2[0]) and a[1] == b2[1] and a[2] == b2[2]
    assert np.array_equal(a[3], b2[3])


@pytest.mark.parametrize("threads", [1, 3])
def test_batch_equals_walker_by_walker(threads):
    """orc_run_batch (the oracle's multi-walker driver: packed coordinates at per-walker offsets,
    OpenMP over walkers) is orc_run_walker applied to each walker, bit for bit: mixed n (so the
    offsets are uneven), both proposals, different start sweeps and sums already in accum."""
    ns = [5, 64, 17, 130]
    walkers, pos, lp, sw, acc = [], [], [], [], []
    for w, n in enumerate(ns):
        L = qi.box_side(n, qi.RHO_HE)
        walkers.append(oracle.make_walker(n, L, 3.07 - 0.02 * w, step=0.7 + 0.05 * w, proposal=w % 2,
                                          recompute_every=3, seed=0xBA7C, wid=100 + w))
        pos.append(qi.jittered_lattice(n, L, 40 + w))
        lp.append(oracle.log_psi(pos[-1], L, 3.07 - 0.02 * w))
        sw.append([0, 5, 2, 11][w])
        acc.append(np.arange(8, dtype=float) * (w + 1))
    bpos, blp, bsw, bacc, used = oracle.run_batch(walkers, pos, lp, sw, 6, 2, accum=np.array(acc), nthreads=threads)
    assert used >= 1
    for w in range(len(ns)):
        p, l, k, a, _ = oracle.run_walker(walkers[w], pos[w], lp[w], sw[w], 6, 2, accum=acc[w])
        assert np.array_equal(bpos[w], p) and blp[w] == l and int(bsw[w]) == k
        assert np.array_equal(bacc[w], a)


def test_margins_decide_acceptance():
    n = 16
    L = qi.box_side(n, qi.RHO_HE)
    pos0 = qi.jittered_lattice(n, L, 8)
    P = oracle.make_walker(n, L, 3.07, step=0.8, seed=5, wid=0)
    _, _, _, acc, mg = oracle.run_walker(P, pos0, 0.0, 0, 5, 0, margins=True)
    assert acc[7] == np.count_nonzero(mg > 0)


def test_init_walker_fcc_subset():
    n = 500
    L = qi.box_side(n, qi.RHO_HE)
    sigma = 0.1
    pos = oracle.init_walker(n, L, 0x5EED0001, 0, sigma)
    assert np.all((pos >= 0) & (pos <= L))
    nc = 5  # smallest nc with 4 nc^3 >= 500
    a = L / nc
    dmin = min(r for _, _, r in _brute_pairs(pos[:, :120], L))
    assert dmin > a / math.sqrt(2) - 12 * sigma
    # every particle sits within a few sigma of a distinct fcc site
    basis = np.array([[0, 0, 0], [.5, .5, 0], [.5, 0, .5], [0, .5, .5]])
    sites = (np.array(list(itertools.product(range(nc), repeat=3)))[:, None, :] + basis[None]).reshape(-1, 3) * a
    d = pos.T[:, None, :] - sites[None, :, :]
    d -= L * np.round(d / L)
    nearest = np.argmin((d ** 2).sum(-1), axis=1)
    assert len(set(nearest.tolist())) == n
    assert np.sqrt((d ** 2).sum(-1)).min(axis=1).max() < 6 * sigma * math.sqrt(3)
    other = oracle.init_walker(n, L, 0x5EED0001, 1, sigma)
    assert not np.array_equal(pos, other)


def test_pair_histogram_by_brute_force_images():
    n, L = 40, 9.0
    pos = qi.uniform_positions(n, L, 12)
    nbins, rmax = 30, 4.5
    got = oracle.pair_hist(pos, L, nbins, rmax)
    want = np.zeros(nbins, dtype=np.uint64)
    for _, _, r in _brute_pairs(pos, L):
        if r < rmax:
            want[min(nbins - 1, int(r * nbins / rmax))] += 1
    assert np.array_equal(got, want)
    assert got.sum() <= n * (n - 1) // 2
