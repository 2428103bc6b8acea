"""Statistical pins of the oracle's Markov chain (CPU only).

The chain is checked against exact expectation values that do not come from the chain:
for two particles the sampled density |psi|^2 = exp(2 u(r)) (Eqs. Probability and Jastrow)
reduces the averages to one-dimensional integrals over the minimum-image cube; with b = 0 the
chain must accept every move and the kinetic energy must vanish; and the three kinetic
estimators must agree in expectation (an identity from integration by parts that holds for
the symmetrised u, which is continuous with its first derivative at L/2).
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
import qmc_inputs as qi

H2M = qi.HBAR2_OVER_M


def _blocks(P, pos, nblocks, per_block, energy_every=1, seed_sweep=0):
    """Run nblocks blocks and return per-block means of (E_L, V, T_L, T_PB, T_F) and the
    accepted fraction of all moves."""
    lp = oracle.log_psi(pos, P.L, P.b, P.m, P.sym)
    k = seed_sweep
    means, acc_total = [], 0.0
    for _ in range(nblocks):
        pos, lp, k, acc, _ = oracle.run_walker(P, pos, lp, k, per_block, energy_every)
        if acc[6] > 0:
            ns = acc[6]
            means.append([acc[0] / ns, acc[2] / ns, acc[3] / ns, acc[4] / ns, acc[5] / ns])
        acc_total += acc[7]
    return np.array(means), acc_total / (nblocks * per_block * P.n), pos


def _two_body_exact(L, b):
    """Exact <V>, <T_L>, <T_PB>, <T_F> for N = 2 at |psi|^2 = exp(2 u(r)) on the minimum-image
    cube of side L, where u and V vanish in the corners r > L/2."""
    h = L / 2
    w = lambda r: 4 * math.pi * r * r * math.exp(2 * oracle.pair_u(r, L, b)[0])  # noqa: E731
    Z = quad(w, 0, h, limit=200, points=[2.0, 3.0])[0] + (L ** 3 - 4 * math.pi / 3 * h ** 3)

    def avg(g):
        return quad(lambda r: w(r) * g(r), 1e-3, h, limit=400, points=[2.0, 3.0])[0] / Z

    lap = lambda r: oracle.pair_u(r, L, b)[2] + 2 * oracle.pair_u(r, L, b)[1] / r  # noqa: E731
    du2 = lambda r: oracle.pair_u(r, L, b)[1] ** 2  # noqa: E731
    V = avg(oracle.aziz)
    TPB = -0.25 * H2M * 2 * avg(lap)
    TF = 0.5 * H2M * 2 * avg(du2)
    TL = -0.5 * H2M * (2 * avg(lap) + 2 * avg(du2))
    return V, TL, TPB, TF


def test_two_particles_match_exact_integrals():
    L, b = 8.0, 3.07
    V, TL, TPB, TF = _two_body_exact(L, b)
    P = oracle.make_walker(2, L, b, step=2.0, seed=0xC0FFEE, wid=0)
    pos = np.array([[1.0, 5.0], [1.0, 5.0], [1.0, 5.0]])
    m, acc, _ = _blocks(P, pos, 200, 1000)
    mu, sd = m.mean(0), m.std(0, ddof=1) / math.sqrt(len(m))
    for got, err, want in zip(mu[1:], sd[1:], (V, TL, TPB, TF)):
        assert abs(got - want) < 4.5 * err + 1e-9, (got, err, want)
    assert 0.05 < acc < 0.95


def test_two_particle_distance_density_matches_exact():
    """The sampled minimum-image pair distance of N = 2 has density 4 pi r^2 exp(2 u(r)) / Z below
    L/2, and the corners of the cube (u = 0) take the rest: 16 bins of 0.25 A plus the corners,
    frequencies over 40 blocks of thinned samples, every bin within 5 standard errors and a
    chi^2 with the block variances within its spread."""
    L, b = 8.0, 3.07
    h = L / 2
    nb = 16
    w = lambda r: 4 * math.pi * r * r * math.exp(2 * oracle.pair_u(r, L, b)[0])  # noqa: E731
    corners = L ** 3 - 4 * math.pi / 3 * h ** 3
    edges = np.linspace(0.0, h, nb + 1)
    inner = [quad(w, edges[i], edges[i + 1], limit=200)[0] for i in range(nb)]
    Z = sum(inner) + corners
    want = np.array(inner + [corners]) / Z
    assert abs(want.sum() - 1.0) < 1e-12

    P = oracle.make_walker(2, L, b, step=2.0, seed=0xD15, wid=0)
    pos = np.array([[1.0, 5.0], [1.0, 5.0], [1.0, 5.0]])
    lp = oracle.log_psi(pos, L, b)
    pos, lp, k, _, _ = oracle.run_walker(P, pos, lp, 0, 100, 0)  # burn-in
    nblocks, per_block = 40, 500
    frac = np.zeros((nblocks, nb + 1))
    for blk in range(nblocks):
        for _ in range(per_block):
            pos, lp, k, _, _ = oracle.run_walker(P, pos, lp, k, 2, 0)
            d = pos[:, 0] - pos[:, 1]
            d -= L * np.round(d / L)
            r = math.sqrt(float(d @ d))
            frac[blk, min(int(r / h * nb), nb) if r < h else nb] += 1.0 / per_block
    mean = frac.mean(0)
    se = frac.std(0, ddof=1) / math.sqrt(nblocks)
    assert np.all(np.abs(mean - want) < 5 * se + 5e-4), np.c_[mean, want, se]
    live = se > 0
    chi2 = float((((mean - want) / np.where(live, se, 1.0)) ** 2)[live].sum())
    dof = int(live.sum())
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)
    # the contact region is excluded: no sample below 2 A (exp(2u) < 1e-3 there)
    assert mean[:8].sum() < 1e-3


def test_no_correlation_limit_accepts_every_move():
    L = 8.0
    P = oracle.make_walker(2, L, 0.0, step=2.0, seed=3, wid=0)
    pos = np.array([[1.0, 5.0], [1.0, 5.0], [1.0, 5.0]])
    m, acc, _ = _blocks(P, pos, 100, 1000)
    assert acc == 1.0
    assert np.all(m[:, 2:] == 0.0)
    # uniform pair density: <V> = int_0^{L/2} 4 pi r^2 V(r) dr / L^3
    want = quad(lambda r: 4 * math.pi * r * r * oracle.aziz(r), 1e-6, L / 2, limit=400, points=[2.0, 3.0])[0] / L ** 3
    got, err = m[:, 1].mean(), m[:, 1].std(ddof=1) / math.sqrt(len(m))
    assert abs(got - want) < 4.5 * err


def test_kinetic_estimators_agree():
    n = 64
    L = qi.box_side(n, qi.RHO_HE)
    P = oracle.make_walker(n, L, 3.07, step=0.8, seed=0x5EED0001, wid=0)
    pos = oracle.init_walker(n, L, 0x5EED0001, 0, 0.1)
    _, _, pos = _blocks(P, pos, 1, 300, energy_every=0)
    m, acc, _ = _blocks(P, pos, 40, 50, seed_sweep=300)
    d1 = m[:, 2] - m[:, 3]   # T_L - T_PB
    d2 = m[:, 4] - m[:, 3]   # T_F - T_PB
    for d in (d1, d2):
        assert abs(d.mean()) < 4.5 * d.std(ddof=1) / math.sqrt(len(d))
    assert 0.2 < acc < 0.9


@pytest.mark.slow
def test_paper_sample_run_energy():
    """Sec. 5.4 sample run: N = 1000 at 0.02186 A^-3, 16 walkers; E/N about -5.80 K.
    Gaussian displacements with RMS 0.5 rho^(-1/3) of the displacement vector (Sec. 7)."""
    gold = os.path.join(os.path.dirname(__file__), "golden", "paper_sample_run.txt")
    rows = np.array([[float(v) for v in ln.split()] for ln in open(gold) if ln.strip() and ln[0] != "#"])
    e_ref = rows[:, 1].mean()
    n, W = 1000, 16
    L = qi.box_side(n, qi.RHO_HE)
    sigma = 0.5 * qi.RHO_HE ** (-1 / 3) / math.sqrt(3)
    walkers = [oracle.make_walker(n, L, qi.B_HE, step=sigma, proposal=1, seed=0x5A3, wid=w) for w in range(W)]
    pos = [oracle.init_walker(n, L, 0x5A3, w, 0.1) for w in range(W)]
    lp = [oracle.log_psi(p, L, qi.B_HE) for p in pos]
    pos, lp, sw, _, _ = oracle.run_batch(walkers, pos, lp, [0] * W, 150, 0)
    pos, lp, sw, acc, _ = oracle.run_batch(walkers, pos, lp, sw, 200, 4)
    e = acc[:, 0] / acc[:, 6] / n
    mu, err = e.mean(), e.std(ddof=1) / math.sqrt(W)
    assert abs(mu - e_ref) < 3 * err + 0.03, (mu, err, e_ref)
