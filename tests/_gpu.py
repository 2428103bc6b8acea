"""Helpers of the GPU tests: pack seeded configurations into the library's SoA layout and
compare with the oracle.  Positions are rounded to the working precision first, so that the
CUDA path and the oracle see the same numbers."""
from __future__ import annotations

import numpy as np
import torch

import paper_1312_1282_gb300 as q
import qmc_inputs as qi

H2M = qi.HBAR2_OVER_M


class Packed:
    def __init__(self, confs, Ls, bs, precision, ms=5.0, steps=0.8, ids=None, junk=123.0):
        W = len(confs)
        ms = np.broadcast_to(np.asarray(ms, dtype=float), (W,))
        steps = np.broadcast_to(np.asarray(steps, dtype=float), (W,))
        ids = list(range(W)) if ids is None else list(ids)
        dt = np.float64 if precision == q.QMC_FP64 else np.float32
        rows, off, blocks = [], 0, []
        self.confs = []
        for w, p in enumerate(confs):
            n = p.shape[1]
            pad = qi.pad4(n)
            rows.append((n, pad, off, ids[w], float(Ls[w]), 0.0, float(bs[w]), float(ms[w]), float(steps[w])))
            blk = np.full((3, pad), junk, dtype=dt)
            blk[:, :n] = p.astype(dt)
            blocks.append(blk.reshape(-1))
            self.confs.append(blk[:, :n].astype(np.float64))  # what the GPU sees, exactly
            off += 3 * pad
        self.d = q.descs(rows)
        self.W = W
        self.precision = precision
        self.dt = torch.float64 if precision == q.QMC_FP64 else torch.float32
        self.host = np.concatenate(blocks)
        self.pos = torch.tensor(self.host, device="cuda")
        self.Ls = [float(x) for x in Ls]
        self.bs = [float(x) for x in bs]
        self.ms = [float(x) for x in ms]
        self.steps = [float(x) for x in steps]
        self.ids = ids

    def positions(self, w, pos=None):
        r = self.d[w]
        src = (self.pos if pos is None else pos).detach().cpu().numpy().astype(np.float64)
        return src[r.offset:r.offset + 3 * r.pad_n].reshape(3, r.pad_n)[:, :r.n]

    def padding(self, w):
        r = self.d[w]
        src = self.pos.detach().cpu().numpy()
        return src[r.offset:r.offset + 3 * r.pad_n].reshape(3, r.pad_n)[:, r.n:]


def lattice_batch(ns, precision, seed=0, rho=qi.RHO_HE, bs=None, **kw):
    confs, Ls = [], []
    for i, n in enumerate(ns):
        L = qi.box_side(n, rho)
        confs.append(qi.jittered_lattice(n, L, seed + i))
        Ls.append(L)
    bs = [qi.B_HE] * len(ns) if bs is None else bs
    return Packed(confs, Ls, bs, precision, **kw)


def zeros(shape, dtype=torch.float64):
    return torch.zeros(shape, dtype=dtype, device="cuda")


def energy_scale(e):
    """Scale of each local-energy output for a relative comparison: its own magnitude for V,
    T_PB and T_F; for T_L = -(hbar^2/2m)(sum lap + sum |F|^2) the magnitudes of the two sums it
    cancels (2|T_PB| + |T_F|); for E_L = V + T_L those plus |V|."""
    e = np.asarray(e, dtype=float)
    s = np.abs(e).copy()
    s[1] = 2 * abs(e[2]) + abs(e[3])
    s[4] = abs(e[0]) + s[1]
    return np.maximum(s, 1e-12)


# ---------------------------------------------------------------------------------------------
# achieved errors, tolerance scales from the oracle's pair terms, per-sweep FP32 chain checks
# ---------------------------------------------------------------------------------------------
def report(test, **values):
    """Append the achieved errors of a parity check to the file named by QMC_PARITY_REPORT (one
    JSON object per line), so that the margin under each tolerance can be read off a run."""
    import json
    import os
    path = os.environ.get("QMC_PARITY_REPORT")
    if path:
        with open(path, "a") as fh:
            row = {k: (v if isinstance(v, str) else float(v) if np.ndim(v) == 0 else np.asarray(v).tolist())
                   for k, v in values.items()}
            fh.write(json.dumps({"test": test, **row}) + "\n")


def _row_distances(conf, L, i):
    """Minimum-image distances from atom i to every atom (numpy; geometry only)."""
    d = conf - conf[:, i:i + 1]
    d -= L * np.rint(d / L)
    return np.sqrt((d ** 2).sum(axis=0))


def oracle_pair_terms(r, L, b, m, sym):
    """oracle.pair_u at each distance: columns (u, u', u'', u_b, u'_b, u''_b, u_m, u'_m, u''_m)."""
    import oracle
    return oracle.pair_u_many(r, L, b, m, sym)


def trial_scale(conf, L, b, m, sym, s, new):
    """Scale of the FP32 error of one trial ratio (Eq. JastrowUpdate): the sum over partners j of
    |u| + |u'| at the old and at the new distance.  An error of relative size e in every pair term
    and of e L in the coordinates gives an error of at most about e times this."""
    n = conf.shape[1]
    keep = np.arange(n) != s
    out = 0.0
    for p in (conf[:, s], np.asarray(new, dtype=float)):
        d = conf[:, keep] - p[:, None]
        d -= L * np.rint(d / L)
        r = np.sqrt((d ** 2).sum(axis=0))
        t = oracle_pair_terms(r[r < 0.5 * L], L, b, m, sym)
        out += np.abs(t[:, 0]).sum() + np.abs(t[:, 1]).sum()
    return out


def grad_scales(conf, L, b, m, sym, h2m, rows=None):
    """Scales of the FP32 errors of the six qmc_energy_grad outputs, each the sum of the
    magnitudes of the pair terms it is built from (so a cancellation in the result does not
    shrink its scale): |ln psi|, the local-energy scale, |d ln psi/db|, sum_{i<j} |u_m|,
    k (m/b) [sum_i sum_j |u'' + 2u'/r| + 2 sum_i |F_i|^2], and
    k [sum_i sum_j |u''_m + 2u'_m/r| + 2 sum_i |F_i| sum_j |u'_m|], with k = hbar^2/2m.
    The row sums over i are exact over all atoms, or, with `rows` (a number), N/rows times their
    sum over that many evenly spaced atoms (large N; the rows of a liquid are alike)."""
    import oracle
    n = conf.shape[1]
    pick = np.arange(n) if rows is None else np.linspace(0, n - 1, rows).astype(int)
    _, F = oracle.local_terms(conf, L, b, m, sym)
    Fn = np.sqrt((F ** 2).sum(axis=1))
    s_um = s_lap = s_lapm = s_fg = 0.0
    for i in pick:
        r = _row_distances(conf, L, i)
        r = r[(np.arange(n) != i) & (r < 0.5 * L)]
        t = oracle_pair_terms(r, L, b, m, sym)
        s_um += np.abs(t[:, 6]).sum()
        s_lap += np.abs(t[:, 2] + 2 * t[:, 1] / r).sum()
        s_lapm += np.abs(t[:, 8] + 2 * t[:, 7] / r).sum()
        s_fg += Fn[i] * np.abs(t[:, 7]).sum()
    f = n / len(pick)
    k = 0.5 * h2m
    lp = oracle.log_psi(conf, L, b, m, sym)
    e = oracle.local_energy(conf, L, b, m, sym, h2m)
    return np.array([abs(lp), energy_scale(e)[4], abs(m / b * lp), 0.5 * f * s_um,
                     k * m / b * (f * s_lap + 2 * (Fn ** 2).sum()), k * (f * s_lapm + 2 * f * s_fg)])


def near_tie(n):
    """Largest |2 Delta - ln xi| (oracle, FP64) at which an FP32 decision may legitimately differ:
    the FP32 error of Delta (pair terms from SFU approximations, about 1e-6 relative, summed over
    n partners) plus that of ln xi (24-bit uniforms)."""
    return 1e-4 if n <= 256 else 1e-3


def fp32_sweeps_vs_oracle(states, accepted, n, L, b, m, step, seed, wid, k0=0, sym=1, proposal=0, sequential=0):
    """Localised FP32 chain parity.  states[k] is the GPU configuration (3, n) before sweep k0 + k
    (k = 0 .. S), accepted[k] the moves the GPU accepted in that sweep.  The oracle reruns every
    sweep from the GPU's own state; a sweep whose result differs must contain a near tie
    (near_tie(n)).  Returns the number of sweeps that agree and the list of (sweep, smallest
    |margin|) of those that do not."""
    import oracle
    P = oracle.make_walker(n, L, b, m, step, sym=sym, proposal=proposal, sequential=sequential, hbar2_over_m=H2M,
                           seed=seed, wid=wid)
    agree, differ = 0, []
    for k in range(len(states) - 1):
        opos, _, _, oacc, mg = oracle.run_walker(P, states[k], 0.0, k0 + k, 1, 0, margins=True)
        if oacc[7] == accepted[k] and np.abs(states[k + 1] - opos).max() < 1e-3:
            agree += 1
        else:
            smallest = float(np.abs(mg).min())
            assert smallest < near_tie(n), (wid, k0 + k, smallest)
            differ.append((k0 + k, smallest))
    return agree, differ
