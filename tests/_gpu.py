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
