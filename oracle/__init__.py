"""FP64 CPU oracle for variational Monte Carlo of liquid 4He (Lutsyshyn, "Fast quantum Monte
Carlo on a GPU").

TEST INFRASTRUCTURE ONLY.  This package is the independent checker for the CUDA library: it is
loaded by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``
and by nothing else.  It shares no code with ``paper_1312_1282_gb300`` and never imports it.
The arithmetic lives in ``qmc_oracle.c`` (plain double precision, one routine per definition of
the paper, each citing the section or equation it follows); this module only compiles it with
gcc and marshals numpy arrays through ctypes.

Parity pins (what fixes each routine independently of itself) are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Walker(C.Structure):
    """Mirror of ``orc_walker_t`` in qmc_oracle.c."""

    _fields_ = [
        ("n", C.c_int),
        ("L", C.c_double),
        ("b", C.c_double),
        ("m", C.c_double),
        ("step", C.c_double),
        ("sym", C.c_int),
        ("proposal", C.c_int),
        ("sequential", C.c_int),
        ("hbar2_over_m", C.c_double),
        ("recompute_every", C.c_int),
        ("seed", C.c_uint64),
        ("wid", C.c_uint32),
    ]


_D = C.POINTER(C.c_double)
_U32 = C.POINTER(C.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
            L.orc_aziz.argtypes = [C.c_double]
            L.orc_aziz.restype = C.c_double
            L.orc_pair_u.argtypes = [C.c_double] * 4 + [C.c_int, _D]
            L.orc_pair_u_many.argtypes = [C.c_int, _D] + [C.c_double] * 3 + [C.c_int, _D]
            geom = [C.c_int, _D, _D, _D, C.c_double, C.c_double, C.c_double, C.c_int]
            L.orc_log_psi.argtypes = geom
            L.orc_log_psi.restype = C.c_double
            L.orc_local_terms.argtypes = geom + [_D, _D, _D, _D]
            L.orc_local_energy.argtypes = geom + [C.c_double, _D]
            L.orc_energy_grad.argtypes = geom + [C.c_double, _D]
            L.orc_trial_delta.argtypes = geom + [C.c_int, C.c_double, C.c_double, C.c_double, _D]
            L.orc_trial_delta.restype = C.c_double
            L.orc_move_randoms.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_int, C.c_int, C.c_uint32,
                                           C.c_uint32, C.c_double, C.POINTER(C.c_int), _D, _D]
            L.orc_init_walker.argtypes = [C.c_int, C.c_double, C.c_uint64, C.c_uint32, C.c_double, _D, _D, _D]
            L.orc_run_walker.argtypes = [C.POINTER(Walker), _D, _D, _D, _D, C.POINTER(C.c_uint64), C.c_int,
                                         C.c_int, _D, _D]
            L.orc_run_batch.argtypes = [C.c_int, C.POINTER(Walker), C.POINTER(C.c_int64), _D, _D, _D, _D,
                                        C.POINTER(C.c_uint64), C.c_int, C.c_int, _D, C.c_int]
            L.orc_run_batch.restype = C.c_int
            L.orc_pair_hist.argtypes = [C.c_int, _D, _D, _D, C.c_double, C.c_int, C.c_double,
                                        C.POINTER(C.c_uint64)]
            L.orc_sizeof_walker.restype = C.c_int
            assert L.orc_sizeof_walker() == C.sizeof(Walker), "orc_walker_t layout mismatch"
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _xyz(pos):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    assert pos.ndim == 2 and pos.shape[0] == 3
    return pos


# ---------------------------------------------------------------------------------------------
# thin wrappers: arrays in, numbers out
# ---------------------------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def aziz(r: float) -> float:
    return lib().orc_aziz(float(r))


def pair_u(r, L, b, m=5.0, sym=1):
    """(u, u', u'', u_b, u'_b, u''_b, u_m, u'_m, u''_m) at distance r."""
    o = np.zeros(9)
    lib().orc_pair_u(float(r), float(L), float(b), float(m), int(sym), _dp(o))
    return o


def pair_u_many(r, L, b, m=5.0, sym=1):
    """pair_u at every distance of the array r: shape r.shape + (9,)."""
    rr = np.ascontiguousarray(r, dtype=np.float64).ravel()
    o = np.zeros((rr.size, 9))
    lib().orc_pair_u_many(rr.size, _dp(rr), float(L), float(b), float(m), int(sym), _dp(o))
    return o.reshape(np.shape(r) + (9,))


def log_psi(pos, L, b, m=5.0, sym=1) -> float:
    p = _xyz(pos)
    return lib().orc_log_psi(p.shape[1], _dp(p[0]), _dp(p[1]), _dp(p[2]), L, b, m, sym)


def local_terms(pos, L, b, m=5.0, sym=1):
    """Per-particle (lap_i, F_i) with F_i as an (n, 3) array."""
    p = _xyz(pos)
    n = p.shape[1]
    lap, fx, fy, fz = (np.zeros(n) for _ in range(4))
    lib().orc_local_terms(n, _dp(p[0]), _dp(p[1]), _dp(p[2]), L, b, m, sym, _dp(lap), _dp(fx), _dp(fy), _dp(fz))
    return lap, np.stack([fx, fy, fz], axis=1)


def local_energy(pos, L, b, m=5.0, sym=1, hbar2_over_m=12.1194):
    """Totals in K: (V, T_L, T_PB, T_F, E_L)."""
    p = _xyz(pos)
    o = np.zeros(5)
    lib().orc_local_energy(p.shape[1], _dp(p[0]), _dp(p[1]), _dp(p[2]), L, b, m, sym, hbar2_over_m, _dp(o))
    return o


def energy_grad(pos, L, b, m=5.0, sym=1, hbar2_over_m=12.1194):
    """(ln psi, E_L, d ln psi/db, d ln psi/dm, dE_L/db, dE_L/dm)."""
    p = _xyz(pos)
    o = np.zeros(6)
    lib().orc_energy_grad(p.shape[1], _dp(p[0]), _dp(p[1]), _dp(p[2]), L, b, m, sym, hbar2_over_m, _dp(o))
    return o


def trial_delta(pos, L, b, m, sym, s, delta):
    """(Delta, new position of particle s) for the move r_s -> wrap(r_s + delta)."""
    p = _xyz(pos)
    npos = np.zeros(3)
    d = lib().orc_trial_delta(p.shape[1], _dp(p[0]), _dp(p[1]), _dp(p[2]), L, b, m, sym, int(s),
                              float(delta[0]), float(delta[1]), float(delta[2]), _dp(npos))
    return d, npos


def pair_hist(pos, L, nbins, rmax):
    """Counts of pairs i < j with r < rmax in nbins equal bins."""
    p = _xyz(pos)
    out = np.zeros(nbins, dtype=np.uint64)
    lib().orc_pair_hist(p.shape[1], _dp(p[0]), _dp(p[1]), _dp(p[2]), L, nbins, rmax,
                        out.ctypes.data_as(C.POINTER(C.c_uint64)))
    return out


def move_randoms(seed, wid, proposal, sequential, n, t, k, step):
    s = C.c_int()
    dl = np.zeros(3)
    xi = C.c_double()
    lib().orc_move_randoms(seed, wid, proposal, sequential, n, t, k, step, C.byref(s), _dp(dl), C.byref(xi))
    return s.value, dl, xi.value


def init_walker(n, L, seed, wid, sigma):
    x, y, z = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_init_walker(n, L, seed, wid, sigma, _dp(x), _dp(y), _dp(z))
    return np.stack([x, y, z])


def make_walker(n, L, b, m=5.0, step=0.8, sym=1, proposal=0, sequential=0, hbar2_over_m=12.1194,
                recompute_every=0, seed=0, wid=0) -> Walker:
    return Walker(n, L, b, m, step, sym, proposal, sequential, hbar2_over_m, recompute_every, seed, wid)


def run_walker(P: Walker, pos, logpsi, sweep, nsweeps, energy_every, accum=None, margins=False):
    """Advance one walker in place.  Returns (pos, logpsi, sweep, accum[8], margins or None)."""
    p = _xyz(pos).copy()
    lp = np.array([float(logpsi)])
    sw = (C.c_uint64 * 1)(int(sweep))
    acc = np.zeros(8) if accum is None else np.array(accum, dtype=np.float64)
    mg = np.zeros(P.n * nsweeps) if margins else None
    lib().orc_run_walker(C.byref(P), _dp(p[0]), _dp(p[1]), _dp(p[2]), _dp(lp), sw, nsweeps, energy_every,
                         _dp(acc), _dp(mg) if margins else None)
    return p, float(lp[0]), int(sw[0]), acc, mg


def run_batch(walkers, pos_list, logpsi, sweeps, nsweeps, energy_every, accum=None, nthreads=0):
    """Advance W walkers (OpenMP over walkers).  pos_list: list of (3, n_w) arrays.
    Returns (pos_list, logpsi[W], sweeps[W], accum[W, 8], threads used)."""
    W = len(walkers)
    arr = (Walker * W)(*walkers)
    ns = [int(w.n) for w in walkers]
    off = np.zeros(W, dtype=np.int64)
    off[1:] = np.cumsum(ns)[:-1]
    tot = int(sum(ns))
    x, y, z = np.zeros(tot), np.zeros(tot), np.zeros(tot)
    for w, p in enumerate(pos_list):
        p = _xyz(p)
        x[off[w]:off[w] + ns[w]] = p[0]
        y[off[w]:off[w] + ns[w]] = p[1]
        z[off[w]:off[w] + ns[w]] = p[2]
    lp = np.array(logpsi, dtype=np.float64).copy()
    sw = (C.c_uint64 * W)(*[int(s) for s in sweeps])
    acc = np.zeros((W, 8)) if accum is None else np.array(accum, dtype=np.float64).reshape(W, 8).copy()
    used = lib().orc_run_batch(W, arr, off.ctypes.data_as(C.POINTER(C.c_int64)), _dp(x), _dp(y), _dp(z),
                               _dp(lp), sw, nsweeps, energy_every, _dp(acc), int(nthreads))
    out = [np.stack([x[off[w]:off[w] + ns[w]], y[off[w]:off[w] + ns[w]], z[off[w]:off[w] + ns[w]]])
           for w in range(W)]
    return out, lp, np.array([int(s) for s in sw], dtype=np.uint64), acc, used
