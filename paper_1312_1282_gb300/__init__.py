"""Python binding of libqmc: variational Monte Carlo of liquid 4He on one GB300 GPU.

The functions named ``qmc_*`` marshal arguments to the C ABI of ``include/qmc.h`` one to one:
device buffers are torch CUDA tensors (positions float32/float64, outputs float64, sweep
counters int64), streams are torch streams.  Every step of the method runs in the CUDA
kernels of ``csrc/``; nothing here computes physics, and there is no CPU fallback: importing
this package without the compiled library raises.

``Batch`` bundles a walker batch with its device state (positions, ln psi, sweep counters,
accumulators) for convenience; ``QmcGrad`` exposes ``qmc_energy_grad`` to torch autograd.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

__all__ = [
    "QMC_FP32", "QMC_FP64", "QMC_CUBE", "QMC_GAUSS", "QmcError", "WalkerDesc", "Options", "lib", "descs",
    "options", "qmc_init_walkers", "qmc_sweep", "qmc_local_energy", "qmc_energy_grad", "qmc_log_psi",
    "qmc_trial_delta", "qmc_pair_hist", "pair_correlation", "qmc_sweep_static", "QMC_STATIC_MAX_WALKERS", "qmc_autotune",
    "qmc_probe_rates", "PROBE_FIELDS", "qmc_capacity", "qmc_status", "qmc_launch_count", "qmc_version",
    "qmc_shutdown", "Batch", "QmcGrad", "ACCUM_FIELDS", "NACC", "ENERGY_FIELDS", "GRAD_FIELDS",
]

QMC_FP32, QMC_FP64 = 0, 1
QMC_CUBE, QMC_GAUSS = 0, 1
QMC_STATIC_MAX_WALKERS = 4096
ACCUM_FIELDS = ("sum_EL", "sum_EL2", "sum_V", "sum_TL", "sum_TPB", "sum_TF", "samples", "accepted",
                "sum_logpsi_drift", "max_logpsi_drift")
NACC = len(ACCUM_FIELDS)  # QMC_ACCUM_FIELDS: doubles per walker in the accumulator record
ENERGY_FIELDS = ("V", "T_L", "T_PB", "T_F", "E_L")
GRAD_FIELDS = ("logpsi", "E_L", "dlogpsi_db", "dlogpsi_dm", "dEL_db", "dEL_dm")
_ERRORS = {-1: "QMC_ERR_ARG", -2: "QMC_ERR_CAPACITY", -3: "QMC_ERR_CUDA", -4: "QMC_ERR_DEVICE", -5: "QMC_ERR_TIMEOUT"}


class QmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class WalkerDesc(C.Structure):
    """qmc_walker_desc (64 bytes)."""

    _fields_ = [("n", C.c_int32), ("pad_n", C.c_int32), ("offset", C.c_int64), ("id", C.c_int64),
                ("L", C.c_double), ("rho", C.c_double), ("b", C.c_double), ("m_exp", C.c_double),
                ("step", C.c_double)]


class Options(C.Structure):
    """qmc_options (40 bytes)."""

    _fields_ = [("precision", C.c_int32), ("proposal", C.c_int32), ("sym", C.c_int32), ("sequential", C.c_int32),
                ("hbar2_over_m", C.c_double), ("recompute_every", C.c_int32), ("threads_per_walker", C.c_int32),
                ("walkers_per_cta", C.c_int32), ("reserved", C.c_int32)]


assert C.sizeof(WalkerDesc) == 64 and C.sizeof(Options) == 40

_lib = None
_VP, _DP = C.c_void_p, C.POINTER(C.c_double)


def lib():
    """The loaded libqmc.so (in-tree build); raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libqmc.so is not built ({_build.LIB}); run __graft_entry__.build() "
                               "or python -m paper_1312_1282_gb300.build")
        L = C.CDLL(_build.LIB)
        D, O = C.POINTER(WalkerDesc), C.POINTER(Options)
        L.qmc_init_walkers.argtypes = [D, C.c_int, C.c_uint64, C.c_double, O, _VP, _VP]
        L.qmc_sweep.argtypes = [D, C.c_int, O, _VP, _VP, _VP, C.c_uint64, C.c_int, C.c_int, _VP, _VP]
        L.qmc_local_energy.argtypes = [D, C.c_int, O, _VP, _VP, _VP]
        L.qmc_energy_grad.argtypes = [D, C.c_int, O, _VP, _VP, _VP]
        L.qmc_log_psi.argtypes = [D, C.c_int, O, _VP, _VP, _VP]
        L.qmc_trial_delta.argtypes = [D, C.c_int, O, _VP, _VP, _VP, C.c_int, _VP, _VP]
        L.qmc_autotune.argtypes = [D, C.c_int, O, _VP, _VP, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.qmc_pair_hist.argtypes = [D, C.c_int, O, _VP, C.c_int, C.c_double, _VP, _VP]
        L.qmc_sweep_static.argtypes = [D, C.c_int, O, _VP, _VP, _VP, C.c_uint64, C.c_int, C.c_int, _VP, _VP, _VP]
        L.qmc_capacity.argtypes = [C.c_int]
        L.qmc_probe_rates.argtypes = [C.c_int, C.c_int, C.c_int, _DP, _VP]
        L.qmc_status.argtypes = [_VP, C.c_int, C.POINTER(C.c_uint32)]
        L.qmc_launch_count.restype = C.c_uint64
        L.qmc_last_error.restype = C.c_char_p
        L.qmc_shutdown.restype = None
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise QmcError(rc, lib().qmc_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("device buffers must be CUDA tensors")
        if not t.is_contiguous():
            raise ValueError("device buffers must be contiguous")
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(int(t))


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def descs(rows) -> C.Array:
    """Build a qmc_walker_desc array from dicts or tuples (n, pad_n, offset, id, L, rho, b, m_exp, step)."""
    rows = list(rows)
    arr = (WalkerDesc * len(rows))()
    for i, r in enumerate(rows):
        if isinstance(r, dict):
            for k, v in r.items():
                setattr(arr[i], k, v)
        else:
            arr[i] = WalkerDesc(*r)
    return arr


def options(precision=QMC_FP32, proposal=QMC_CUBE, sym=1, sequential=0, hbar2_over_m=12.1194, recompute_every=50,
            threads_per_walker=0, walkers_per_cta=0) -> Options:
    return Options(precision, proposal, sym, sequential, hbar2_over_m, recompute_every, threads_per_walker,
                   walkers_per_cta, 0)


# ---------------------------------------------------------------------------------------------
# one-to-one wrappers of the C ABI
# ---------------------------------------------------------------------------------------------
_NVTX = os.environ.get("QMC_NVTX") == "1"


def _traced(fn):
    """With QMC_NVTX=1 in the environment, each call is an NVTX range named after the C entry
    point (visible to Nsight tools; a no-op otherwise)."""
    if not _NVTX:
        return fn
    import functools

    @functools.wraps(fn)
    def wrapper(*args, **kwargs):
        torch.cuda.nvtx.range_push(fn.__name__)
        try:
            return fn(*args, **kwargs)
        finally:
            torch.cuda.nvtx.range_pop()

    return wrapper


@_traced
def qmc_init_walkers(d, seed, jitter_sigma, opt, pos, stream=None):
    return _check(lib().qmc_init_walkers(d, len(d), seed, jitter_sigma, C.byref(opt), _ptr(pos), _stream(stream)))


@_traced
def qmc_sweep(d, opt, pos, logpsi, sweep, seed, nsweeps, energy_every, accum, stream=None):
    return _check(lib().qmc_sweep(d, len(d), C.byref(opt), _ptr(pos), _ptr(logpsi), _ptr(sweep), seed, nsweeps,
                                  energy_every, _ptr(accum), _stream(stream)))


@_traced
def qmc_sweep_static(d, opt, pos, logpsi, sweep, seed, nsweeps, energy_every, accum, err=None, stream=None):
    """qmc_sweep without any device allocation by the library (fixed scratch array; at most
    QMC_STATIC_MAX_WALKERS walkers; calls overlapping on the GPU must not be issued)."""
    return _check(lib().qmc_sweep_static(d, len(d), C.byref(opt), _ptr(pos), _ptr(logpsi), _ptr(sweep), seed,
                                         nsweeps, energy_every, _ptr(accum), _ptr(err), _stream(stream)))


@_traced
def qmc_local_energy(d, opt, pos, out, stream=None):
    return _check(lib().qmc_local_energy(d, len(d), C.byref(opt), _ptr(pos), _ptr(out), _stream(stream)))


@_traced
def qmc_energy_grad(d, opt, pos, out, stream=None):
    return _check(lib().qmc_energy_grad(d, len(d), C.byref(opt), _ptr(pos), _ptr(out), _stream(stream)))


@_traced
def qmc_log_psi(d, opt, pos, out, stream=None):
    return _check(lib().qmc_log_psi(d, len(d), C.byref(opt), _ptr(pos), _ptr(out), _stream(stream)))


@_traced
def qmc_trial_delta(d, opt, pos, s, delta, M, out, stream=None):
    return _check(lib().qmc_trial_delta(d, len(d), C.byref(opt), _ptr(pos), _ptr(s), _ptr(delta), M, _ptr(out),
                                        _stream(stream)))


@_traced
def qmc_pair_hist(d, opt, pos, nbins, rmax, hist, stream=None):
    return _check(lib().qmc_pair_hist(d, len(d), C.byref(opt), _ptr(pos), nbins, rmax, _ptr(hist), _stream(stream)))


def pair_correlation(counts, n, L, rmax, samples):
    """g(r) from summed pair counts (qmc_pair_hist) of `samples` configurations of n atoms in a
    cube of side L: counts over the ideal-gas expectation of each spherical shell."""
    counts = np.asarray(counts, dtype=np.float64)
    nb = counts.shape[-1]
    edges = np.linspace(0.0, rmax, nb + 1)
    shell = 4.0 * np.pi / 3.0 * (edges[1:] ** 3 - edges[:-1] ** 3) / L ** 3
    return 0.5 * (edges[1:] + edges[:-1]), counts / (samples * n * (n - 1) / 2.0 * shell)


@_traced
def qmc_autotune(d, opt, pos, stream=None) -> tuple[int, int]:
    """The measured launch shape of qmc_sweep for this batch: (threads per walker, walkers per CTA)."""
    t, g = C.c_int(0), C.c_int(0)
    _check(lib().qmc_autotune(d, len(d), C.byref(opt), _ptr(pos), _stream(stream), C.byref(t), C.byref(g)))
    return t.value, g.value


PROBE_FIELDS = ("ffma", "ffma2", "fmnmx", "rsqrt", "dfma", "pair_evals")


def qmc_probe_rates(blocks_per_sm=4, threads=256, iters=2000, stream=None) -> dict:
    """Measured rates per second per SM on the current GPU (include/qmc_probe.h): lane operations
    of FP32 FMA (scalar, packed), FP32 min, SFU rsqrt, FP64 FMA, and pair evaluations of the
    sweep's partner arithmetic alone."""
    out = (C.c_double * len(PROBE_FIELDS))()
    _check(lib().qmc_probe_rates(blocks_per_sm, threads, iters, out, _stream(stream)))
    return dict(zip(PROBE_FIELDS, list(out)))


def qmc_capacity(precision) -> int:
    r = lib().qmc_capacity(precision)
    if r < 0:
        _check(r)
    return r


def qmc_status(stream=None, timeout_ms=0):
    bits = C.c_uint32(0)
    rc = lib().qmc_status(_stream(stream), timeout_ms, C.byref(bits))
    _check(rc)
    return bits.value


def qmc_launch_count() -> int:
    return int(lib().qmc_launch_count())


def qmc_version() -> int:
    return int(lib().qmc_version())


def qmc_shutdown():
    lib().qmc_shutdown()


# ---------------------------------------------------------------------------------------------
# convenience: a batch of walkers with its device state
# ---------------------------------------------------------------------------------------------

class Batch:
    """W walkers with positions, ln psi, sweep counters and accumulators on the current GPU.

    walkers: list of (n, L, b) or (n, L, b, m, step) tuples; ids are id0 + index.
    """

    def __init__(self, walkers, precision=QMC_FP32, step=0.8, m=5.0, id0=0, device=None, **opt_kw):
        self.device = torch.device(device or "cuda")
        rows, off = [], 0
        for w, spec in enumerate(walkers):
            n, L, b = int(spec[0]), float(spec[1]), float(spec[2])
            mm = float(spec[3]) if len(spec) > 3 else m
            st = float(spec[4]) if len(spec) > 4 else step
            pad = (n + 3) // 4 * 4
            rows.append((n, pad, off, id0 + w, L, 0.0, b, mm, st))
            off += 3 * pad
        self.d = descs(rows)
        self.W = len(rows)
        self.opt = options(precision=precision, **opt_kw)
        dt = torch.float64 if precision == QMC_FP64 else torch.float32
        self.pos = torch.zeros(off, dtype=dt, device=self.device)
        self.logpsi = torch.zeros(self.W, dtype=torch.float64, device=self.device)
        self.sweeps = torch.zeros(self.W, dtype=torch.int64, device=self.device)
        self.accum = torch.zeros(self.W, NACC, dtype=torch.float64, device=self.device)
        self.seed = 0

    @property
    def n(self):
        return np.array([r.n for r in self.d])

    def init(self, seed, jitter_sigma=0.1, stream=None):
        self.seed = int(seed)
        qmc_init_walkers(self.d, self.seed, jitter_sigma, self.opt, self.pos, stream)
        qmc_log_psi(self.d, self.opt, self.pos, self.logpsi, stream)
        return self

    def sweep(self, nsweeps, energy_every=0, stream=None):
        qmc_sweep(self.d, self.opt, self.pos, self.logpsi, self.sweeps, self.seed, nsweeps, energy_every,
                  self.accum, stream)
        return self

    def local_energy(self, stream=None):
        out = torch.empty(self.W, 5, dtype=torch.float64, device=self.device)
        qmc_local_energy(self.d, self.opt, self.pos, out, stream)
        return out

    def log_psi(self, stream=None):
        out = torch.empty(self.W, dtype=torch.float64, device=self.device)
        qmc_log_psi(self.d, self.opt, self.pos, out, stream)
        return out

    def energy_grad(self, stream=None):
        out = torch.empty(self.W, 6, dtype=torch.float64, device=self.device)
        qmc_energy_grad(self.d, self.opt, self.pos, out, stream)
        return out

    def autotune(self, stream=None):
        return qmc_autotune(self.d, self.opt, self.pos, stream)

    def walker_positions(self, w):
        """(3, n) view of walker w's coordinates."""
        r = self.d[w]
        return self.pos[r.offset:r.offset + 3 * r.pad_n].view(3, r.pad_n)[:, :r.n]

    def set_params(self, b=None, m=None):
        for r in self.d:
            if b is not None:
                r.b = float(b)
            if m is not None:
                r.m_exp = float(m)


class QmcGrad(torch.autograd.Function):
    """(ln psi, E_L) per walker as differentiable functions of the Jastrow parameters (b, m).

    forward(batch, b, m) sets every walker's (b, m), calls qmc_energy_grad and returns two [W]
    tensors; backward contracts the incoming gradients with the per-walker derivatives.
    Positions are held fixed (their gradient is not provided)."""

    @staticmethod
    def forward(ctx, batch, b, m):
        batch.set_params(float(b), float(m))
        out = batch.energy_grad()
        ctx.save_for_backward(out)
        return out[:, 0].clone(), out[:, 1].clone()

    @staticmethod
    def backward(ctx, g_lp, g_el):
        (out,) = ctx.saved_tensors
        gb = (g_lp * out[:, 2]).sum() + (g_el * out[:, 4]).sum()
        gm = (g_lp * out[:, 3]).sum() + (g_el * out[:, 5]).sum()
        return None, gb.to(torch.float64), gm.to(torch.float64)


def vmc_energy_gradient(EL: torch.Tensor, dlogpsi: torch.Tensor, dEL: torch.Tensor | None = None) -> torch.Tensor:
    """VMC estimator of d<E>/da = 2(<E_L O_a> - <E_L><O_a>) + <dE_L/da>, O_a = d ln psi/da,
    from per-sample tensors (the last term has zero expectation and reduces variance only)."""
    g = 2.0 * ((EL * dlogpsi).mean() - EL.mean() * dlogpsi.mean())
    if dEL is not None:
        g = g + dEL.mean()
    return g
