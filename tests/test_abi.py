"""The C-ABI library builds for sm_103a, loads, and exports what include/qmc.h declares
(CPU only: no compute call is made here)."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

import paper_1312_1282_gb300 as q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qmc.h")
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def _declared():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(qmc_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_builds_and_loads():
    q._build.build()
    assert os.path.exists(q._build.LIB)
    assert q.qmc_version() == 110


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert {"qmc_init_walkers", "qmc_sweep", "qmc_local_energy", "qmc_energy_grad", "qmc_probe_rates"} <= set(names)
    lib = C.CDLL(q._build.LIB)
    for nm in names:
        assert hasattr(lib, nm), nm
    out = subprocess.run(["nm", "-D", "--defined-only", q._build.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(names) <= exported


def test_struct_layouts_match_header():
    assert C.sizeof(q.WalkerDesc) == 64
    assert C.sizeof(q.Options) == 40
    assert q.WalkerDesc.offset.offset == 8 and q.WalkerDesc.L.offset == 24 and q.WalkerDesc.step.offset == 56
    assert q.Options.hbar2_over_m.offset == 16 and q.Options.threads_per_walker.offset == 28
    assert q.Options.walkers_per_cta.offset == 32 and q.Options.reserved.offset == 36
    src = open(HEADER).read()
    assert int(re.search(r"#define QMC_ACCUM_FIELDS (\d+)", src).group(1)) == q.NACC == 10
    assert int(re.search(r"#define QMC_VERSION (\d+)", src).group(1)) == 110


def test_capacity_matches_shared_memory():
    # 227 KB of shared memory per CTA holds 3 coordinate blocks of n floats / doubles
    assert 19000 < q.qmc_capacity(q.QMC_FP32) <= 232448 // 12
    assert 9500 < q.qmc_capacity(q.QMC_FP64) <= 232448 // 24
    assert q.qmc_capacity(q.QMC_FP32) >= 10000  # the N = 10 000 walker fits in FP32


def test_host_side_argument_errors_need_no_device():
    d = q.descs([(64, 64, 0, 0, 14.3, 0.0, 3.07, 5.0, 0.8)])
    bad = q.options(precision=7)
    with pytest.raises(q.QmcError, match="ARG"):
        q.qmc_local_energy(d, bad, 16, 16, stream=0)
    with pytest.raises(q.QmcError, match="ARG"):
        q.qmc_local_energy(d, q.options(threads_per_walker=48), 16, 16, stream=0)
    for kw in (dict(walkers_per_cta=9), dict(walkers_per_cta=-1), dict(walkers_per_cta=4, threads_per_walker=128)):
        with pytest.raises(q.QmcError, match="ARG"):
            q.qmc_local_energy(d, q.options(**kw), 16, 16, stream=0)
    o = q.options()
    o.reserved = 1
    with pytest.raises(q.QmcError, match="reserved"):
        q.qmc_local_energy(d, o, 16, 16, stream=0)
    with pytest.raises(q.QmcError, match="ARG"):
        q.qmc_sweep(d, q.options(), 16, 16, 16, 0, -1, 0, 16, stream=0)
    with pytest.raises(q.QmcError, match="ARG"):   # misaligned position pointer
        q.qmc_log_psi(d, q.options(), 20, 16, stream=0)
    assert q.lib().qmc_local_energy(d, 0, C.byref(q.options()), C.c_void_p(16), C.c_void_p(16), None) == -1
    for bad in ((0, 256, 10), (4, 48, 10), (4, 256, 0)):
        with pytest.raises(q.QmcError, match="ARG"):
            q.qmc_probe_rates(*bad, stream=0)


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(q._build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(q, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        q.lib()
