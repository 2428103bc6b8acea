"""Host logic of the trial-step tuner (bisection to a target acceptance), driven by a stand-in
for qmc_sweep whose acceptance is a known decreasing function of the step: the bracket moves
the right way, the result is the root of the move-weighted acceptance, every probe restarts the
sums, and bad arguments are refused."""
import numpy as np
import pytest
import torch
from scipy.optimize import brentq

import paper_1312_1282_gb300 as q
from paper_1312_1282_gb300 import tuning


def _rate(n, step):
    # acceptance of one walker: falls with the step, faster for the larger walker
    return 1.0 / (1.0 + (step / (1.0 if n < 100 else 1.6)) ** 2)


def _fake_sweep(calls):
    def sweep(d, opt, pos, logpsi, sw, seed, nsweeps, energy_every, accum, stream=None):
        assert energy_every == 0
        calls.append(float(d[0].step))
        for w in range(len(d)):
            accum[w, 7] += _rate(d[w].n, d[w].step) * d[w].n * nsweeps
    return sweep


def _descs_of(ns):
    def make(step):
        rows, off = [], 0
        for w, n in enumerate(ns):
            rows.append((n, n, off, w, 10.0, 0.0, 3.0, 5.0, step))
            off += 3 * n
        return q.descs(rows)
    return make


def test_bisection_converges_to_the_weighted_root(monkeypatch):
    calls = []
    monkeypatch.setattr(tuning, "qmc_sweep", _fake_sweep(calls))
    ns = [64, 64, 64, 512]
    acc = torch.full((len(ns), 8), 7.0, dtype=torch.float64)
    step, rates = tuning.tune_step(_descs_of(ns), None, None, None, None, 1, acc, target=0.5, probes=40)
    total = sum(ns)

    def weighted(s):
        return sum(n * _rate(n, s) for n in ns) / total - 0.5

    root = brentq(weighted, 0.1, 3.0, xtol=1e-14)
    assert abs(step - root) < 1e-9
    assert len(rates) == len(calls) == 40
    # the first probe runs at the start step, and each acceptance is the move-weighted one
    assert calls[0] == 0.8
    for s, r in zip(calls, rates):
        assert r == pytest.approx(weighted(s) + 0.5, rel=1e-12)
    # every probe starts from zeroed sums: accum holds the last probe only
    last = calls[-1]
    np.testing.assert_allclose(acc[:, 7].numpy(), [_rate(n, last) * n * 4 for n in ns], rtol=1e-12)


def test_five_probes_bracket_the_root(monkeypatch):
    """The default five probes of four sweeps (the benchmark workloads) shrink [0.1, 3.0] by 2^5."""
    calls = []
    monkeypatch.setattr(tuning, "qmc_sweep", _fake_sweep(calls))
    acc = torch.zeros((2, 8), dtype=torch.float64)
    step, rates = tuning.tune_step(_descs_of([64, 64]), None, None, None, None, 1, acc)
    assert len(calls) == 5
    assert abs(step - 1.0) <= 2.9 / 2 ** 5
    # above the target the step grows, below it shrinks
    for s0, s1, r in zip(calls, calls[1:] + [step], rates):
        assert (s1 > s0) == (r > 0.5)


@pytest.mark.parametrize("kw", [dict(target=0.0), dict(target=1.0), dict(lo=0.0), dict(lo=2.0, hi=1.0),
                                dict(probes=0), dict(sweeps=0)])
def test_bad_arguments_are_refused(kw):
    with pytest.raises(ValueError):
        tuning.tune_step(_descs_of([64]), None, None, None, None, 1, torch.zeros((1, 8)), **kw)
