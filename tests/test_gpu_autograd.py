"""QmcGrad: (ln psi, E_L) of each walker as differentiable functions of the Jastrow (b, m),
backed by qmc_energy_grad; the backward pass is checked against central differences of the
forward values (FP64, fixed configurations)."""
import numpy as np
import pytest
import torch

import paper_1312_1282_gb300 as q
import qmc_inputs as qi

pytestmark = pytest.mark.gpu


def _loss(batch, b, m, wl, we):
    lp, el = q.QmcGrad.apply(batch, b, m)
    return (wl * lp).sum() + (we * el).sum()


def test_backward_matches_central_differences():
    n, W = 64, 6
    L = qi.box_side(n, qi.RHO_HE)
    batch = q.Batch([(n, L, 3.07)] * W, precision=q.QMC_FP64, step=0.8).init(0x5EED0009)
    batch.sweep(30)
    g = torch.Generator().manual_seed(3)
    wl = torch.randn(W, generator=g, dtype=torch.float64).cuda()
    we = torch.randn(W, generator=g, dtype=torch.float64).cuda()
    b = torch.tensor(3.07, dtype=torch.float64, requires_grad=True)
    m = torch.tensor(5.0, dtype=torch.float64, requires_grad=True)
    loss = _loss(batch, b, m, wl, we)
    loss.backward()
    h = 1e-4

    def f(bb, mm):
        with torch.no_grad():
            return float(_loss(batch, torch.tensor(bb, dtype=torch.float64), torch.tensor(mm, dtype=torch.float64),
                               wl, we))

    def fd(fun, x0):
        c = lambda hh: (fun(x0 + hh) - fun(x0 - hh)) / (2 * hh)  # noqa: E731
        return (4 * c(h) - c(2 * h)) / 3

    gb = fd(lambda x: f(x, 5.0), 3.07)
    gm = fd(lambda x: f(3.07, x), 5.0)
    assert float(b.grad) == pytest.approx(gb, rel=1e-6, abs=1e-6)
    assert float(m.grad) == pytest.approx(gm, rel=1e-6, abs=1e-6)


def test_vmc_gradient_estimator_sign():
    """The VMC estimator 2(<E_L O_b> - <E_L><O_b>) points downhill of <E>(b): at b well below the
    optimum (about 3.07 A here) the energy falls as b grows."""
    n, W = 64, 256
    L = qi.box_side(n, qi.RHO_HE)
    batch = q.Batch([(n, L, 2.6)] * W, precision=q.QMC_FP32, step=0.8).init(0x5EED000A)
    batch.sweep(300)
    EL, Ob = [], []
    for _ in range(10):
        batch.sweep(10)
        out = batch.energy_grad()
        EL.append(out[:, 1])
        Ob.append(out[:, 2])
    EL, Ob = torch.cat(EL), torch.cat(Ob)
    grad = q.vmc_energy_gradient(EL, Ob)
    assert float(grad) < 0
    assert np.isfinite(float(grad))
