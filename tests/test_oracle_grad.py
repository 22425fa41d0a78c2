"""Pins for the oracle's gradient of unrolled FGP (the reference for the adjoint
kernel): autograd through ``oracle.fgp.fgp`` against FP64 central finite
differences, with respect to b (random directions and single entries) and lam."""
import numpy as np
import pytest
import torch

from oracle.fgp import fgp
from oracle.ops import DT, TV_TYPES, Constraint
from phantoms import noisy_phantom


def loss_of(bu, bv, lam, K, tv_type, C, gt):
    res = fgp((bu, bv), lam, K, tv_type, 0.5, C)
    return ((res.x[0] - gt[0]) ** 2).sum() + ((res.x[1] - gt[1]) ** 2).sum()


@pytest.mark.parametrize("tv_type", TV_TYPES)
def test_unrolled_gradient_fd(tv_type):
    m, n, K = 12, 10, 15
    clean, noisy = noisy_phantom(m, n, 0.15, seed=13)
    gt = (torch.tensor(clean.real), torch.tensor(clean.imag))
    C = Constraint(amp_max=1.0)
    bu = torch.tensor(noisy.real, requires_grad=True)
    bv = torch.tensor(noisy.imag, requires_grad=True)
    lam = torch.tensor(0.07, dtype=DT, requires_grad=True)
    loss = loss_of(bu, bv, lam, K, tv_type, C, gt)
    gu, gv, gl = torch.autograd.grad(loss, (bu, bv, lam))
    h = 1e-6
    rng = np.random.default_rng(1)
    with torch.no_grad():
        for _ in range(3):
            du = torch.tensor(rng.standard_normal((m, n)))
            dv = torch.tensor(rng.standard_normal((m, n)))
            lp = loss_of(bu + h * du, bv + h * dv, lam, K, tv_type, C, gt)
            lm = loss_of(bu - h * du, bv - h * dv, lam, K, tv_type, C, gt)
            fd = float(lp - lm) / (2 * h)
            an = float((gu * du).sum() + (gv * dv).sum())
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
        lp = loss_of(bu, bv, lam + h, K, tv_type, C, gt)
        lm = loss_of(bu, bv, lam - h, K, tv_type, C, gt)
        fd = float(lp - lm) / (2 * h)
        assert abs(fd - float(gl)) <= 1e-6 * max(1.0, abs(float(gl)))
        # a few single entries
        for (j, k) in [(0, 0), (m - 1, n - 1), (5, 3)]:
            e = torch.zeros(m, n, dtype=DT)
            e[j, k] = 1.0
            fd = float(loss_of(bu + h * e, bv, lam, K, tv_type, C, gt) - loss_of(bu - h * e, bv, lam, K, tv_type, C, gt)) / (2 * h)
            assert abs(fd - float(gu[j, k])) <= 1e-6 * max(1.0, abs(float(gu[j, k])))
