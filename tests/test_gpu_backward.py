"""GPU differentiation through unrolled FGP (ctv_unrolled_forward / _backward,
UnrolledFGP) against the oracle's FP64 autograd of Algorithm 2, against FP64
finite differences of the oracle, and (forward) bit-for-bit against
ctv_denoise_batched with the same configuration."""
import numpy as np
import pytest
import torch

import paper_2109_05496_gb300 as ctv
from oracle.fgp import fgp
from oracle.ops import DT
from phantoms import noisy_phantom, to_c64
from tests.helpers import TV_NAMES, f32, oracle_constraint

pytestmark = pytest.mark.gpu

# Gradients of the unrolled iteration are those of a piecewise smooth map: where a
# projection (P_S, P_C) switches branch within the rounding error of the forward
# iterates, the FP32 and FP64 sweeps differentiate different pieces and their
# gradients differ by O(1) there (the FP64 oracle's own gradient moves by 0.3% of
# its largest entry under an input change of 1e-7 on a 128^2 image, 50
# iterations, TV1 anisotropic). Small seeded inputs below stay away from kinks:
# bar 1e-4, 25x the largest difference measured on them. On the full-size
# 8 x 1024^2 workload some pixel always sits near a kink; there the oracle's own
# lambda-gradient moves by 1.2-2.9% (and its derivative along a random input
# direction by 0.5-1.6%) under a 1e-6 relative input change, the size of the
# FP32 forward error after 50 iterations, while the GPU agreed within 6.3e-5 and
# 8.7e-4: bar 2e-3.
GRAD_TOL = 1e-4
FULL_SIZE_GRAD_TOL = 2e-3


def oracle_grads(b_np, lams, K, tv, alpha, Co, xbar_np):
    """d<xbar, x>/db and d<xbar, x>/dlam of the oracle in FP64, per image."""
    gb, gl = [], []
    for i in range(b_np.shape[0]):
        bb = torch.tensor(b_np[i].astype(np.complex128))
        bu = bb.real.clone().requires_grad_(True)
        bv = bb.imag.clone().requires_grad_(True)
        lam = torch.tensor(f32(lams[i]), dtype=DT, requires_grad=True)
        res = fgp((bu, bv), lam, K, tv, f32(alpha), Co)
        xb = torch.tensor(xbar_np[i].astype(np.complex128))
        loss = (res.x[0] * xb.real).sum() + (res.x[1] * xb.imag).sum()
        du, dv, dl = torch.autograd.grad(loss, (bu, bv, lam))
        gb.append((du + 1j * dv).numpy())
        gl.append(float(dl))
    return np.stack(gb), np.array(gl)


def gpu_grads(b_np, lams, K, tv, alpha, C, xbar_np, ckpt, config=-1):
    b = torch.from_numpy(b_np.astype(np.complex64)).cuda().requires_grad_(True)
    lt = torch.tensor(lams, dtype=torch.float32, device="cuda", requires_grad=True)
    x = ctv.denoise_unrolled(b, lt, tv, K, C, alpha, ckpt, config)
    xb = torch.from_numpy(xbar_np.astype(np.complex64)).cuda()
    # <xbar, x> in the real-pair inner product; torch's complex gradient is dL/dRe + i dL/dIm
    loss = (x.real * xb.real).sum() + (x.imag * xb.imag).sum()
    loss.backward()
    torch.cuda.synchronize()
    return x.detach(), b.grad.cpu().numpy(), lt.grad.cpu().numpy()


def make(Bn, m, n, seed, sigma=0.15):
    imgs = np.stack([to_c64(noisy_phantom(m, n, sigma, seed=seed + i)[1]) for i in range(Bn)])
    rng = np.random.default_rng(seed + 99)
    xbar = (rng.standard_normal((Bn, m, n)) + 1j * rng.standard_normal((Bn, m, n))).astype(np.complex64)
    return imgs, xbar


@pytest.mark.parametrize("tv", TV_NAMES)
@pytest.mark.parametrize("kind", ["amp", "amp_rect", "none"])
def test_unrolled_gradient_matches_oracle(tv, kind):
    Bn, m, n, K, ckpt = 2, 37, 70, 13, 4
    imgs, xbar = make(Bn, m, n, seed=7)
    lams = [0.04, 0.09]
    if kind == "none":
        C, Co = ctv.NO_CONSTRAINT, None
    elif kind == "amp":
        C, Co = ctv.Constraint(amp_max=1.0), oracle_constraint(1.0)
    else:
        r = (3, 5, 30, 61)
        C, Co = ctv.Constraint(amp_max=1.0, rect=r), oracle_constraint(1.0, rect=r)
    _, gb, gl = gpu_grads(imgs, lams, K, tv, 0.5, C, xbar, ckpt)
    ob, ol = oracle_grads(imgs, lams, K, tv, 0.5, Co, xbar)
    scale = np.abs(ob).max()
    # GRAD_TOL: away from the projections' kinks the FP32 reverse sweep agrees with
    # the FP64 one to about 5e-7 of the largest entry (dL/db) and 4e-6 (dL/dlambda)
    # on these inputs; see the module docstring for inputs near a kink
    assert np.abs(gb - ob).max() <= GRAD_TOL * scale, np.abs(gb - ob).max() / scale
    np.testing.assert_allclose(gl, ol, rtol=GRAD_TOL, atol=GRAD_TOL * np.abs(ol).max())


@pytest.mark.parametrize("ckpt", [1, 3, 10, 50])
def test_checkpoint_spacing_does_not_change_result(ckpt):
    imgs, xbar = make(1, 40, 33, seed=3)
    ref = None
    _, gb, gl = gpu_grads(imgs, [0.05], 10, "tv1_iso", 0.5, ctv.Constraint(amp_max=1.0), xbar, ckpt)
    _, gb1, gl1 = gpu_grads(imgs, [0.05], 10, "tv1_iso", 0.5, ctv.Constraint(amp_max=1.0), xbar, 10)
    # The spacing decides which reverse-step kernel runs (two steps per pass where
    # a segment has two left, else one); the two are compiled separately, so the
    # compiler may fuse a multiply and an add in one and not in the other, and
    # the FP32 partial sums of dL/dlambda group pixels differently: equal up to
    # FP32 rounding, not bit for bit.
    np.testing.assert_allclose(gb, gb1, rtol=0, atol=1e-5 * np.abs(gb1).max())
    np.testing.assert_allclose(gl, gl1, rtol=1e-5)


def test_unrolled_forward_equals_batched_denoise():
    imgs, _ = make(3, 64, 96, seed=11)
    b = torch.from_numpy(imgs).cuda()
    lams = torch.tensor([0.02, 0.05, 0.08], device="cuda")
    for tv in TV_NAMES:
        x1 = ctv.denoise_unrolled(b, lams, tv, 25, ctv.Constraint(amp_max=1.0), 0.5, 10, 2)
        x2 = ctv.denoise(b, lams, tv, 25, ctv.Constraint(amp_max=1.0), 0.5, config=2)
        assert torch.equal(x1, x2)


@pytest.mark.parametrize("tv", TV_NAMES)
def test_finite_differences_fp64_32x32(tv):
    # FP64 central differences of the oracle's loss ||x - x_gt||^2 along random
    # directions against the GPU gradient (the gradient of the same loss)
    m = n = 32
    K = 20
    clean, noisy = noisy_phantom(m, n, 0.15, seed=5)
    b_np = to_c64(noisy)[None]
    gt = torch.tensor(clean)
    lam = 0.06
    Co = oracle_constraint(1.0)

    def loss64(bc, lamv):
        res = fgp((bc.real.clone(), bc.imag.clone()), lamv, K, tv, 0.5, Co)
        return float(((res.x[0] - gt.real) ** 2).sum() + ((res.x[1] - gt.imag) ** 2).sum())

    b = torch.from_numpy(b_np).cuda().requires_grad_(True)
    lt = torch.tensor([lam], dtype=torch.float32, device="cuda", requires_grad=True)
    x = ctv.denoise_unrolled(b, lt, tv, K, ctv.Constraint(amp_max=1.0), 0.5, 5)
    g = torch.from_numpy(clean.astype(np.complex64)).cuda()[None]
    loss = ((x - g).abs() ** 2).sum()
    loss.backward()
    gb = b.grad.cpu().numpy()[0].astype(np.complex128)
    bc = torch.tensor(b_np[0].astype(np.complex128))
    rng = np.random.default_rng(2)
    # central differences of step h = 1e-6 in FP64: the bar (2e-3, relative to
    # max(1, |fd|)) leaves room for a difference whose interval crosses a kink
    h = 1e-6
    for _ in range(3):
        d = torch.tensor(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))
        fd = (loss64(bc + h * d, f32(lam)) - loss64(bc - h * d, f32(lam))) / (2 * h)
        an = float((gb.real * d.real.numpy()).sum() + (gb.imag * d.imag.numpy()).sum())
        assert abs(fd - an) <= 2e-3 * max(1.0, abs(fd))
    fd = (loss64(bc, f32(lam) + h) - loss64(bc, f32(lam) - h)) / (2 * h)
    assert abs(fd - float(lt.grad)) <= 2e-3 * max(1.0, abs(fd))


def test_full_size_gradient_window():
    # the differentiation workload: 8 x 1024^2, 50 iterations, checkpoints every 10;
    # the gradient at sample pixels against the oracle on a window around them
    # (the gradient at a pixel depends only on inputs within about 3K pixels)
    Bn, m, n, K = 8, 1024, 1024, 50
    imgs = np.stack([to_c64(noisy_phantom(m, n, 0.1, seed=500 + i)[1]) for i in range(Bn)])
    rng = np.random.default_rng(8)
    xbar = (rng.standard_normal((Bn, m, n)) + 1j * rng.standard_normal((Bn, m, n))).astype(np.complex64)
    lams = np.linspace(0.02, 0.09, Bn)
    C = ctv.Constraint(amp_max=1.0)
    _, gb, gl = gpu_grads(imgs, lams, K, "tv1_iso", 0.5, C, xbar, 10)
    assert np.all(np.isfinite(gb)) and np.all(np.isfinite(gl))
    R = 3 * K + 8
    for (i, j, k) in [(0, 500, 500), (5, 3, 1020)]:
        j0, j1 = max(0, j - R), min(m, j + R + 1)
        k0, k1 = max(0, k - R), min(n, k + R + 1)
        ob, _ = oracle_grads(imgs[i:i + 1, j0:j1, k0:k1], [lams[i]], K, "tv1_iso", 0.5, oracle_constraint(1.0),
                             xbar[i:i + 1, j0:j1, k0:k1])
        want = ob[0, j - j0, k - k0]
        scale = np.abs(ob).max()
        assert abs(gb[i, j, k] - want) <= FULL_SIZE_GRAD_TOL * scale


def _oracle_forward_derivative(b_np, lam, K, tv, alpha, Co, xbar_np, db=None):
    """d<xbar, x_K>/dlam (db None) or the derivative along the input direction db,
    by forward-mode FP64 differentiation of the oracle (one pass, no stored graph)."""
    import torch.autograd.forward_ad as fwAD
    bb = torch.tensor(b_np.astype(np.complex128))
    xb = torch.tensor(xbar_np.astype(np.complex128))
    with fwAD.dual_level():
        if db is None:
            lam_d = fwAD.make_dual(torch.tensor(f32(lam), dtype=DT), torch.tensor(1.0, dtype=DT))
            b_pair = (bb.real.clone(), bb.imag.clone())
        else:
            lam_d = f32(lam)
            d = torch.tensor(db)
            b_pair = (fwAD.make_dual(bb.real.clone(), d.real.clone()), fwAD.make_dual(bb.imag.clone(), d.imag.clone()))
        res = fgp(b_pair, lam_d, K, tv, f32(alpha), Co)
        loss = (res.x[0] * xb.real).sum() + (res.x[1] * xb.imag).sum()
        return float(fwAD.unpack_dual(loss).tangent)


def test_full_size_lambda_gradient_and_directional_derivative():
    # The differentiation workload (8 x 1024^2, 50 iterations, checkpoints every
    # 10): lambda-bar of two whole images, and <b-bar, d> along a random input
    # direction d, against forward-mode FP64 derivatives of the oracle's unrolled
    # Algorithm 2 on the full image (an independent differentiation mode: no
    # reverse sweep, no checkpoints).
    Bn, m, n, K = 8, 1024, 1024, 50
    imgs = np.stack([to_c64(noisy_phantom(m, n, 0.1, seed=600 + i)[1]) for i in range(Bn)])
    rng = np.random.default_rng(9)
    xbar = (rng.standard_normal((Bn, m, n)) + 1j * rng.standard_normal((Bn, m, n))).astype(np.complex64)
    lams = np.linspace(0.02, 0.09, Bn)
    C, Co = ctv.Constraint(amp_max=1.0), oracle_constraint(1.0)
    _, gb, gl = gpu_grads(imgs, lams, K, "tv1_iso", 0.5, C, xbar, 10)
    for i in (1, 6):
        want = _oracle_forward_derivative(imgs[i], lams[i], K, "tv1_iso", 0.5, Co, xbar[i])
        assert abs(gl[i] - want) <= FULL_SIZE_GRAD_TOL * abs(want), (gl[i], want)
        d = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
        want_b = _oracle_forward_derivative(imgs[i], lams[i], K, "tv1_iso", 0.5, Co, xbar[i], db=d)
        got_b = float((gb[i].real.astype(np.float64) * d.real + gb[i].imag.astype(np.float64) * d.imag).sum())
        assert abs(got_b - want_b) <= FULL_SIZE_GRAD_TOL * abs(want_b), (got_b, want_b)
