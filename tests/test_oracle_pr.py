"""Pins for the phase-retrieval oracle: the propagator of Eq. (23) and its
adjoint, the gradient of Eq. (27) against FP64 finite differences of Eq. (24),
the error-reduction identity for a unitary A, and Algorithm 1 / Eq. (14)."""
import math

import numpy as np
import pytest
import torch

from oracle import pr
from oracle.fgp import primal_value
from oracle.ops import DT, Constraint, tv
from phantoms import angular_spectrum_tf, fresnel_tf, pr_object, simulate_intensity

CT = torch.complex128


def rand_c(m, n, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return torch.complex(scale * torch.randn(m, n, generator=g, dtype=DT),
                         scale * torch.randn(m, n, generator=g, dtype=DT))


def test_propagator_adjoint():
    m, n, M, N = 12, 10, 24, 20
    H = torch.tensor(fresnel_tf(M, N, 532e-9, 2e-6, 5e-3))
    x, z = rand_c(m, n, 1), rand_c(m, n, 2)
    lhs = torch.vdot(pr.propagate(x, H).flatten(), z.flatten())
    rhs = torch.vdot(x.flatten(), pr.propagate_adjoint(z, H).flatten())
    assert abs(complex(lhs - rhs)) < 1e-12 * abs(complex(lhs))


def test_propagator_unpadded_is_unitary_and_matches_eq23():
    m = n = 16
    H = torch.tensor(angular_spectrum_tf(m, n, 500e-9, 5e-6, 5e-3))
    assert float((H.abs() - 1).abs().max()) < 1e-12       # no evanescent waves at these settings
    x = rand_c(m, n, 3)
    Ax = pr.propagate(x, H)
    assert abs(float(Ax.abs().pow(2).sum()) - float(x.abs().pow(2).sum())) < 1e-10 * float(x.abs().pow(2).sum())
    # Eq. (23) by an explicit DFT matrix (no FFT): F^{-1} diag(H) F
    W = torch.tensor(np.exp(-2j * np.pi * np.outer(np.arange(m), np.arange(m)) / m))
    Fx = W @ x @ W.T
    back = (W.conj() @ (Fx * H) @ W.conj().T) / (m * n)
    assert float((back - Ax).abs().max()) < 1e-12


@pytest.mark.parametrize("padded", [False, True])
def test_fidelity_gradient_finite_differences(padded):
    m, n = 8, 8
    M, N = (16, 16) if padded else (8, 8)
    H = torch.tensor(fresnel_tf(M, N, 532e-9, 2e-6, 5e-3))
    x_gt = torch.tensor(pr_object(m, n, seed=5, blur_sigma=1.0))
    sqrt_y = torch.tensor(np.sqrt(simulate_intensity(x_gt.numpy(), H.numpy(), seed=1, photons=0)))
    x = x_gt + 0.1 * rand_c(m, n, 7)
    g = pr.fidelity_grad(x, sqrt_y, H)
    h = 1e-6
    for j in range(m):
        for k in range(0, n, 3):
            for unit in (1.0, 1j):
                e = torch.zeros(m, n, dtype=CT)
                e[j, k] = unit
                fd = (pr.fidelity(x + h * e, sqrt_y, H) - pr.fidelity(x - h * e, sqrt_y, H)) / (2 * h)
                an = float(g[j, k].real) if unit == 1.0 else float(g[j, k].imag)
                assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


def test_error_reduction_identity():
    # A unitary (no padding, |H| = 1): x - grad F(x) = A^*(sqrt(y) * A x / |A x|)
    m = n = 10
    H = torch.tensor(fresnel_tf(m, n, 532e-9, 2e-6, 5e-3))
    x = rand_c(m, n, 11)
    sqrt_y = torch.rand(m, n, dtype=DT, generator=torch.Generator().manual_seed(3))
    lhs = x - pr.fidelity_grad(x, sqrt_y, H)
    xi = pr.propagate(x, H)
    rhs = pr.propagate_adjoint(sqrt_y * xi / xi.abs(), H)
    assert float((lhs - rhs).abs().max()) < 1e-12


def test_zero_field_convention():
    # A x = 0 everywhere: the unit phase is 1, so grad F = A^*(-sqrt(y))
    m = n = 6
    H = torch.tensor(fresnel_tf(m, n, 532e-9, 2e-6, 5e-3))
    sqrt_y = torch.ones(m, n, dtype=DT)
    g = pr.fidelity_grad(torch.zeros(m, n, dtype=CT), sqrt_y, H)
    want = pr.propagate_adjoint(-sqrt_y.to(CT), H)
    assert float((g - want).abs().max()) < 1e-14


def _pr_problem(m=32, seed=3):
    M = 2 * m
    H = torch.tensor(fresnel_tf(M, M, 532e-9, 2e-6, 5e-3))
    x_gt = pr_object(m, m, seed=seed, blur_sigma=2.0)
    y = simulate_intensity(x_gt, H.numpy(), seed=seed + 1, photons=1e4)
    sqrt_y = torch.tensor(np.sqrt(y))
    x0 = pr.propagate_adjoint(sqrt_y.to(CT), H)
    return H, sqrt_y, x0, x_gt


def test_fista_decreases_objective_and_beats_ista():
    H, sqrt_y, x0, _ = _pr_problem()
    tau, gamma = 0.01, 1.0
    C = Constraint(amp_max=1.0)

    def objective(x):
        return pr.fidelity(x, sqrt_y, H) + tau * float(tv(x.real, x.imag, "tv1_aniso"))

    xf, _ = pr.fista_pr(x0, sqrt_y, H, tau, gamma, 40, 10, "tv1_aniso", 0.5, C)
    xi, _ = pr.fista_pr(x0, sqrt_y, H, tau, gamma, 40, 10, "tv1_aniso", 0.5, C, accelerate=False)
    f0 = objective(torch.complex(*[t for t in (x0.real / torch.clamp(x0.abs(), min=1), x0.imag / torch.clamp(x0.abs(), min=1))]))
    assert objective(xf) < f0 and objective(xi) < f0
    assert objective(xf) <= objective(xi)
    assert float(xf.abs().max()) <= 1 + 1e-12          # x_K lies in C


def test_fista_one_step_is_prox_of_gradient_step():
    # K = 1: x_1 = prox_{gamma R}(x_0 - gamma grad F(x_0)), the prox being Algorithm 2
    from oracle.fgp import fgp
    H, sqrt_y, x0, _ = _pr_problem(16, 5)
    tau, gamma = 0.02, 0.8
    C = Constraint(amp_max=1.0)
    x1, _ = pr.fista_pr(x0, sqrt_y, H, tau, gamma, 1, 7, "tv2_iso", 0.5, C)
    v = x0 - gamma * pr.fidelity_grad(x0, sqrt_y, H)
    res = fgp((v.real.clone(), v.imag.clone()), tau * gamma, 7, "tv2_iso", 0.5, C)
    assert float((x1 - torch.complex(*res.x)).abs().max()) == 0.0


def test_line_search_reduces_to_fixed_step_and_backtracks():
    H, sqrt_y, x0, _ = _pr_problem(24, 7)
    C = Constraint(amp_max=1.0)
    # a step that always passes the sufficient-decrease test: identical to the fixed-step run
    x_ls, gam = pr.fista_pr_ls(x0, sqrt_y, H, 0.01, 0.25, 0.5, 6, 5, "tv1_aniso", 0.5, C)
    assert gam == [0.25] * 6
    x_fx, _ = pr.fista_pr(x0, sqrt_y, H, 0.01, 0.25, 6, 5, "tv1_aniso", 0.5, C)
    assert float((x_ls - x_fx).abs().max()) == 0.0
    # a step that is far too long is shortened, never lengthened, and each accepted
    # step satisfies the sufficient-decrease inequality at the iterate it was taken from
    x_ls, gam = pr.fista_pr_ls(x0, sqrt_y, H, 0.01, 64.0, 0.5, 6, 5, "tv1_aniso", 0.5, C, accelerate=False)
    assert gam[0] < 64.0 and all(a >= b for a, b in zip(gam, gam[1:]))
    z = torch.as_tensor(x0).to(torch.complex128)
    from oracle.fgp import fgp as _fgp
    g = pr.fidelity_grad(z, sqrt_y, H)
    v = z - gam[0] * g
    res = _fgp((v.real.clone(), v.imag.clone()), 0.01 * gam[0], 5, "tv1_aniso", 0.5, C)
    x1 = torch.complex(*res.x)
    d = x1 - z
    rhs = pr.fidelity(z, sqrt_y, H) + float((d.real * g.real + d.imag * g.imag).sum()) + \
        float((d.abs() ** 2).sum()) / (2 * gam[0])
    assert pr.fidelity(x1, sqrt_y, H) <= rhs


def _ill_conditioned_quadratic(m, n, seed, spread):
    """F(x) = 1/2 sum mu |x - c|^2 with mu spread log-uniformly over [spread, 1]:
    convex, gradient Lipschitz constant L = 1, minimiser x* = c, F* = 0."""
    g = torch.Generator().manual_seed(seed)
    mu = torch.logspace(math.log10(spread), 0.0, m * n, dtype=DT).reshape(m, n)
    mu = mu.flatten()[torch.randperm(m * n, generator=g)].reshape(m, n)
    c = rand_c(m, n, seed + 1)

    def F(x):
        return 0.5 * float((mu * (x - c).abs() ** 2).sum())

    def grad_F(x):
        return mu * (x - c)

    return F, grad_F, c


def test_fista_momentum_beck_teboulle_rate():
    # With tau = 0 and no constraint the prox of Algorithm 1 is the identity, so the
    # iteration is accelerated gradient descent on F. Beck and Teboulle (2009),
    # Theorem 4.4: with step gamma = 1/L, F(x_k) - F* <= 2 ||x_0 - x*||^2 / (gamma (k+1)^2)
    # for every k >= 1. ISTA (Eq. (14)) only has an O(1/k) rate, and on this
    # ill-conditioned F it leaves that bound, so an iteration that lost its momentum
    # fails here. (A wrong extrapolation weight can still meet the bound; the
    # estimate-sequence identity below is the pin for the weight itself.)
    m = n = 16
    F, grad_F, c = _ill_conditioned_quadratic(m, n, 21, 1e-4)
    x0 = torch.zeros(m, n, dtype=CT)
    R2 = float(((x0 - c).abs() ** 2).sum())
    K, gamma = 300, 1.0

    def run(accelerate):
        vals = []
        pr.fista_pr(x0, None, None, 0.0, gamma, K, 1, "tv1_aniso", 0.5, None, accelerate=accelerate,
                    F=F, grad_F=grad_F, callback=lambda k, x: vals.append(F(x)))
        return vals

    fista, ista = run(True), run(False)
    assert len(fista) == K
    for k in range(1, K + 1):
        assert fista[k - 1] <= 2.0 * R2 / (gamma * (k + 1) ** 2)
    assert any(ista[k - 1] > 2.0 * R2 / (gamma * (k + 1) ** 2) for k in range(1, K + 1))
    assert fista[199] < 0.1 * ista[199]


def test_fista_momentum_estimate_sequence_identity():
    # Nesterov's method in its two-sequence form (Tseng 2008; the u_k of Beck and
    # Teboulle's proof of Theorem 4.4 is v_k - x*): with no prox to apply,
    #     v_k = x_{k-1} + t_k (x_k - x_{k-1})   obeys   v_k = v_{k-1} - gamma t_k grad F(z_k),
    # v_0 = x_0, where z_k is the point whose gradient step gave x_k and t_k is the
    # positive root of t_k^2 - t_k = t_{k-1}^2 (t_1 = 1). It holds only for the
    # extrapolation weight (t_k - 1)/t_{k+1} of Algorithm 1, step 5.
    m, n = 12, 10
    F, grad_F, c = _ill_conditioned_quadratic(m, n, 31, 1e-3)
    x0 = rand_c(m, n, 33)
    gamma, K = 0.8, 60
    zs, xs = [], [x0]

    def grad_rec(z):
        zs.append(z.clone())
        return grad_F(z)

    pr.fista_pr(x0, None, None, 0.0, gamma, K, 1, "tv1_aniso", 0.5, None, F=F, grad_F=grad_rec,
                callback=lambda k, x: xs.append(x.clone()))
    assert len(zs) == K and len(xs) == K + 1
    t = [None, 1.0]
    for _ in range(K):
        tp = t[-1]
        t.append(0.5 + math.sqrt(0.25 + tp * tp))   # root of s^2 - s - tp^2 = 0
    v_prev = x0
    for k in range(1, K + 1):
        v = xs[k - 1] + t[k] * (xs[k] - xs[k - 1])
        want = v_prev - gamma * t[k] * grad_F(zs[k - 1])
        assert float((v - want).abs().max()) <= 1e-10 * max(1.0, float(want.abs().max()))
        v_prev = v
