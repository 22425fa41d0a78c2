"""Phase retrieval by FISTA with the complex constrained TV prox, FP64 on the CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/ops.py``).

Forward model (Sec. V-A, Eq. (22)/(23)): A(x) = F^{-1}{ F[x] * H }. With a
zero-padded grid of M x N >= m x n the operator reads

    A = crop_{m x n} o IFFT2_{M x N} o (H *) o FFT2_{M x N} o pad_{M x N},

which is Eq. (23) itself when M = m and N = n. The object sits in the top-left
m x n corner of the padded grid; a circular shift of the placement does not
change A because the propagation is shift invariant. The adjoint is the same
chain with conj(H).

Fidelity (Eq. (24)): F(x) = 1/2 || |A x| - sqrt(y) ||^2, gradient (Eq. (27)):
A^*[(A x / |A x|) (|A x| - sqrt(y))], with A x / |A x| := 1 where A x = 0 (the
"certain complex argument" of App. C).

Algorithm 1 (FISTA), with grad F taken at z_k (step 3 prints y_k; read as z_k)
and x_0 standing in for x_{k-1} at k = 1. The prox of gamma * R with
R = tau TV + I_C is problem (15) with lam = tau * gamma (Sec. IV), solved by
``oracle.fgp.fgp``; across outer iterations the FGP dual is warm-started from
the previous q with t reset to 1.
"""
from __future__ import annotations

import math
from typing import Callable, Optional

import torch

from .fgp import fgp
from .ops import DT, Constraint

CT = torch.complex128


def pad(x: torch.Tensor, M: int, N: int) -> torch.Tensor:
    m, n = x.shape
    out = torch.zeros(M, N, dtype=CT)
    out[:m, :n] = x
    return out


def propagate(x: torch.Tensor, H: torch.Tensor) -> torch.Tensor:
    """A(x), Eq. (23) on the padded grid of H's shape."""
    m, n = x.shape
    M, N = H.shape
    return torch.fft.ifft2(torch.fft.fft2(pad(x, M, N)) * H)[:m, :n]


def propagate_adjoint(z: torch.Tensor, H: torch.Tensor) -> torch.Tensor:
    """A^*(z): pad, FFT2, multiply by conj(H), IFFT2, crop."""
    m, n = z.shape
    M, N = H.shape
    return torch.fft.ifft2(torch.fft.fft2(pad(z, M, N)) * H.conj())[:m, :n]


def unit_phase(xi: torch.Tensor) -> torch.Tensor:
    """xi / |xi|, with 1 where xi = 0."""
    a = xi.abs()
    safe = torch.where(a > 0, a, torch.ones_like(a))
    return torch.where(a > 0, xi / safe, torch.ones_like(xi))


def fidelity(x: torch.Tensor, sqrt_y: torch.Tensor, H: torch.Tensor) -> float:
    """F(x) of Eq. (24)."""
    xi = propagate(x, H)
    return 0.5 * float(((xi.abs() - sqrt_y) ** 2).sum())


def fidelity_grad(x: torch.Tensor, sqrt_y: torch.Tensor, H: torch.Tensor) -> torch.Tensor:
    """Eq. (27) as a complex image (the real pair (Re, Im) of App. C, Eq. (44)/(45))."""
    xi = propagate(x, H)
    return propagate_adjoint(unit_phase(xi) * (xi.abs() - sqrt_y), H)


def fista_pr(x0, sqrt_y, H, tau: float, gamma: float, outer: int, inner: int = 10,
             tv_type: str = "tv1_aniso", alpha: float = 0.5, C: Optional[Constraint] = None,
             accelerate: bool = True, warm_start: bool = True, record_loss: bool = False,
             F: Optional[Callable] = None, grad_F: Optional[Callable] = None,
             callback: Optional[Callable] = None):
    """Algorithm 1 (accelerate=True) or ISTA, Eq. (14) (accelerate=False).

    F and grad_F default to the fidelity of Eq. (24) and its gradient, Eq. (27),
    for (sqrt_y, H); a caller may pass another smooth fidelity (a complex image
    in, a float or a complex image out) to run the same iteration on it.
    callback(k, x_k), if given, sees every iterate (k = 1 .. outer).
    Returns (x_K, losses) where losses[k] = F(z_k) when record_loss is set."""
    x0 = torch.as_tensor(x0).to(CT)
    if F is None or grad_F is None:
        sqrt_y = torch.as_tensor(sqrt_y).to(DT)
        H = torch.as_tensor(H).to(CT)
    if F is None:
        F = lambda x: fidelity(x, sqrt_y, H)           # noqa: E731
    if grad_F is None:
        grad_F = lambda x: fidelity_grad(x, sqrt_y, H)  # noqa: E731
    lam = tau * gamma
    z = x0.clone()
    x_prev = x0.clone()
    t = 1.0
    q = None
    losses = []
    for k in range(1, outer + 1):
        if record_loss:
            losses.append(F(z))
        v = z - gamma * grad_F(z)
        res = fgp((v.real.clone(), v.imag.clone()), lam, inner, tv_type, alpha, C,
                  q0=q if warm_start else None)
        q = res.q
        x = torch.complex(res.x[0], res.x[1])
        if accelerate:
            t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
            z = x + ((t - 1.0) / t_next) * (x - x_prev)
            t = t_next
        else:
            z = x
        x_prev = x
        if callback is not None:
            callback(k, x)
    return x_prev, losses


def fista_pr_ls(x0, sqrt_y, H, tau: float, gamma0: float, eta: float, outer: int, inner: int = 10,
                tv_type: str = "tv1_aniso", alpha: float = 0.5, C: Optional[Constraint] = None,
                accelerate: bool = True, max_trials: int = 60):
    """Algorithm 1 (or Eq. (14)) with the step chosen by backtracking: starting from
    the previous step, gamma <- eta * gamma until
        F(x) <= F(z) + <x - z, grad F(z)> + ||x - z||^2 / (2 gamma),
    x being the prox step from z with that gamma (the FGP warm start is the
    previous outer iteration's dual for every trial). Returns (x_K, gammas)."""
    x0 = torch.as_tensor(x0).to(CT)
    sqrt_y = torch.as_tensor(sqrt_y).to(DT)
    H = torch.as_tensor(H).to(CT)
    z = x0.clone()
    x_prev = x0.clone()
    t = 1.0
    q = None
    gamma = float(gamma0)
    gammas = []
    for _ in range(outer):
        Fz = fidelity(z, sqrt_y, H)
        g = fidelity_grad(z, sqrt_y, H)
        for _trial in range(max_trials):
            v = z - gamma * g
            res = fgp((v.real.clone(), v.imag.clone()), tau * gamma, inner, tv_type, alpha, C, q0=q)
            x = torch.complex(res.x[0], res.x[1])
            d = x - z
            rhs = Fz + float((d.real * g.real + d.imag * g.imag).sum()) + float((d.abs() ** 2).sum()) / (2 * gamma)
            if fidelity(x, sqrt_y, H) <= rhs:
                break
            gamma *= eta
        gammas.append(gamma)
        q = res.q
        if accelerate:
            t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
            z = x + ((t - 1.0) / t_next) * (x - x_prev)
            t = t_next
        else:
            z = x
        x_prev = x
    return x_prev, gammas
