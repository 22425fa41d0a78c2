"""Dual (fast) gradient projection for problem (1)/(15), FP64 on the CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/ops.py``).

Follows Prop. 1 and Algorithm 2 step by step in the paper's notation:

    w      = b - lam * L^T(r_k)                      (argument of P_C, Eq. (18)/(19))
    grad h = -2 lam L(P_C(w))                         Eq. (19)
    q_k    = P_S(r_k - grad h / (16 lam^2))           Alg. 2, step 3
    t_k+1  = (1 + sqrt(1 + 4 t_k^2)) / 2              Alg. 2, step 4
    r_k+1  = q_k + ((t_k - 1)/t_k+1) (q_k - q_k-1)    Alg. 2, step 5

and returns x_K = P_C(b - lam L^T(q_K)) (Eq. (18); Algorithm 2 does not print
its output, this is the reading used throughout).

Dual value used for the duality gap: App. A, Eq. (30) multiplied by lam,

    D(q) = 1/2 (||b||^2 - ||w||^2 + ||w - P_C(w)||^2),   w = b - lam L^T(q),

so that P(x) - D(q) >= 0 for every x in C and q in S, with
P(x) = 1/2 ||x - b||^2 + lam TV(x) (problem (1)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import torch

from .ops import DT, L, LT, P_C, P_S, Constraint, tv, zeros_dual


def grad_h(r, b, lam, C, ):
    """Eq. (19): gradient of h at r (h as in Eq. (16))."""
    wu, wv = LT(r)
    w = (b[0] - lam * wu, b[1] - lam * wv)
    x = P_C(w[0], w[1], C)
    return tuple(-2.0 * lam * d for d in L(x[0], x[1]))


def primal_value(x, b, lam, tv_type, alpha=0.5):
    """Objective of problem (1) at x (x is assumed to lie in C)."""
    return 0.5 * (((x[0] - b[0]) ** 2).sum() + ((x[1] - b[1]) ** 2).sum()) + lam * tv(x[0], x[1], tv_type, alpha)


def dual_value(q, b, lam, C):
    """lam times the Lagrange dual function of App. A, Eq. (30)."""
    lu, lv = LT(q)
    wu, wv = b[0] - lam * lu, b[1] - lam * lv
    pu, pv = P_C(wu, wv, C)
    nb = (b[0] ** 2).sum() + (b[1] ** 2).sum()
    nw = (wu ** 2).sum() + (wv ** 2).sum()
    nh = ((wu - pu) ** 2).sum() + ((wv - pv) ** 2).sum()
    return 0.5 * (nb - nw + nh)


def primal_from_dual(q, b, lam, C):
    """Eq. (18): x = P_C(b - lam L^T(q))."""
    lu, lv = LT(q)
    return P_C(b[0] - lam * lu, b[1] - lam * lv, C)


@dataclass
class FGPResult:
    x: tuple                       # (u, v) of x_K, Eq. (18)
    q: tuple                       # q_K (paper shapes)
    r: tuple                       # r_{K+1}
    t: float                       # t_{K+1}
    iters: int
    history: List[dict] = field(default_factory=list)


def nesterov_t(K: int) -> List[float]:
    """t_1 .. t_{K+1} of Alg. 2, step 4."""
    t = [1.0]
    for _ in range(K):
        t.append((1.0 + math.sqrt(1.0 + 4.0 * t[-1] * t[-1])) / 2.0)
    return t


def fgp(b, lam, K: int, tv_type: str = "tv1_iso", alpha: float = 0.5,
        C: Optional[Constraint] = None, q0=None, accelerate: bool = True,
        check_every: int = 0, gap_tol: float = 0.0) -> FGPResult:
    """Algorithm 2 (accelerate=True) or the plain gradient projection (21).

    b:   pair (u, v) of FP64 m x n tensors.
    q0:  optional warm start; q_0 = r_1 = q0 and t_1 = 1.
    check_every > 0 evaluates primal, dual and gap at q_k every check_every
    iterations (at q_k, never at the extrapolated r_k) and, when gap_tol > 0,
    stops at the first check with gap <= gap_tol * max(primal, 1e-30).
    """
    m, n = b[0].shape
    if lam == 0 or K == 0:
        if q0 is None:
            q0 = zeros_dual(m, n)
        x = primal_from_dual(q0, b, lam, C) if lam != 0 else P_C(b[0], b[1], C)
        return FGPResult(x=x, q=q0, r=q0, t=1.0, iters=0)
    proj = P_S[tv_type]
    q_prev = zeros_dual(m, n) if q0 is None else tuple(t.clone() for t in q0)
    r = q_prev
    t = 1.0
    hist = []
    k_done = 0
    for k in range(1, K + 1):
        g = grad_h(r, b, lam, C)
        step = 1.0 / (16.0 * lam * lam)
        q = proj(tuple(ri - step * gi for ri, gi in zip(r, g)), alpha)
        if accelerate:
            t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
            beta = (t - 1.0) / t_next
            r = tuple(qi + beta * (qi - pi) for qi, pi in zip(q, q_prev))
            t = t_next
        else:                                   # Eq. (21)
            r = q
        q_prev = q
        k_done = k
        if check_every and k % check_every == 0:
            x = primal_from_dual(q, b, lam, C)
            P = float(primal_value(x, b, lam, tv_type, alpha))
            D = float(dual_value(q, b, lam, C))
            hist.append({"k": k, "primal": P, "dual": D, "gap": P - D})
            if gap_tol > 0 and P - D <= gap_tol * max(P, 1e-30):
                break
    x = primal_from_dual(q_prev, b, lam, C)
    return FGPResult(x=x, q=q_prev, r=r, t=t, iters=k_done, history=hist)


def denoise(b_complex, lam, K, tv_type="tv1_iso", alpha=0.5, C=None, **kw):
    """Convenience wrapper on complex input (numpy or torch); returns complex128 torch."""
    bt = torch.as_tensor(b_complex)
    b = (bt.real.to(DT), bt.imag.to(DT))
    res = fgp(b, lam, K, tv_type, alpha, C, **kw)
    return torch.complex(res.x[0], res.x[1]), res


def stats(x, q, b, lam, tv_type, alpha, C):
    P = float(primal_value(x, b, lam, tv_type, alpha))
    D = float(dual_value(q, b, lam, C))
    return {"primal": P, "dual": D, "gap": P - D}
