"""Discrete operators of the complex TV model, written out in FP64 on the CPU.

TEST INFRASTRUCTURE ONLY. This package is the oracle that the CUDA path is
checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library never does.

Representation (Sec. II, "real-pair view"): a complex image x = u + i v is the
pair of real m x n tensors (u, v). The finite-difference group of Eq. (5)/(6) and
the dual variable of Prop. 1 keep the paper's own, unpadded shapes:

    q = (r1, r2, s1, s2),  r1, s1: (m-1) x n (vertical),  r2, s2: m x (n-1).

Indices j (row) and k (column) are 0-based here; the paper counts from 1.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Tuple

import torch
import torch.nn.functional as F

DT = torch.float64

TV_TYPES = ("tv1_iso", "tv1_aniso", "tv2_iso", "tv2_aniso")


# --------------------------------------------------------------------------
# Linear map L (image -> finite differences) and its adjoint L^T
# --------------------------------------------------------------------------
def finite_differences(u: torch.Tensor) -> Tuple[torch.Tensor, torch.Tensor]:
    """Eq. (5): vertical u1[j,k] = u[j,k] - u[j+1,k] ((m-1) x n) and horizontal
    u2[j,k] = u[j,k] - u[j,k+1] (m x (n-1))."""
    return u[:-1, :] - u[1:, :], u[:, :-1] - u[:, 1:]


def L(u: torch.Tensor, v: torch.Tensor):
    """The map of Prop. 1 from x = (u, v) to p = (u1, u2, v1, v2), Eq. (5)/(6)."""
    u1, u2 = finite_differences(u)
    v1, v2 = finite_differences(v)
    return u1, u2, v1, v2


def finite_differences_adjoint(p1: torch.Tensor, p2: torch.Tensor) -> torch.Tensor:
    """Adjoint of ``finite_differences`` under <a, b> = sum a*b (Sec. II).

    sum_j (u[j]-u[j+1]) p1[j] = sum_j u[j] (p1[j] - p1[j-1]) with p1 = 0 outside
    rows 0..m-2; the same along columns for p2. Shapes: p1 (m-1) x n, p2 m x (n-1).
    """
    # F.pad takes (left, right, top, bottom) for the last two dims.
    down = F.pad(p1, (0, 0, 0, 1)) - F.pad(p1, (0, 0, 1, 0))
    across = F.pad(p2, (0, 1, 0, 0)) - F.pad(p2, (1, 0, 0, 0))
    return down + across


def LT(q):
    """L^T of Prop. 1 for q = (r1, r2, s1, s2): returns the image pair."""
    r1, r2, s1, s2 = q
    return finite_differences_adjoint(r1, r2), finite_differences_adjoint(s1, s2)


def zeros_dual(m: int, n: int):
    return (torch.zeros(m - 1, n, dtype=DT), torch.zeros(m, n - 1, dtype=DT),
            torch.zeros(m - 1, n, dtype=DT), torch.zeros(m, n - 1, dtype=DT))


# --------------------------------------------------------------------------
# TV seminorms, Eq. (3), (4), (7)-(10)
# --------------------------------------------------------------------------
def tv_real_iso(u: torch.Tensor) -> torch.Tensor:
    """Eq. (3): isotropic TV of a real image (interior terms + last column + last row)."""
    u1, u2 = finite_differences(u)
    inner = torch.sqrt(u1[:, :-1] ** 2 + u2[:-1, :] ** 2).sum()
    col = u1[:, -1:].abs().sum()       # j = 1..m-1, k = n
    row = u2[-1:, :].abs().sum()       # j = m, k = 1..n-1
    return inner + col + row


def tv_real_aniso(u: torch.Tensor) -> torch.Tensor:
    """Eq. (4): anisotropic TV of a real image."""
    u1, u2 = finite_differences(u)
    inner = (u1[:, :-1].abs() + u2[:-1, :].abs()).sum()
    col = u1[:, -1:].abs().sum()
    row = u2[-1:, :].abs().sum()
    return inner + col + row


def tv1_iso(u, v, alpha=None):
    """Eq. (7): type-I isotropic complex TV."""
    u1, u2, v1, v2 = L(u, v)
    inner = torch.sqrt(u1[:, :-1] ** 2 + v1[:, :-1] ** 2
                       + u2[:-1, :] ** 2 + v2[:-1, :] ** 2).sum()
    col = torch.sqrt(u1[:, -1:] ** 2 + v1[:, -1:] ** 2).sum()
    row = torch.sqrt(u2[-1:, :] ** 2 + v2[-1:, :] ** 2).sum()
    return inner + col + row


def tv1_aniso(u, v, alpha=None):
    """Eq. (8): type-I anisotropic complex TV."""
    u1, u2, v1, v2 = L(u, v)
    inner = (torch.sqrt(u1[:, :-1] ** 2 + v1[:, :-1] ** 2)
             + torch.sqrt(u2[:-1, :] ** 2 + v2[:-1, :] ** 2)).sum()
    col = torch.sqrt(u1[:, -1:] ** 2 + v1[:, -1:] ** 2).sum()
    row = torch.sqrt(u2[-1:, :] ** 2 + v2[-1:, :] ** 2).sum()
    return inner + col + row


def tv2_iso(u, v, alpha=0.5):
    """Eq. (9): alpha * TVi(Re x) + (1 - alpha) * TVi(Im x)."""
    return alpha * tv_real_iso(u) + (1.0 - alpha) * tv_real_iso(v)


def tv2_aniso(u, v, alpha=0.5):
    """Eq. (10): alpha * TVa(Re x) + (1 - alpha) * TVa(Im x)."""
    return alpha * tv_real_aniso(u) + (1.0 - alpha) * tv_real_aniso(v)


TV = {"tv1_iso": tv1_iso, "tv1_aniso": tv1_aniso, "tv2_iso": tv2_iso, "tv2_aniso": tv2_aniso}


def tv(u, v, tv_type: str, alpha: float = 0.5):
    return TV[tv_type](u, v, alpha)


# --------------------------------------------------------------------------
# Projection onto C, Eq. (25)/(26), plus a support set
# --------------------------------------------------------------------------
@dataclass
class Constraint:
    """The closed convex set C of problem (1) as a product of per-pixel sets.

    amp_max: None for no bound, else |x| <= amp_max (Eq. (25) uses 1).
    box:     None, or (re_lo, re_hi, im_lo, im_hi) bounds on Re x and Im x
             (used without amp_max: each part is then projected independently).
    rect:    None, or (j0, k0, j1, k1): x = 0 outside rows [j0, j1) x cols [k0, k1).
    mask:    None, or a bool m x n tensor: x = 0 where mask is False.
    """
    amp_max: Optional[float] = 1.0
    rect: Optional[Tuple[int, int, int, int]] = None
    mask: Optional[torch.Tensor] = None
    box: Optional[Tuple[float, float, float, float]] = None

    def support(self, m: int, n: int) -> Optional[torch.Tensor]:
        s = None
        if self.rect is not None:
            j0, k0, j1, k1 = self.rect
            s = torch.zeros(m, n, dtype=torch.bool)
            s[max(j0, 0):max(j1, 0), max(k0, 0):max(k1, 0)] = True
        if self.mask is not None:
            s = self.mask.clone() if s is None else (s & self.mask)
        return s


def _scale_into_ball(sq: torch.Tensor, radius: float) -> torch.Tensor:
    """Factor radius / max{radius, sqrt(sq)} used by Eq. (20), (26), (33), (35), (37).

    Written so that autograd stays finite at sq = 0; radius 0 gives 0 (the only
    point of a radius-0 ball)."""
    if radius == 0.0:
        return torch.zeros_like(sq)
    outside = sq > radius * radius
    safe = torch.where(outside, sq, torch.ones_like(sq))
    return torch.where(outside, radius / torch.sqrt(safe), torch.ones_like(sq))


def P_C(u, v, C: Optional[Constraint]):
    """Projection onto C. Eq. (26) scales each pixel by 1/max{1, |x|}; a support
    set zeroes pixels outside it. C is a product of per-pixel closed convex sets
    ({0} or a disk), so applying the per-pixel projections in turn is exact."""
    if C is None:
        return u, v
    if C.amp_max is not None:
        f = _scale_into_ball(u * u + v * v, float(C.amp_max))
        u, v = u * f, v * f
    elif C.box is not None:
        lo_r, hi_r, lo_i, hi_i = (float(t) for t in C.box)
        u, v = torch.clamp(u, lo_r, hi_r), torch.clamp(v, lo_i, hi_i)
    s = C.support(u.shape[0], u.shape[1])
    if s is not None:
        z = torch.zeros_like(u)
        u, v = torch.where(s, u, z), torch.where(s, v, z)
    return u, v


# --------------------------------------------------------------------------
# Projection onto S, Eq. (20), (33), (35), (37)
# --------------------------------------------------------------------------
def P_S_tv1_iso(q, alpha=None):
    """Eq. (20): interior pixels use the joint norm of (r1, r2, s1, s2); the
    last column has only (r1, s1) and the last row only (r2, s2)."""
    r1, r2, s1, s2 = q
    fi = _scale_into_ball(r1[:, :-1] ** 2 + r2[:-1, :] ** 2 + s1[:, :-1] ** 2 + s2[:-1, :] ** 2, 1.0)
    fc = _scale_into_ball(r1[:, -1:] ** 2 + s1[:, -1:] ** 2, 1.0)
    fr = _scale_into_ball(r2[-1:, :] ** 2 + s2[-1:, :] ** 2, 1.0)
    r1n = torch.cat([r1[:, :-1] * fi, r1[:, -1:] * fc], dim=1)
    s1n = torch.cat([s1[:, :-1] * fi, s1[:, -1:] * fc], dim=1)
    r2n = torch.cat([r2[:-1, :] * fi, r2[-1:, :] * fr], dim=0)
    s2n = torch.cat([s2[:-1, :] * fi, s2[-1:, :] * fr], dim=0)
    return r1n, r2n, s1n, s2n


def P_S_tv1_aniso(q, alpha=None):
    """Eq. (33): (r1, s1) and (r2, s2) are scaled into the unit disk separately."""
    r1, r2, s1, s2 = q
    f1 = _scale_into_ball(r1 ** 2 + s1 ** 2, 1.0)
    f2 = _scale_into_ball(r2 ** 2 + s2 ** 2, 1.0)
    return r1 * f1, r2 * f2, s1 * f1, s2 * f2


def _real_iso_ball(a1, a2, radius):
    """Eq. (35) for one of the real/imaginary parts: interior (a1, a2) into the
    ball of the given radius, edge entries into [-radius, radius]."""
    fi = _scale_into_ball(a1[:, :-1] ** 2 + a2[:-1, :] ** 2, radius)
    fc = _scale_into_ball(a1[:, -1:] ** 2, radius)
    fr = _scale_into_ball(a2[-1:, :] ** 2, radius)
    a1n = torch.cat([a1[:, :-1] * fi, a1[:, -1:] * fc], dim=1)
    a2n = torch.cat([a2[:-1, :] * fi, a2[-1:, :] * fr], dim=0)
    return a1n, a2n


def P_S_tv2_iso(q, alpha=0.5):
    """Eq. (35): r into radius alpha, s into radius 1 - alpha."""
    r1, r2, s1, s2 = q
    r1n, r2n = _real_iso_ball(r1, r2, float(alpha))
    s1n, s2n = _real_iso_ball(s1, s2, 1.0 - float(alpha))
    return r1n, r2n, s1n, s2n


def P_S_tv2_aniso(q, alpha=0.5):
    """Eq. (37): every r entry into [-alpha, alpha], every s entry into [-(1-alpha), 1-alpha]."""
    r1, r2, s1, s2 = q
    a, c = float(alpha), 1.0 - float(alpha)
    return (r1 * _scale_into_ball(r1 ** 2, a), r2 * _scale_into_ball(r2 ** 2, a),
            s1 * _scale_into_ball(s1 ** 2, c), s2 * _scale_into_ball(s2 ** 2, c))


P_S = {"tv1_iso": P_S_tv1_iso, "tv1_aniso": P_S_tv1_aniso,
       "tv2_iso": P_S_tv2_iso, "tv2_aniso": P_S_tv2_aniso}


def in_S(q, tv_type: str, alpha: float = 0.5, slack: float = 1e-12) -> bool:
    """Membership in S written from the inequalities (17), (32), (34), (36)."""
    r1, r2, s1, s2 = q
    a, c = alpha, 1.0 - alpha
    ok = True
    if tv_type == "tv1_iso":     # (17)
        ok &= bool(((r1[:, :-1] ** 2 + r2[:-1, :] ** 2 + s1[:, :-1] ** 2 + s2[:-1, :] ** 2) <= 1 + slack).all())
        ok &= bool(((r1[:, -1:] ** 2 + s1[:, -1:] ** 2) <= 1 + slack).all())
        ok &= bool(((r2[-1:, :] ** 2 + s2[-1:, :] ** 2) <= 1 + slack).all())
    elif tv_type == "tv1_aniso":  # (32)
        ok &= bool(((r1 ** 2 + s1 ** 2) <= 1 + slack).all())
        ok &= bool(((r2 ** 2 + s2 ** 2) <= 1 + slack).all())
    elif tv_type == "tv2_iso":    # (34), edge ranges read as j < m-1 / k < n-1
        ok &= bool(((r1[:, :-1] ** 2 + r2[:-1, :] ** 2) <= a * a + slack).all())
        ok &= bool((r1[:, -1:].abs() <= a + slack).all()) and bool((r2[-1:, :].abs() <= a + slack).all())
        ok &= bool(((s1[:, :-1] ** 2 + s2[:-1, :] ** 2) <= c * c + slack).all())
        ok &= bool((s1[:, -1:].abs() <= c + slack).all()) and bool((s2[-1:, :].abs() <= c + slack).all())
    elif tv_type == "tv2_aniso":  # (36)
        ok &= bool((r1.abs() <= a + slack).all()) and bool((r2.abs() <= a + slack).all())
        ok &= bool((s1.abs() <= c + slack).all()) and bool((s2.abs() <= c + slack).all())
    else:
        raise ValueError(tv_type)
    return ok


def dual_inner(p, q) -> torch.Tensor:
    return sum((a * b).sum() for a, b in zip(p, q))


def pair_inner(x, y) -> torch.Tensor:
    return (x[0] * y[0]).sum() + (x[1] * y[1]).sum()
