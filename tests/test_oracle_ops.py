"""Pins for the oracle's operators: adjointness and ||D||^2 <= 8 (Sec. IV-B),
TV against a term-by-term restatement of Eq. (3), (4), (7)-(10), and the
projections P_C (Eq. (26)) and P_S (Eq. (20), (33), (35), (37)) against the
sets they project onto."""
import math

import numpy as np
import pytest
import torch

from oracle import exact
from oracle.ops import (DT, LT, L, P_C, P_S, TV_TYPES, Constraint, dual_inner, in_S,
                        pair_inner, tv, tv_real_aniso, tv_real_iso)

SHAPES = [(1, 1), (1, 5), (5, 1), (2, 2), (3, 5), (6, 4), (7, 7)]


def rand_pair(m, n, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (scale * torch.randn(m, n, generator=g, dtype=DT),
            scale * torch.randn(m, n, generator=g, dtype=DT))


def rand_dual(m, n, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return tuple(scale * torch.randn(*s, generator=g, dtype=DT)
                 for s in [(m - 1, n), (m, n - 1), (m - 1, n), (m, n - 1)])


@pytest.mark.parametrize("m,n", SHAPES)
def test_adjointness(m, n):
    x = rand_pair(m, n, 1)
    q = rand_dual(m, n, 2)
    lhs = dual_inner(L(*x), q)
    rhs = pair_inner(x, LT(q))
    assert abs(float(lhs - rhs)) <= 1e-13 * max(1.0, abs(float(lhs)))


def test_adjoint_explicit_stencil():
    # (L^T p)[j,k] = p1[j,k] - p1[j-1,k] + p2[j,k] - p2[j,k-1], zero outside the paper's ranges
    m, n = 4, 5
    q = rand_dual(m, n, 3)
    out = LT(q)[0]
    r1, r2 = q[0], q[1]
    for j in range(m):
        for k in range(n):
            want = 0.0
            if j < m - 1:
                want += r1[j, k]
            if j >= 1:
                want -= r1[j - 1, k]
            if k < n - 1:
                want += r2[j, k]
            if k >= 1:
                want -= r2[j, k - 1]
            assert abs(float(out[j, k]) - float(want)) < 1e-14


def test_norm_D_bound():
    # ||D||^2 = ||D^T D|| <= 8 for one real image (Sec. IV-B: Lipschitz 16 lam^2 = 2 lam^2 * 8)
    for m, n in [(8, 8), (32, 32), (5, 9)]:
        val = exact.norm_D_squared(m, n, iters=2000)
        assert val <= 8.0 + 1e-9
    assert exact.norm_D_squared(64, 64, iters=3000) > 7.9


@pytest.mark.parametrize("tv_type", TV_TYPES)
@pytest.mark.parametrize("m,n", SHAPES)
def test_tv_matches_term_list(tv_type, m, n):
    u, v = rand_pair(m, n, 11)
    alpha = 0.3
    got = float(tv(u, v, tv_type, alpha))
    want = exact.tv_value_terms(u.numpy(), v.numpy(), exact.tv_terms(m, n, tv_type, alpha))
    assert got == pytest.approx(want, rel=1e-13, abs=1e-13)


def test_tv_real_reductions():
    # Eq. (7)/(8) on a real image reduce to Eq. (3)/(4); Eq. (9)/(10) with alpha=1 too
    u, _ = rand_pair(6, 7, 5)
    z = torch.zeros_like(u)
    assert float(tv(u, z, "tv1_iso")) == pytest.approx(float(tv_real_iso(u)), rel=1e-14)
    assert float(tv(u, z, "tv1_aniso")) == pytest.approx(float(tv_real_aniso(u)), rel=1e-14)
    assert float(tv(u, z, "tv2_iso", 1.0)) == pytest.approx(float(tv_real_iso(u)), rel=1e-14)
    assert float(tv(z, u, "tv2_aniso", 0.0)) == pytest.approx(float(tv_real_aniso(u)), rel=1e-14)
    # a constant image has zero TV for every type
    c = torch.full((4, 4), 0.7, dtype=DT)
    for t in TV_TYPES:
        assert float(tv(c, -c, t)) == 0.0


def test_tv_isotropic_not_above_anisotropic():
    u, v = rand_pair(9, 9, 8)
    assert float(tv(u, v, "tv1_iso")) <= float(tv(u, v, "tv1_aniso")) + 1e-12
    assert float(tv(u, v, "tv2_iso")) <= float(tv(u, v, "tv2_aniso")) + 1e-12


def _scale_into_S(q, tv_type, alpha):
    """A point of S built without P_S: shrink q by a common factor until it is in S."""
    lo, hi = 0.0, 1.0
    if in_S(q, tv_type, alpha, slack=0.0):
        return q
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if in_S(tuple(mid * t for t in q), tv_type, alpha, slack=0.0):
            lo = mid
        else:
            hi = mid
    return tuple(lo * t for t in q)


@pytest.mark.parametrize("tv_type", TV_TYPES)
@pytest.mark.parametrize("m,n", [(1, 4), (4, 1), (3, 3), (5, 6)])
@pytest.mark.parametrize("alpha", [0.5, 0.2])
def test_P_S_is_the_projection(tv_type, m, n, alpha):
    proj = P_S[tv_type]
    for seed in range(4):
        z = rand_dual(m, n, 100 + seed, scale=2.0)
        pz = proj(z, alpha)
        assert in_S(pz, tv_type, alpha)
        # idempotent
        ppz = proj(pz, alpha)
        for a, b in zip(pz, ppz):
            assert torch.allclose(a, b, atol=1e-15)
        # variational inequality <z - P z, y - P z> <= 0 for points y of S
        for s2 in range(6):
            y = _scale_into_S(rand_dual(m, n, 500 + 10 * seed + s2, scale=1.5), tv_type, alpha)
            vi = dual_inner(tuple(a - b for a, b in zip(z, pz)), tuple(a - b for a, b in zip(y, pz)))
            assert float(vi) <= 1e-12


def test_P_S_alpha_edges():
    # alpha = 1: s is projected onto the radius-0 ball (reading of Eq. (35)/(37) at alpha in {0, 1})
    q = rand_dual(3, 4, 9, scale=2.0)
    for t in ("tv2_iso", "tv2_aniso"):
        r1, r2, s1, s2 = P_S[t](q, 1.0)
        assert float(s1.abs().max()) == 0.0 and float(s2.abs().max()) == 0.0
        r1, r2, s1, s2 = P_S[t](q, 0.0)
        assert float(r1.abs().max()) == 0.0 and float(r2.abs().max()) == 0.0


def test_P_C_projection():
    m, n = 6, 7
    C = Constraint(amp_max=1.0, rect=(1, 2, 5, 6))
    sup = C.support(m, n)
    for seed in range(4):
        z = rand_pair(m, n, 40 + seed, scale=1.5)
        p = P_C(*z, C)
        amp = torch.sqrt(p[0] ** 2 + p[1] ** 2)
        assert float(amp.max()) <= 1 + 1e-15
        assert float(p[0][~sup].abs().max()) == 0.0
        # Eq. (26) inside the support: x / max{1, |x|}
        a = torch.sqrt(z[0] ** 2 + z[1] ** 2)
        want = z[0] / torch.clamp(a, min=1.0)
        assert torch.allclose(p[0][sup], want[sup], atol=1e-15)
        pp = P_C(*p, C)
        assert torch.allclose(pp[0], p[0]) and torch.allclose(pp[1], p[1])
        for s2 in range(5):
            y = rand_pair(m, n, 900 + s2)
            ya = torch.sqrt(y[0] ** 2 + y[1] ** 2)
            f = torch.where(ya > 1, 1 / ya, torch.ones_like(ya)) * sup
            y = (y[0] * f, y[1] * f)
            vi = pair_inner((z[0] - p[0], z[1] - p[1]), (y[0] - p[0], y[1] - p[1]))
            assert float(vi) <= 1e-12
    # amp_max other than 1
    z = rand_pair(3, 3, 77, scale=3.0)
    p = P_C(*z, Constraint(amp_max=0.5))
    assert float(torch.sqrt(p[0] ** 2 + p[1] ** 2).max()) <= 0.5 + 1e-15


def test_P_C_box():
    # the box of the real and imaginary parts: componentwise clamps, in the set,
    # idempotent and satisfying the variational inequality
    m, n = 5, 6
    box = (-0.4, 0.7, -0.2, 0.5)
    C = Constraint(amp_max=None, box=box)
    for seed in range(3):
        z = rand_pair(m, n, 60 + seed, scale=1.2)
        p = P_C(*z, C)
        assert float(p[0].min()) >= box[0] and float(p[0].max()) <= box[1]
        assert float(p[1].min()) >= box[2] and float(p[1].max()) <= box[3]
        pp = P_C(*p, C)
        assert torch.equal(pp[0], p[0]) and torch.equal(pp[1], p[1])
        for s2 in range(4):
            y = rand_pair(m, n, 700 + s2)
            y = (torch.clamp(y[0], box[0], box[1]), torch.clamp(y[1], box[2], box[3]))
            vi = pair_inner((z[0] - p[0], z[1] - p[1]), (y[0] - p[0], y[1] - p[1]))
            assert float(vi) <= 1e-12
