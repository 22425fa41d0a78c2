"""Pins for the oracle's FGP (Algorithm 2), GP (Eq. (21)) and duality gap (App. A).

Closed forms (constant b, lam = 0, large lam, two pixels), reductions (real or
imaginary b against the real FGP of Beck and Teboulle; 1-D against an exact
active-set solver), certificates on 4 x 4 and 8 x 8 (gap -> 0 with q in S,
agreement with a projected-subgradient primal solver) and the monotone dual of
plain GP."""
import math

import numpy as np
import pytest
import torch

from oracle import exact
from oracle.fgp import dual_value, fgp, primal_value
from oracle.ops import DT, P_C, TV_TYPES, Constraint, in_S, tv
from phantoms import noisy_phantom, support_rect


def pair(z):
    z = torch.as_tensor(np.asarray(z, dtype=np.complex128))
    return (z.real.clone(), z.imag.clone())


def rand_complex(m, n, seed, scale=0.6):
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))


CONSTRAINTS = {
    "none": None,
    "amp": Constraint(amp_max=1.0),
    "amp_rect": Constraint(amp_max=1.0, rect=(1, 1, 6, 7)),
}


# ---------------------------------------------------------------- P1, P2
@pytest.mark.parametrize("tv_type", TV_TYPES)
def test_constant_image(tv_type):
    b = pair(np.full((5, 6), 1.3 * np.exp(0.4j)))
    C = Constraint(amp_max=1.0)
    res = fgp(b, 0.2, 25, tv_type, 0.5, C)
    pc = P_C(*b, C)
    assert torch.equal(res.x[0], pc[0]) and torch.equal(res.x[1], pc[1])
    for t in res.q:
        assert float(t.abs().max()) == 0.0
    assert float(tv(*res.x, tv_type)) == 0.0


@pytest.mark.parametrize("tv_type", TV_TYPES)
def test_lambda_zero(tv_type):
    b = pair(rand_complex(4, 5, 3, 1.0))
    C = Constraint(amp_max=1.0, rect=(0, 1, 3, 5))
    res = fgp(b, 0.0, 10, tv_type, 0.5, C)
    pc = P_C(*b, C)
    assert torch.equal(res.x[0], pc[0]) and torch.equal(res.x[1], pc[1])


# ---------------------------------------------------------------- P3
@pytest.mark.parametrize("tv_type", TV_TYPES)
def test_large_lambda_gives_constant(tv_type):
    # for lam above a finite threshold the minimiser is the constant c = P_disk(mean b)
    bz = rand_complex(6, 6, 21, 0.5) + 0.3
    b = pair(bz)
    C = Constraint(amp_max=1.0)
    res = fgp(b, 4.0, 6000, tv_type, 0.5, C, check_every=500)
    mean = bz.mean()
    c = mean / max(1.0, abs(mean))
    assert np.max(np.abs(res.x[0].numpy() - c.real)) < 2e-5
    assert np.max(np.abs(res.x[1].numpy() - c.imag)) < 2e-5


# ---------------------------------------------------------------- P4
@pytest.mark.parametrize("iso", [True, False])
def test_real_input_matches_real_fgp(iso):
    rng = np.random.default_rng(5)
    bre = rng.uniform(-1.5, 1.5, (7, 9))
    lam, K = 0.15, 30
    C = Constraint(amp_max=1.0)
    t1 = "tv1_iso" if iso else "tv1_aniso"
    res = fgp((torch.tensor(bre), torch.zeros(7, 9, dtype=DT)), lam, K, t1, 0.5, C)
    x_ref, p_ref, q_ref = exact.real_fgp(bre, lam, K, iso, -1.0, 1.0)
    assert float(res.x[1].abs().max()) == 0.0            # s stays 0, x stays real
    assert float(res.q[2].abs().max()) == 0.0 and float(res.q[3].abs().max()) == 0.0
    assert np.max(np.abs(res.x[0].numpy() - x_ref)) < 1e-12
    assert np.max(np.abs(res.q[0].numpy() - p_ref[:-1, :])) < 1e-12
    assert np.max(np.abs(res.q[1].numpy() - q_ref[:, :-1])) < 1e-12
    # type II: the real part sees lam * alpha, with r = alpha * r'
    alpha = 0.3
    t2 = "tv2_iso" if iso else "tv2_aniso"
    res2 = fgp((torch.tensor(bre), torch.zeros(7, 9, dtype=DT)), lam, K, t2, alpha, C)
    x2, p2, _ = exact.real_fgp(bre, lam * alpha, K, iso, -1.0, 1.0)
    assert np.max(np.abs(res2.x[0].numpy() - x2)) < 1e-12
    assert np.max(np.abs(res2.q[0].numpy() - alpha * p2[:-1, :])) < 1e-12
    # purely imaginary input under type II sees lam * (1 - alpha)
    res3 = fgp((torch.zeros(7, 9, dtype=DT), torch.tensor(bre)), lam, K, t2, alpha, C)
    x3, _, _ = exact.real_fgp(bre, lam * (1 - alpha), K, iso, -1.0, 1.0)
    assert float(res3.x[0].abs().max()) == 0.0
    assert np.max(np.abs(res3.x[1].numpy() - x3)) < 1e-12


# ---------------------------------------------------------------- P5
@pytest.mark.parametrize("tv_type", TV_TYPES)
@pytest.mark.parametrize("shape", [(1, 2), (2, 1)])
@pytest.mark.parametrize("b1,b2,lam", [(0.3 + 0.2j, -0.1 + 0.4j, 0.05),   # |d| > 2 lam: split
                                      (0.3 + 0.2j, 0.25 + 0.1j, 0.2)])    # |d| <= 2 lam: merge
def test_two_pixel_closed_form(tv_type, shape, b1, b2, lam):
    alpha = 0.4
    b = np.array([b1, b2]).reshape(shape)
    res = fgp(pair(b), lam, 3000, tv_type, alpha, None)
    x1, x2 = exact.two_pixel(b1, b2, lam, tv_type, alpha)
    got = (res.x[0] + 1j * res.x[1]).numpy().ravel()
    assert abs(got[0] - x1) < 1e-9 and abs(got[1] - x2) < 1e-9


# ---------------------------------------------------------------- P6
@pytest.mark.parametrize("m", [2, 5, 7])
@pytest.mark.parametrize("tv_type", ["tv1_iso", "tv1_aniso"])
def test_1d_exact(m, tv_type):
    rng = np.random.default_rng(m)
    bre = rng.uniform(-1, 1, m)
    lam = 0.12
    want = exact.tv1d_exact(bre, lam)
    res = fgp((torch.tensor(bre).reshape(m, 1), torch.zeros(m, 1, dtype=DT)), lam, 4000, tv_type)
    assert np.max(np.abs(res.x[0].numpy().ravel() - want)) < 1e-8
    # the same problem laid out as a 1 x m row
    res = fgp((torch.tensor(bre).reshape(1, m), torch.zeros(1, m, dtype=DT)), lam, 4000, tv_type)
    assert np.max(np.abs(res.x[0].numpy().ravel() - want)) < 1e-8


# ---------------------------------------------------------------- P7
@pytest.mark.parametrize("tv_type", TV_TYPES)
@pytest.mark.parametrize("cname", list(CONSTRAINTS))
def test_certificate_and_primal_solver(tv_type, cname):
    m, n = 4, 5
    C = CONSTRAINTS[cname]
    if C is not None and C.rect is not None:
        C = Constraint(amp_max=1.0, rect=(1, 1, 4, 4))
    bz = rand_complex(m, n, 31, 0.8)
    b = pair(bz)
    lam, alpha = 0.12, 0.35
    res = fgp(b, lam, 6000, tv_type, alpha, C)
    assert in_S(res.q, tv_type, alpha, slack=1e-12)
    P = float(primal_value(res.x, b, lam, tv_type, alpha))
    D = float(dual_value(res.q, b, lam, C))
    assert P - D >= -1e-12 * P               # weak duality
    assert P - D <= 1e-9 * P                 # certificate: x is optimal to 1e-9
    # an independent primal solver (projected subgradient, term-list TV, no S)
    terms = exact.tv_terms(m, n, tv_type, alpha)
    sup = None if C is None or C.rect is None else C.support(m, n).numpy()
    amp = None if C is None else C.amp_max
    su, sv, best = exact.projected_subgradient(bz.real, bz.imag, lam, terms, amp, sup, iters=40000)
    assert best >= P - 1e-9 * P
    assert best - P <= 2e-4 * P
    # strong convexity: ||x_sub - x*||^2 <= 2 (P(x_sub) - P*)
    dist2 = float(((res.x[0].numpy() - su) ** 2 + (res.x[1].numpy() - sv) ** 2).sum())
    assert dist2 <= 2 * (best - P) + 1e-9


# ---------------------------------------------------------------- gap behaviour
@pytest.mark.parametrize("tv_type", TV_TYPES)
def test_gap_nonnegative_and_rate(tv_type):
    clean, noisy = noisy_phantom(24, 20, 0.1, seed=4)
    b = pair(noisy)
    C = Constraint(amp_max=1.0, rect=support_rect(24, 20))
    lam = 0.05
    res = fgp(b, lam, 300, tv_type, 0.5, C, check_every=10)
    gaps = [h["gap"] for h in res.history]
    P0 = res.history[0]["primal"]
    assert all(g >= -1e-12 * P0 for g in gaps)
    # running minimum of the gap goes to zero
    assert min(gaps) < 1e-4 * P0
    assert min(gaps[-5:]) <= min(gaps[:5])


@pytest.mark.parametrize("tv_type", TV_TYPES)
def test_gp_dual_monotone(tv_type):
    # plain gradient projection (21) with step 1/(16 lam^2) never decreases the dual value
    _, noisy = noisy_phantom(12, 10, 0.2, seed=9)
    b = pair(noisy)
    C = Constraint(amp_max=1.0)
    lam = 0.1
    res = fgp(b, lam, 200, tv_type, 0.5, C, accelerate=False, check_every=1)
    d = [h["dual"] for h in res.history]
    assert all(d[i + 1] >= d[i] - 1e-12 * abs(d[i]) for i in range(len(d) - 1))
    # and FGP reaches a smaller gap than GP after the same number of iterations
    res_f = fgp(b, lam, 200, tv_type, 0.5, C, check_every=200)
    assert res_f.history[-1]["gap"] <= res.history[-1]["gap"] * 1.0001


def test_gap_stopping():
    _, noisy = noisy_phantom(16, 16, 0.1, seed=2)
    b = pair(noisy)
    res = fgp(b, 0.05, 500, "tv1_iso", 0.5, Constraint(amp_max=1.0), check_every=10, gap_tol=1e-6)
    assert res.iters < 500 and res.iters % 10 == 0
    h = res.history[-1]
    assert h["gap"] <= 1e-6 * h["primal"]
    assert all(x["gap"] > 1e-6 * x["primal"] for x in res.history[:-1])


def test_warm_start_fixed_point():
    # starting from a converged dual leaves x unchanged
    _, noisy = noisy_phantom(10, 12, 0.1, seed=6)
    b = pair(noisy)
    C = Constraint(amp_max=1.0)
    res = fgp(b, 0.05, 3000, "tv1_aniso", 0.5, C)
    res2 = fgp(b, 0.05, 5, "tv1_aniso", 0.5, C, q0=res.q)
    assert max(float((res2.x[0] - res.x[0]).abs().max()), float((res2.x[1] - res.x[1]).abs().max())) < 1e-6


@pytest.mark.parametrize("tv_type", TV_TYPES)
def test_certificate_box_constraint(tv_type):
    # box on the real and imaginary parts (with a support): gap certificate and the
    # independent primal solver agree
    m, n = 4, 5
    box = (-0.3, 0.6, -0.5, 0.2)
    C = Constraint(amp_max=None, box=box, rect=(0, 1, 4, 5))
    bz = rand_complex(m, n, 41, 0.8)
    b = pair(bz)
    lam, alpha = 0.1, 0.4
    res = fgp(b, lam, 6000, tv_type, alpha, C)
    P = float(primal_value(res.x, b, lam, tv_type, alpha))
    D = float(dual_value(res.q, b, lam, C))
    assert -1e-12 * P <= P - D <= 1e-9 * P
    terms = exact.tv_terms(m, n, tv_type, alpha)
    su, sv, best = exact.projected_subgradient(bz.real, bz.imag, lam, terms, None, C.support(m, n).numpy(),
                                               iters=40000, box=box)
    assert P - 1e-9 * P <= best <= P + 2e-4 * P
