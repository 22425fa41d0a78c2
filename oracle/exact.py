"""Small independent solvers that pin the oracle (numpy, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/ops.py``).

None of these reuses ``ops``/``fgp``: they restate the model from the paper in
a different form, so a mistake in the vectorised oracle (a dropped edge term,
a wrong sign, a transposed index) shows up as a disagreement.

* ``tv_terms``      TV of Eq. (3), (4), (7)-(10) built term by term with loops.
* ``projected_subgradient``  a primal solver of problem (1) that never touches
                    the dual set S.
* ``tv1d_exact``    exact 1-D TV denoising by enumerating the dual active sets.
* ``two_pixel``     closed form of problem (1) on a 1 x 2 image with C = C^{1x2}.
* ``real_fgp``      the real-valued FGP of Beck and Teboulle (their notation:
                    L(p, q) a divergence on zero-padded arrays), used to check
                    the complex oracle on real or imaginary input.
"""
from __future__ import annotations

import itertools
import math
from typing import List, Optional, Tuple

import numpy as np


# --------------------------------------------------------------------------
# TV as an explicit list of norm terms
# --------------------------------------------------------------------------
def _idx(j, k, n, part, m):
    """Column of u[j,k] (part 0) or v[j,k] (part 1) in the stacked vector [u; v]."""
    return part * m * n + j * n + k


def tv_terms(m: int, n: int, tv_type: str, alpha: float = 0.5):
    """Return (A, groups, weights) with TV(x) = sum_g weights[g] * ||A[groups[g]] @ xvec||_2.

    xvec = [u.ravel(); v.ravel()]. Each row of A is one finite difference
    (u or v, vertical or horizontal); each group is the set of differences
    under one square root (or absolute value) of Eq. (3), (4), (7)-(10)."""
    rows: List[np.ndarray] = []
    groups: List[List[int]] = []
    weights: List[float] = []

    def diff_row(part, j, k, vertical):
        a = np.zeros(2 * m * n)
        a[_idx(j, k, n, part, m)] = 1.0
        if vertical:
            a[_idx(j + 1, k, n, part, m)] = -1.0
        else:
            a[_idx(j, k + 1, n, part, m)] = -1.0
        return a

    def add(group_rows, w):
        ids = []
        for r in group_rows:
            rows.append(r)
            ids.append(len(rows) - 1)
        groups.append(ids)
        weights.append(w)

    for j in range(m):
        for k in range(n):
            has_v = j < m - 1   # vertical difference exists
            has_h = k < n - 1   # horizontal difference exists
            if not (has_v or has_h):
                continue
            if tv_type == "tv1_iso":
                g = []
                if has_v:
                    g += [diff_row(0, j, k, True), diff_row(1, j, k, True)]
                if has_h:
                    g += [diff_row(0, j, k, False), diff_row(1, j, k, False)]
                add(g, 1.0)
            elif tv_type == "tv1_aniso":
                if has_v:
                    add([diff_row(0, j, k, True), diff_row(1, j, k, True)], 1.0)
                if has_h:
                    add([diff_row(0, j, k, False), diff_row(1, j, k, False)], 1.0)
            elif tv_type == "tv2_iso":
                for part, w in ((0, alpha), (1, 1.0 - alpha)):
                    g = []
                    if has_v:
                        g.append(diff_row(part, j, k, True))
                    if has_h:
                        g.append(diff_row(part, j, k, False))
                    add(g, w)
            elif tv_type == "tv2_aniso":
                for part, w in ((0, alpha), (1, 1.0 - alpha)):
                    if has_v:
                        add([diff_row(part, j, k, True)], w)
                    if has_h:
                        add([diff_row(part, j, k, False)], w)
            else:
                raise ValueError(tv_type)
    A = np.array(rows) if rows else np.zeros((0, 2 * m * n))
    return A, groups, np.array(weights)


def tv_value_terms(u: np.ndarray, v: np.ndarray, terms) -> float:
    A, groups, w = terms
    d = A @ np.concatenate([u.ravel(), v.ravel()])
    return float(sum(wi * math.sqrt(sum(d[i] ** 2 for i in g)) for g, wi in zip(groups, w)))


def _project_C(xu, xv, amp_max, support, box=None):
    if amp_max is not None:
        a = np.sqrt(xu * xu + xv * xv)
        f = amp_max / np.maximum(amp_max, a)
        xu, xv = xu * f, xv * f
    elif box is not None:
        xu, xv = np.clip(xu, box[0], box[1]), np.clip(xv, box[2], box[3])
    if support is not None:
        xu, xv = xu * support, xv * support
    return xu, xv


def projected_subgradient(bu, bv, lam, terms, amp_max=None, support=None,
                          iters=200000, step0=None, box=None):
    """Minimise 1/2||x - b||^2 + lam TV(x) over C with a projected subgradient
    method (steps c/sqrt(k)), returning the best iterate found. Uses only the
    term-list TV and the projection onto C."""
    m, n = bu.shape
    A, groups, w = terms
    ng = len(groups)
    # group id of every row, for a vectorised subgradient
    gid = np.zeros(A.shape[0], dtype=int)
    for g, ids in enumerate(groups):
        gid[ids] = g
    wrow = w[gid]
    b = np.concatenate([bu.ravel(), bv.ravel()])
    sup = None if support is None else np.concatenate([support.ravel(), support.ravel()]).astype(float)

    def proj(x):
        xu, xv = x[: m * n].reshape(m, n), x[m * n:].reshape(m, n)
        pu, pv = _project_C(xu, xv, amp_max, None if sup is None else support.astype(float), box)
        return np.concatenate([pu.ravel(), pv.ravel()])

    def obj(x):
        d = A @ x
        gn = np.sqrt(np.bincount(gid, weights=d * d, minlength=ng))
        return 0.5 * float(((x - b) ** 2).sum()) + lam * float((w * gn).sum())

    x = proj(b.copy())
    best, best_x = obj(x), x.copy()
    step0 = step0 if step0 is not None else 0.5
    for k in range(1, iters + 1):
        d = A @ x
        gn = np.sqrt(np.bincount(gid, weights=d * d, minlength=ng))
        safe = np.where(gn[gid] > 0, gn[gid], 1.0)
        sub = A.T @ (wrow * np.where(gn[gid] > 0, d / safe, 0.0))
        gvec = (x - b) + lam * sub
        x = proj(x - (step0 / math.sqrt(k)) * gvec)
        if k % 50 == 0 or k == iters:
            f = obj(x)
            if f < best:
                best, best_x = f, x.copy()
    return best_x[: m * n].reshape(m, n), best_x[m * n:].reshape(m, n), best


# --------------------------------------------------------------------------
# Exact 1-D TV denoising (real, unconstrained) by active-set enumeration
# --------------------------------------------------------------------------
def tv1d_exact(b: np.ndarray, lam: float) -> np.ndarray:
    """argmin_x 1/2||x - b||^2 + lam sum_j |x_j - x_{j+1}| for a short real vector.

    Dual: min_{|p_j| <= 1} 1/2||b - lam D^T p||^2. For every assignment of each
    p_j to -1, +1 or free, solve the free part exactly and keep the assignment
    that satisfies the KKT conditions; x = b - lam D^T p is then the unique
    primal minimiser."""
    m = len(b)
    if m < 2 or lam == 0:
        return b.copy()
    Dm = np.zeros((m - 1, m))
    for j in range(m - 1):
        Dm[j, j], Dm[j, j + 1] = 1.0, -1.0
    best = None
    for pattern in itertools.product((-1, 0, 1), repeat=m - 1):
        pat = np.array(pattern)
        free = np.where(pat == 0)[0]
        p = pat.astype(float)
        if len(free):
            act = np.where(pat != 0)[0]
            # stationarity on the free coordinates: D_F (b - lam D^T p) = 0
            rhs = Dm[free] @ (b - lam * Dm[act].T @ p[act])
            Mf = lam * Dm[free] @ Dm[free].T
            try:
                p[free] = np.linalg.solve(Mf, rhs)
            except np.linalg.LinAlgError:
                continue
            if np.any(np.abs(p[free]) > 1 + 1e-12):
                continue
        x = b - lam * Dm.T @ p
        grad = -lam * (Dm @ x)          # gradient of the dual objective in p
        # KKT for the box: at p = +1 the gradient must be <= 0, at -1 >= 0
        ok = True
        for j in range(m - 1):
            if pat[j] == 1 and grad[j] > 1e-10:
                ok = False
            if pat[j] == -1 and grad[j] < -1e-10:
                ok = False
        if ok:
            best = x
            break
    if best is None:
        raise RuntimeError("no KKT point found")
    return best


# --------------------------------------------------------------------------
# Two-pixel closed form
# --------------------------------------------------------------------------
def two_pixel(b1: complex, b2: complex, lam: float, tv_type: str, alpha: float = 0.5):
    """Minimiser of 1/2|x1-b1|^2 + 1/2|x2-b2|^2 + lam TV for two neighbouring pixels.

    With s = x1 + x2 and e = x1 - x2 the objective splits into |s - (b1+b2)|^2/4
    (so s = b1 + b2) and |e - d|^2/4 + lam TV(e), d = b1 - b2. Type I: TV(e) = |e|
    (complex modulus) and e = d max(0, 1 - 2 lam/|d|). Type II: TV(e) =
    alpha |Re e| + (1-alpha)|Im e|, a soft threshold of each part."""
    d = b1 - b2
    s = b1 + b2
    if tv_type.startswith("tv1"):
        a = abs(d)
        e = 0.0 if a <= 2 * lam else d * (1 - 2 * lam / a)
    else:
        def soft(z, t):
            return math.copysign(max(abs(z) - t, 0.0), z)
        e = complex(soft(d.real, 2 * lam * alpha), soft(d.imag, 2 * lam * (1 - alpha)))
    return (s + e) / 2, (s - e) / 2


# --------------------------------------------------------------------------
# Real FGP of Beck & Teboulle (zero-padded m x n arrays, divergence notation)
# --------------------------------------------------------------------------
def real_fgp(b: np.ndarray, lam: float, K: int, iso: bool, lo=-np.inf, hi=np.inf):
    """Real constrained TV denoising by FGP on zero-padded dual arrays p, q.

    Div(p, q)[i,j] = p[i,j] + q[i,j] - p[i-1,j] - q[i,j-1] with p[m-1,:] = 0 and
    q[:, n-1] = 0 (the padded slots); Grad x = (x[i]-x[i+1], x[j]-x[j+1]).
    Returns (x, p, q) after K iterations; the dual pair is m x n each."""
    m, n = b.shape

    def div(p, q):
        out = p + q
        out[1:, :] -= p[:-1, :]
        out[:, 1:] -= q[:, :-1]
        return out

    def grad(x):
        gp = np.zeros_like(x)
        gq = np.zeros_like(x)
        gp[:-1, :] = x[:-1, :] - x[1:, :]
        gq[:, :-1] = x[:, :-1] - x[:, 1:]
        return gp, gq

    def proj_box(x):
        return np.clip(x, lo, hi)

    def proj_dual(p, q):
        if iso:
            nr = np.maximum(1.0, np.sqrt(p * p + q * q))
            return p / nr, q / nr
        return p / np.maximum(1.0, np.abs(p)), q / np.maximum(1.0, np.abs(q))

    p_old = np.zeros((m, n))
    q_old = np.zeros((m, n))
    rp, rq = p_old.copy(), q_old.copy()
    t = 1.0
    for _ in range(K):
        x = proj_box(b - lam * div(rp, rq))
        gp, gq = grad(x)
        p, q = proj_dual(rp + gp / (8 * lam), rq + gq / (8 * lam))
        t_new = (1 + math.sqrt(1 + 4 * t * t)) / 2
        c = (t - 1) / t_new
        rp, rq = p + c * (p - p_old), q + c * (q - q_old)
        p_old, q_old, t = p, q, t_new
    x = proj_box(b - lam * div(p_old, q_old))
    return x, p_old, q_old


def norm_D_squared(m: int, n: int, iters: int = 500, seed: int = 0) -> float:
    """Largest eigenvalue of D^T D for one real m x n image, by power iteration,
    with D written as explicit stencils (no use of ``ops``)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((m, n))
    lam = 0.0
    for _ in range(iters):
        gp = np.zeros((m, n)); gq = np.zeros((m, n))
        gp[:-1, :] = x[:-1, :] - x[1:, :]
        gq[:, :-1] = x[:, :-1] - x[:, 1:]
        y = gp + gq
        y[1:, :] -= gp[:-1, :]
        y[:, 1:] -= gq[:, :-1]
        lam = float(np.linalg.norm(y) / np.linalg.norm(x))
        x = y / np.linalg.norm(y)
    return lam
