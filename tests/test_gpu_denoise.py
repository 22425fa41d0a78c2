"""GPU parity of the fused FGP path (ctv_denoise / ctv_denoise_batched) against
the FP64 oracle, element by element, after the same number of iterations.

Bar (for every floating-point result): max|x_gpu - x_oracle| <= 1e-4 ||b||_inf and
|P(x_gpu) - P(x_oracle)| <= 1e-6 P(x_oracle), P evaluated in FP64 by the oracle."""
import math

import numpy as np
import pytest
import torch

import paper_2109_05496_gb300 as ctv
from paper_2109_05496_gb300 import build as ctv_build
from oracle.fgp import dual_value, primal_value
from oracle.ops import in_S, P_C as oracle_PC
from phantoms import noisy_phantom, phantom, support_rect, to_c64
from tests.helpers import (TV_NAMES, dual_from_paper, dual_to_paper, f32, objective, oracle_constraint,
                           padded_slots_zero, run_oracle)

pytestmark = pytest.mark.gpu

XTOL = 1e-4
OBJTOL = 1e-6
CONFIGS = [row[0] for row in ctv_build.config_table()]


def cons_pair(kind, m, n, seed=0):
    """(library constraint, oracle constraint) of one kind."""
    if kind == "none":
        return ctv.NO_CONSTRAINT, None
    if kind == "amp":
        return ctv.Constraint(amp_max=1.0), oracle_constraint(1.0)
    if kind == "amp_rect":
        r = support_rect(m, n)
        return ctv.Constraint(amp_max=1.0, rect=r), oracle_constraint(1.0, rect=r)
    if kind == "amp_mask":
        rng = np.random.default_rng(seed)
        mk = rng.uniform(size=(m, n)) < 0.8
        return (ctv.Constraint(amp_max=1.0, mask=torch.from_numpy(mk.astype(np.uint8)).cuda()),
                oracle_constraint(1.0, mask=mk))
    raise ValueError(kind)


def gpu_denoise(b_np, lam, K, tv, alpha, C, config=-1, **kw):
    b = torch.from_numpy(to_c64(b_np)).cuda()
    x, st = ctv.denoise(b, lam, tv, K, C, alpha, return_stats=True, config=config, **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy(), st


def check_parity(x_gpu, res, b_pair, b_np, lam, tv, alpha):
    xo = (res.x[0] + 1j * res.x[1]).numpy()
    binf = float(np.abs(to_c64(b_np)).max())
    err = float(np.max(np.abs(x_gpu.astype(np.complex128) - xo))) if xo.size else 0.0
    assert err <= XTOL * max(binf, 1e-30), "max|dx| = %g > %g" % (err, XTOL * binf)
    Pg = objective(x_gpu, b_pair, lam, tv, alpha)
    Po = objective(xo, b_pair, lam, tv, alpha)
    assert abs(Pg - Po) <= OBJTOL * abs(Po) + 1e-300, "objective %r vs %r" % (Pg, Po)
    return err


# --------------------------------------------------------------- C1: 256^2, 100 iterations
@pytest.mark.parametrize("config", CONFIGS)
def test_phantom_256_tv1_iso(config):
    _, noisy = noisy_phantom(256, 256, 0.1, seed=1)
    Cg, Co = cons_pair("amp", 256, 256)
    x, st = gpu_denoise(noisy, 0.05, 100, "tv1_iso", 0.5, Cg, config=config)
    b, res = run_oracle(noisy, 0.05, 100, "tv1_iso", 0.5, Co)
    check_parity(x, res, b, noisy, 0.05, "tv1_iso", 0.5)
    assert st["iters"] == 100 and not st["stopped"] and st["status"] == 0
    # the fused FP64 reductions against the oracle's FP64 evaluation of the same point
    P = float(primal_value(res.x, b, f32(0.05), "tv1_iso", 0.5))
    D = float(dual_value(res.q, b, f32(0.05), Co))
    assert st["primal"] == pytest.approx(P, rel=1e-6)
    assert st["dual"] == pytest.approx(D, rel=1e-6)
    assert abs(st["gap"] - (P - D)) <= 2e-6 * P


# --------------------------------------------------------------- all TV types x constraints, ragged tiles
@pytest.mark.parametrize("config", CONFIGS)
@pytest.mark.parametrize("kind", ["none", "amp", "amp_rect", "amp_mask"])
@pytest.mark.parametrize("tv", TV_NAMES)
def test_types_constraints_ragged(tv, kind, config):
    m, n = 67, 131
    _, noisy = noisy_phantom(m, n, 0.2, seed=3)
    Cg, Co = cons_pair(kind, m, n, seed=5)
    alpha = 0.4
    lam = 0.08
    x, st = gpu_denoise(noisy, lam, 23, tv, alpha, Cg, config=config)
    b, res = run_oracle(noisy, lam, 23, tv, alpha, Co)
    check_parity(x, res, b, noisy, lam, tv, alpha)


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (45, 1), (2, 3), (3, 2), (17, 65), (129, 63), (200, 7)])
@pytest.mark.parametrize("tv", TV_NAMES)
@pytest.mark.parametrize("config", CONFIGS)
def test_degenerate_shapes(shape, tv, config):
    m, n = shape
    rng = np.random.default_rng(m * 1000 + n)
    b_np = 0.7 * (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))
    Cg, Co = cons_pair("amp", m, n)
    x, st = gpu_denoise(b_np, 0.1, 17, tv, 0.5, Cg, config=config)
    b, res = run_oracle(b_np, 0.1, 17, tv, 0.5, Co)
    check_parity(x, res, b, b_np, 0.1, tv, 0.5)


@pytest.mark.parametrize("tv", ["tv2_iso", "tv2_aniso"])
@pytest.mark.parametrize("alpha", [0.0, 1.0, 0.25])
def test_type2_alpha_edges(tv, alpha):
    _, noisy = noisy_phantom(40, 50, 0.1, seed=8)
    Cg, Co = cons_pair("amp", 40, 50)
    x, _ = gpu_denoise(noisy, 0.06, 20, tv, alpha, Cg)
    b, res = run_oracle(noisy, 0.06, 20, tv, alpha, Co)
    check_parity(x, res, b, noisy, 0.06, tv, alpha)


# --------------------------------------------------------------- closed forms on the GPU
@pytest.mark.parametrize("tv", TV_NAMES)
def test_lambda_zero_and_zero_iters(tv):
    _, noisy = noisy_phantom(33, 70, 0.3, seed=4)
    noisy = noisy * 1.5
    Cg, Co = cons_pair("amp_rect", 33, 70)
    bt = torch.as_tensor(to_c64(noisy).astype(np.complex128))
    want = oracle_PC(bt.real, bt.imag, Co)
    want = (want[0] + 1j * want[1]).numpy()
    for lam, K in [(0.0, 50), (0.1, 0)]:
        x, st = gpu_denoise(noisy, lam, K, tv, 0.5, Cg)
        assert np.max(np.abs(x - want)) <= 1e-6
        assert st["iters"] == 0
        if lam == 0.0:
            assert abs(st["gap"]) <= 1e-6 * max(st["primal"], 1e-30)


@pytest.mark.parametrize("tv", TV_NAMES)
def test_constant_image_stays_projected(tv):
    b_np = np.full((50, 60), 1.4 * np.exp(0.7j))
    Cg, _ = cons_pair("amp", 50, 60)
    x, st = gpu_denoise(b_np, 0.2, 40, tv, 0.5, Cg)
    want = np.complex64(np.exp(0.7j))
    assert np.max(np.abs(x - want)) <= 1e-6
    assert st["primal"] == pytest.approx(0.5 * 50 * 60 * abs(to_c64(np.array([1.4 * np.exp(0.7j)]))[0] - want) ** 2,
                                         rel=1e-5)


# --------------------------------------------------------------- dual state: export, feasibility, warm start
@pytest.mark.parametrize("tv", TV_NAMES)
def test_dual_export_and_warm_start(tv):
    m, n = 70, 90
    _, noisy = noisy_phantom(m, n, 0.1, seed=12)
    Cg, Co = cons_pair("amp", m, n)
    b = torch.from_numpy(to_c64(noisy)).cuda()
    dual = torch.zeros(m * n * 4, dtype=torch.float32, device="cuda")
    x1 = ctv.denoise(b, 0.05, tv, 30, Cg, 0.5, dual_state=dual)
    torch.cuda.synchronize()
    assert padded_slots_zero(dual, m, n)
    q = dual_to_paper(dual, m, n)
    assert in_S(q, tv, 0.5, slack=1e-5)
    bp, res = run_oracle(noisy, 0.05, 30, tv, 0.5, Co)
    for a, c in zip(q, res.q):
        assert float((a - c).abs().max()) <= 1e-3
    # warm start from the exported q, against the oracle warm-started from the same q
    x2 = ctv.denoise(b, 0.05, tv, 15, Cg, 0.5, dual_state=dual, warm_start=True)
    torch.cuda.synchronize()
    _, res2 = run_oracle(noisy, 0.05, 15, tv, 0.5, Co, q0=q)
    check_parity(x2.cpu().numpy(), res2, bp, noisy, 0.05, tv, 0.5)


# --------------------------------------------------------------- gap stopping
# A check whose interval ends in a pass of fewer than T iterations is evaluated in
# that pass (strip configurations of up to four rows per thread); otherwise, or
# for other configurations, by the separate gap kernel after the pass. The cases
# below run both: every = 10 ends its intervals in a short pass for T = 3, 4, 6, 8;
# every = 12 is a multiple of T = 3, 4, 6 (separate kernel) but not of 8.
@pytest.mark.parametrize("tv", ["tv1_iso", "tv2_aniso"])
@pytest.mark.parametrize("config,every", [(-1, 10), (11, 10), (11, 12), (14, 10), (14, 12), (7, 10), (7, 12),
                                          (16, 10), (17, 12), (5, 10), (6, 10), (18, 10), (18, 12)])
def test_gap_stopping(tv, config, every):
    m, n = 96, 80
    _, noisy = noisy_phantom(m, n, 0.1, seed=21)
    Cg, Co = cons_pair("amp_rect", m, n)
    tol = 2e-4
    x, st = gpu_denoise(noisy, 0.05, 400, tv, 0.5, Cg, check_every=every, gap_tol=tol, config=config)
    assert st["stopped"] and st["iters"] % every == 0 and 0 < st["iters"] < 400
    k = st["iters"]
    b, res = run_oracle(noisy, 0.05, k, tv, 0.5, Co, check_every=every)
    check_parity(x, res, b, noisy, 0.05, tv, 0.5)
    gaps = {h["k"]: h for h in res.history}
    # the oracle agrees that the test passed at k and had not passed one check earlier
    assert gaps[k]["gap"] <= tol * gaps[k]["primal"] * 1.05
    if k - every in gaps:
        assert gaps[k - every]["gap"] > tol * gaps[k - every]["primal"] * 0.95


# --------------------------------------------------------------- batched, per-image lambda
@pytest.mark.parametrize("tv", TV_NAMES)
def test_batched_per_image_lambda(tv):
    B, m, n = 3, 60, 75
    imgs = [noisy_phantom(m, n, 0.1, seed=40 + i)[1] for i in range(B)]
    lams = [0.02, 0.07, 0.0]
    Cg, Co = cons_pair("amp", m, n)
    b = torch.from_numpy(np.stack([to_c64(i) for i in imgs])).cuda()
    x, st = ctv.denoise(b, torch.tensor(lams), tv, 25, Cg, 0.5, return_stats=True)
    torch.cuda.synchronize()
    xs = x.cpu().numpy()
    for i in range(B):
        bp, res = run_oracle(imgs[i], lams[i], 25, tv, 0.5, Co)
        check_parity(xs[i], res, bp, imgs[i], lams[i], tv, 0.5)
        P = float(primal_value(res.x, bp, f32(lams[i]), tv, 0.5))
        assert st[i]["primal"] == pytest.approx(P, rel=1e-6)


# --------------------------------------------------------------- full size (2048^2, 200 iterations), sampled
@pytest.mark.parametrize("tv", TV_NAMES)
def test_full_size_sampled(tv):
    m = n = 2048
    K = 200
    lam = 0.05
    _, noisy = noisy_phantom(m, n, 0.1, seed=2048)
    rect = support_rect(m, n)
    Cg = ctv.Constraint(amp_max=1.0, rect=rect)
    b = torch.from_numpy(to_c64(noisy)).cuda()
    dual = torch.empty(m * n * 4, dtype=torch.float32, device="cuda")
    x, st = ctv.denoise(b, lam, tv, K, Cg, 0.5, dual_state=dual, return_stats=True)
    torch.cuda.synchronize()
    xg = x.cpu().numpy()
    binf = float(np.abs(to_c64(noisy)).max())
    R = K + 2
    for (j, k) in [(1024, 1000), (0, 2047), (300, 1800)]:
        j0, j1 = max(0, j - R), min(m, j + R + 1)
        k0, k1 = max(0, k - R), min(n, k + R + 1)
        wrect = (rect[0] - j0, rect[1] - k0, rect[2] - j0, rect[3] - k0)
        Co = oracle_constraint(1.0, rect=wrect)
        _, res = run_oracle(noisy[j0:j1, k0:k1], lam, K, tv, 0.5, Co)
        xo = complex(res.x[0][j - j0, k - k0], res.x[1][j - j0, k - k0])
        assert abs(complex(xg[j, k]) - xo) <= XTOL * binf
    # properties that hold at any size
    amp = np.abs(xg)
    assert amp.max() <= 1 + 1e-6
    assert np.all(xg[: rect[0], :] == 0) and np.all(xg[:, rect[3]:] == 0)
    assert padded_slots_zero(dual, m, n)
    d = dual.reshape(m, n, 4)
    if tv == "tv1_iso":
        assert float(d.pow(2).sum(-1).max()) <= 1 + 1e-5
    elif tv == "tv2_aniso":
        assert float(d.abs().max()) <= 0.5 + 1e-6
    assert st["gap"] >= -1e-6 * st["primal"]
    # the fused FP64 objective against the oracle's FP64 evaluation of the GPU's x
    bt = torch.as_tensor(to_c64(noisy).astype(np.complex128))
    P = objective(xg, (bt.real, bt.imag), lam, tv, 0.5)
    assert st["primal"] == pytest.approx(P, rel=1e-6)


# --------------------------------------------------------------- full size (2048^2, 200 iterations), whole image
@pytest.mark.parametrize("tv", TV_NAMES)
def test_full_size_whole_image(tv):
    # The headline workload's solve (2048^2, amplitude bound plus support
    # rectangle, 200 iterations) against the oracle on the whole image: every
    # pixel within 1e-4 ||b||_inf and the objective within 1e-6, after the same
    # iteration count; and the fused FP64 primal value against the oracle's
    # evaluation of the GPU's x.
    m = n = 2048
    K = 200
    lam = 0.05
    _, noisy = noisy_phantom(m, n, 0.1, seed=2049)
    rect = support_rect(m, n)
    Cg = ctv.Constraint(amp_max=1.0, rect=rect)
    x, st = gpu_denoise(noisy, lam, K, tv, 0.5, Cg)
    bp, res = run_oracle(noisy, lam, K, tv, 0.5, oracle_constraint(1.0, rect=rect))
    check_parity(x, res, bp, noisy, lam, tv, 0.5)
    assert st["iters"] == K and st["status"] == 0
    assert st["primal"] == pytest.approx(objective(x, bp, lam, tv, 0.5), rel=1e-6)


# --------------------------------------------------------------- argument errors
def test_invalid_arguments_raise():
    b = torch.zeros(8, 8, dtype=torch.complex64, device="cuda")
    with pytest.raises(RuntimeError):
        ctv.denoise(b, -1.0, "tv1_iso", 5)
    with pytest.raises(RuntimeError):
        ctv.denoise(b, float("nan"), "tv1_iso", 5)
    with pytest.raises(RuntimeError):
        ctv.denoise(b, 0.1, "tv2_iso", 5, alpha=1.5)
    with pytest.raises(RuntimeError):
        ctv.denoise(b, 0.1, "tv1_iso", -1)
    with pytest.raises(RuntimeError):
        ctv.denoise(b, 0.1, "tv1_iso", 5, config=99)


# --------------------------------------------------------------- box constraint, plain gradient projection
@pytest.mark.parametrize("config", [0, 3, 5])
@pytest.mark.parametrize("tv", TV_NAMES)
def test_box_constraint(tv, config):
    m, n = 70, 90
    _, noisy = noisy_phantom(m, n, 0.15, seed=17)
    box = (-0.5, 0.8, -0.3, 0.6)
    Cg = ctv.Constraint(amp_max=None, box=box, rect=(5, 3, 60, 85))
    Co = oracle_constraint(None, rect=(5, 3, 60, 85))
    Co.box = box
    x, _ = gpu_denoise(noisy, 0.06, 25, tv, 0.5, Cg, config=config)
    b, res = run_oracle(noisy, 0.06, 25, tv, 0.5, Co)
    check_parity(x, res, b, noisy, 0.06, tv, 0.5)


def test_box_and_amplitude_are_exclusive():
    b = torch.zeros(8, 8, dtype=torch.complex64, device="cuda")
    with pytest.raises(RuntimeError):
        ctv.denoise(b, 0.1, "tv1_iso", 5, ctv.Constraint(amp_max=1.0, box=(-1, 1, -1, 1)))


@pytest.mark.parametrize("tv", TV_NAMES)
def test_plain_gradient_projection(tv):
    # Eq. (21): the same kernels with the extrapolation switched off
    m, n = 64, 80
    _, noisy = noisy_phantom(m, n, 0.1, seed=19)
    Cg, Co = cons_pair("amp", m, n)
    x, st = gpu_denoise(noisy, 0.05, 40, tv, 0.5, Cg, plain_gp=True)
    b, res = run_oracle(noisy, 0.05, 40, tv, 0.5, Co, accelerate=False)
    check_parity(x, res, b, noisy, 0.05, tv, 0.5)
    assert st["iters"] == 40


# --------------------------------------------------------------- finalize with and without statistics
@pytest.mark.parametrize("tv", TV_NAMES)
@pytest.mark.parametrize("kind", ["amp_rect", "none"])
def test_light_finalize_matches_gap_finalize(tv, kind):
    # Without gap checks and without statistics the solve ends with the finalize
    # that writes only x (and q); with statistics it ends with the gap kernel.
    # Both evaluate Eq. (18) the same way, so x and the exported q agree bit for bit.
    m, n = 83, 131
    _, noisy = noisy_phantom(m, n, 0.1, seed=31)
    Cg, _ = cons_pair(kind, m, n)
    b = torch.from_numpy(to_c64(noisy)).cuda()
    x_light, x_stats = torch.empty_like(b), torch.empty_like(b)
    d_light = torch.zeros(m * n * 4, dtype=torch.float32, device="cuda")
    d_stats = torch.zeros_like(d_light)
    opts = ctv.make_opts(23, 0, 0.0, 0.5)
    ctv.ctv_denoise(b, x_light, 0.05, Cg, tv, opts, dual_state=d_light)
    st = ctv.ctv_denoise(b, x_stats, 0.05, Cg, tv, opts, dual_state=d_stats, want_stats=True)
    torch.cuda.synchronize()
    assert st["iters"] == 23
    assert torch.equal(x_light, x_stats)
    assert torch.equal(d_light, d_stats)


def test_light_finalize_row_stride():
    # images that are column windows of wider buffers (row stride ld > n)
    m, n, ld = 57, 70, 96
    _, noisy = noisy_phantom(m, ld, 0.1, seed=32)
    wide = torch.from_numpy(to_c64(noisy)).cuda()
    b = wide[:, 3:3 + n]
    out_a = torch.zeros_like(wide)
    out_b = torch.zeros_like(wide)
    opts = ctv.make_opts(17, 0, 0.0, 0.5)
    C = ctv.Constraint(amp_max=1.0)
    ctv.ctv_denoise(b, out_a[:, 3:3 + n], 0.04, C, "tv2_iso", opts)
    ctv.ctv_denoise(b, out_b[:, 3:3 + n], 0.04, C, "tv2_iso", opts, want_stats=True)
    ref = ctv.denoise(b.contiguous(), 0.04, "tv2_iso", 17, C, 0.5)
    torch.cuda.synchronize()
    assert torch.equal(out_a, out_b)
    assert torch.equal(out_a[:, 3:3 + n], ref)
    assert not out_a[:, :3].any() and not out_a[:, 3 + n:].any()   # nothing written outside the window


# --------------------------------------------------------------- stop graphs (early-stopping solves on large images)
@pytest.mark.parametrize("tv,tol,K", [("tv1_iso", 1e-4, 200), ("tv2_aniso", 1e-4, 200), ("tv1_aniso", 1e-12, 200),
                                      ("tv2_iso", 1e-12, 95), ("tv1_iso", 3e-4, 95)])
def test_stop_graph_matches_plain_launches(tv, tol, K):
    # From 512^2 pixels on, a solve with gap checks and a tolerance runs as a CUDA
    # graph whose check intervals are conditional nodes; with profiling on it
    # launches its passes one by one instead. Same kernels, same order: the same
    # x, the same stopping iteration. A call with new arguments launches plainly,
    # the second identical call builds the graph, later ones reuse it.
    from paper_2109_05496_gb300 import _lib
    lib = _lib.load()
    m, n = 520, 530
    _, noisy = noisy_phantom(m, n, 0.1, seed=41)
    Cg, _ = cons_pair("amp_rect", m, n)
    b = torch.from_numpy(to_c64(noisy)).cuda()
    x0 = torch.empty_like(b)
    x = torch.empty_like(b)
    opts = ctv.make_opts(K, 10, tol, 0.5)
    lib.ctv_profile_enable(1)
    try:
        s0 = ctv.ctv_denoise(b, x0, 0.05, Cg, tv, opts, want_stats=True)
    finally:
        lib.ctv_profile_enable(0)
    runs = []
    for _ in range(3):   # plain (first sight), graph built, graph reused
        x.fill_(0)
        st = ctv.ctv_denoise(b, x, 0.05, Cg, tv, opts, want_stats=True)
        torch.cuda.synchronize()
        runs.append((st, x.clone()))
    torch.cuda.synchronize()
    if tol > 1e-6:
        assert s0["stopped"] and 0 < s0["iters"] < K
    else:
        assert not s0["stopped"] and s0["iters"] == K
    for s, xr in runs:
        assert (s["iters"], s["stopped"]) == (s0["iters"], s0["stopped"])
        assert s["primal"] == pytest.approx(s0["primal"], rel=1e-12)
        assert s["gap"] == pytest.approx(s0["gap"], rel=1e-9, abs=1e-12 * s0["primal"])
        assert torch.equal(xr, x0)


def test_stop_graph_changed_arguments_rebuild():
    # a different lambda or output buffer is a different graph, not a stale one
    m, n = 512, 512
    _, noisy = noisy_phantom(m, n, 0.1, seed=42)
    b = torch.from_numpy(to_c64(noisy)).cuda()
    C = ctv.Constraint(amp_max=1.0)
    opts = ctv.make_opts(120, 10, 1e-5, 0.5)
    outs = {}
    for lam in (0.03, 0.03, 0.08, 0.08, 0.03):   # second sights build graphs; the last call reuses one
        x = torch.empty_like(b)
        st = ctv.ctv_denoise(b, x, lam, C, "tv1_iso", opts, want_stats=True)
        torch.cuda.synchronize()
        ref = ctv.denoise(b, lam, "tv1_iso", st["iters"], C, 0.5)   # plain solve of the same length
        torch.cuda.synchronize()
        assert torch.equal(x, ref)
        outs.setdefault(lam, []).append((st["iters"], x))
    for lam, rs in outs.items():
        assert all(r[0] == rs[0][0] and torch.equal(r[1], rs[0][1]) for r in rs)


def test_batched_stopping_is_per_image():
    # A batch large enough for a stop graph if it were one image: each image must
    # stop on its own check, whatever the others do.
    B, m, n = 4, 260, 260
    imgs = np.stack([to_c64(noisy_phantom(m, n, 0.1, seed=60 + i)[1]) for i in range(B)])
    lams = torch.tensor([0.01, 0.1, 0.03, 0.06], dtype=torch.float32, device="cuda")
    b = torch.from_numpy(imgs).cuda()
    C = ctv.Constraint(amp_max=1.0)
    opts = ctv.make_opts(150, 10, 1e-5, 0.5)
    for _ in range(3):   # also after the library has seen the arguments before
        x = torch.empty_like(b)
        st = ctv.ctv_denoise_batched(b, x, lams, C, "tv1_iso", opts, want_stats=True)
        torch.cuda.synchronize()
        for i in range(B):
            xi = torch.empty_like(b[i])
            si = ctv.ctv_denoise(b[i], xi, float(lams[i]), C, "tv1_iso", opts, want_stats=True)
            torch.cuda.synchronize()
            assert st[i]["iters"] == si["iters"]
            assert torch.equal(x[i], xi)
