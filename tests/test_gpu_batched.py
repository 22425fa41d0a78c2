"""Batched denoising of uneven images in one graph replay (ctv_plan_*): parity
with the FP64 oracle per image, and bit-for-bit agreement with a loop of
ctv_denoise calls using the same kernel configuration."""
import numpy as np
import pytest
import torch

import paper_2109_05496_gb300 as ctv
from phantoms import batch_params, batch_shapes, noisy_phantom, to_c64
from tests.helpers import TV_NAMES, oracle_constraint, run_oracle
from tests.test_gpu_denoise import check_parity

pytestmark = pytest.mark.gpu


def make_batch(count, lo, hi, seed, sigma=0.1):
    shapes = batch_shapes(count, lo, hi, seed)
    lams, types = batch_params(count, seed + 1)
    imgs = []
    for i, (m, n) in enumerate(shapes):
        _, noisy = noisy_phantom(m, n, sigma, seed=seed * 1000 + i)
        imgs.append(to_c64(noisy))
    return shapes, lams, types, imgs


def plan_images(imgs, lams, types, rects=None):
    out = []
    for i, a in enumerate(imgs):
        b = torch.from_numpy(a).cuda()
        C = ctv.Constraint(amp_max=1.0, rect=None if rects is None else rects[i])
        out.append({"b": b, "x": torch.empty_like(b), "lam": float(lams[i]), "tv": TV_NAMES[int(types[i])],
                    "alpha": 0.5, "C": C})
    return out


@pytest.mark.parametrize("config", [2, 5, 6, 7, 11, 14, 18])
def test_plan_matches_oracle_and_loop(config):
    shapes, lams, types, imgs = make_batch(14, 3, 150, seed=5)
    ims = plan_images(imgs, lams, types)
    K = 27
    plan = ctv.Plan(ims, K, config=config)
    plan.execute()
    st = plan.stats()
    for i, im in enumerate(ims):
        tv = TV_NAMES[int(types[i])]
        bp, res = run_oracle(imgs[i], lams[i], K, tv, 0.5, oracle_constraint(1.0))
        check_parity(im["x"].cpu().numpy(), res, bp, imgs[i], lams[i], tv, 0.5)
        assert st[i]["iters"] == K
        # the same kernels one image at a time give the same bits
        x1 = ctv.denoise(im["b"], float(lams[i]), tv, K, im["C"], 0.5, config=config)
        assert torch.equal(x1, im["x"])
    # a second replay reproduces the first
    before = [im["x"].clone() for im in ims]
    plan.execute()
    torch.cuda.synchronize()
    for a, im in zip(before, ims):
        assert torch.equal(a, im["x"])


def test_plan_autotune_picks_a_plan_configuration():
    # config "auto": every plan configuration is timed on these images and the
    # fastest kept; its results are those of a plan built with that configuration
    shapes, lams, types, imgs = make_batch(10, 3, 180, seed=8)
    ims = plan_images(imgs, lams, types)
    plan = ctv.Plan(ims, 20, config="auto")
    cfg = plan.info()["config"]
    assert cfg in (2, 5, 6, 7, 11, 14, 18)
    plan.execute()
    torch.cuda.synchronize()
    got = [im["x"].clone() for im in ims]
    ref = ctv.Plan(ims, 20, config=cfg)
    ref.execute()
    torch.cuda.synchronize()
    for a, im in zip(got, ims):
        assert torch.equal(a, im["x"])


def test_plan_gap_stopping_per_image():
    shapes, lams, types, imgs = make_batch(8, 40, 120, seed=9)
    ims = plan_images(imgs, lams, types)
    plan = ctv.Plan(ims, 300, check_every=10, gap_tol=3e-4)
    plan.execute()
    st = plan.stats()
    for i, im in enumerate(ims):
        tv = TV_NAMES[int(types[i])]
        x1, s1 = ctv.denoise(im["b"], float(lams[i]), tv, 300, im["C"], 0.5, check_every=10, gap_tol=3e-4,
                             config=plan.info()["config"], return_stats=True)
        assert st[i]["iters"] == s1["iters"] and st[i]["stopped"] == s1["stopped"]
        assert torch.equal(x1, im["x"])


def test_plan_gap_runs_span_images():
    # about 6000 gap tiles, more than the resident blocks of the gap / finalize
    # launch, so each block evaluates a run of tiles that crosses image borders;
    # per-image stopping, final statistics and x agree with one-image solves
    shapes, lams, types, imgs = make_batch(48, 150, 260, seed=12)
    ims = plan_images(imgs, lams, types)
    plan = ctv.Plan(ims, 200, check_every=10, gap_tol=1e-4)
    plan.execute()
    st = plan.stats()
    stopped = 0
    for i, im in enumerate(ims):
        tv = TV_NAMES[int(types[i])]
        x1, s1 = ctv.denoise(im["b"], float(lams[i]), tv, 200, im["C"], 0.5, check_every=10, gap_tol=1e-4,
                             config=plan.info()["config"], return_stats=True)
        assert st[i]["iters"] == s1["iters"] and st[i]["stopped"] == s1["stopped"]
        stopped += int(s1["stopped"])
        assert torch.equal(x1, im["x"])
        # the plan sums FP32 partials of 4 pixels per thread in FP64, a single-image
        # solve sums per column in compensated FP32 and per warp in FP64: the same
        # terms, rounded in different groups (about 1e-10 apart in practice)
        for key in ("primal", "dual"):
            assert st[i][key] == pytest.approx(s1[key], rel=1e-8)
        assert st[i]["gap"] == pytest.approx(s1["gap"], rel=1e-6, abs=1e-8 * abs(s1["primal"]))
    assert 0 < stopped < len(ims)


def test_plan_full_workload_sampled():
    # 512 images, sides log-uniform in [64, 1024], lambda ~ U[0.01, 0.1], mixed TV types, 100 iterations
    shapes, lams, types, imgs = make_batch(512, 64, 1024, seed=2021)
    ims = plan_images(imgs, lams, types)
    plan = ctv.Plan(ims, 100)
    plan.execute()
    torch.cuda.synchronize()
    info = plan.info()
    assert info["pixel_iters"] == pytest.approx(100 * sum(m * n for m, n in shapes))
    order = np.argsort([m * n for m, n in shapes])
    for i in list(order[:3]) + [int(order[len(order) // 2])]:
        tv = TV_NAMES[int(types[i])]
        bp, res = run_oracle(imgs[i], lams[i], 100, tv, 0.5, oracle_constraint(1.0))
        check_parity(ims[i]["x"].cpu().numpy(), res, bp, imgs[i], lams[i], tv, 0.5)
    for i in list(order[-2:]) + list(order[100:103]):
        tv = TV_NAMES[int(types[i])]
        x1 = ctv.denoise(ims[i]["b"], float(lams[i]), tv, 100, ims[i]["C"], 0.5, config=info["config"])
        assert torch.equal(x1, ims[i]["x"])


def test_plan_full_workload_oracle_subset():
    # The 512-image workload against the oracle: every image of at most 256^2
    # pixels and 32 seeded random larger ones, element by element after 100
    # iterations, with the objective bar of the single-image tests.
    from tests.helpers import objective, oracle_x_many
    from tests.test_gpu_denoise import OBJTOL, XTOL
    shapes, lams, types, imgs = make_batch(512, 64, 1024, seed=2021)
    ims = plan_images(imgs, lams, types)
    plan = ctv.Plan(ims, 100)
    plan.execute()
    torch.cuda.synchronize()
    px = np.array([m * n for m, n in shapes])
    small = [i for i in range(len(shapes)) if px[i] <= 256 * 256]
    rng = np.random.default_rng(77)
    large = sorted(rng.choice([i for i in range(len(shapes)) if px[i] > 256 * 256], 32, replace=False).tolist())
    picked = small + large
    assert len(small) > 100
    jobs = [(imgs[i], float(lams[i]), 100, TV_NAMES[int(types[i])], 0.5, 1.0) for i in picked]
    xo_all = oracle_x_many(jobs)
    for i, xo in zip(picked, xo_all):
        tv = TV_NAMES[int(types[i])]
        xg = ims[i]["x"].cpu().numpy()
        binf = float(np.abs(imgs[i]).max())
        assert float(np.abs(xg.astype(np.complex128) - xo).max()) <= XTOL * binf, i
        bt = torch.as_tensor(imgs[i].astype(np.complex128))
        bp = (bt.real.clone(), bt.imag.clone())
        Pg, Po = objective(xg, bp, lams[i], tv, 0.5), objective(xo, bp, lams[i], tv, 0.5)
        assert abs(Pg - Po) <= OBJTOL * abs(Po), i


def test_plan_rejects_unsupported_configuration():
    shapes, lams, types, imgs = make_batch(2, 20, 40, seed=3)
    with pytest.raises(RuntimeError):
        ctv.Plan(plan_images(imgs, lams, types), 10, config=13)
