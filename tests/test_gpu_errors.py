"""Asynchronous errors: a NaN or an infinity in an input is reported as
CTV_ENONFINITE, in ctv_stats.status where a call returns statistics and by
ctv_get_last_error for every solve, and the context stays usable afterwards.
The bad values are planted in the inputs on the host; no kernel is made to fail."""
import math

import numpy as np
import pytest
import torch

import paper_2109_05496_gb300 as ctv
from phantoms import fresnel_tf, noisy_phantom, pr_object, simulate_intensity, to_c64

pytestmark = pytest.mark.gpu

ENONFINITE = 5


def _image(m, n, seed=3):
    _, noisy = noisy_phantom(m, n, 0.1, seed=seed)
    return to_c64(noisy)


@pytest.fixture(autouse=True)
def clean_word():
    ctv.get_last_error()          # start from a cleared word
    yield
    ctv.get_last_error()


@pytest.mark.parametrize("bad", [math.nan, math.inf, -math.inf])
@pytest.mark.parametrize("with_stats", [True, False])
def test_denoise_reports_nonfinite_b(bad, with_stats):
    m, n = 96, 80
    b_np = _image(m, n)
    b_np[37, 11] = complex(bad, 0.0) if bad != -math.inf else complex(0.0, bad)
    b = torch.from_numpy(b_np).cuda()
    # with statistics: the gap kernels read b; without: the light finalize does
    x, st = ctv.denoise(b, 0.05, "tv1_iso", 20, ctv.Constraint(amp_max=1.0), return_stats=True) if with_stats \
        else (ctv.denoise(b, 0.05, "tv1_iso", 20, ctv.Constraint(amp_max=1.0)), None)
    if st is not None:
        assert st["status"] == ENONFINITE
    assert ctv.get_last_error() == ENONFINITE
    assert ctv.get_last_error() == 0                   # read and cleared
    # the context is still usable and a finite image reports nothing
    good = torch.from_numpy(_image(m, n)).cuda()
    x2, st2 = ctv.denoise(good, 0.05, "tv1_iso", 20, ctv.Constraint(amp_max=1.0), return_stats=True)
    assert st2["status"] == 0 and bool(torch.isfinite(torch.view_as_real(x2)).all())
    assert ctv.get_last_error() == 0


def test_denoise_with_gap_checks_reports_nonfinite_b():
    m = n = 128
    b_np = _image(m, n)
    b_np[0, 0] = complex(math.nan, math.nan)
    b = torch.from_numpy(b_np).cuda()
    _, st = ctv.denoise(b, 0.05, "tv2_aniso", 40, ctv.Constraint(amp_max=1.0), check_every=10, gap_tol=1e-6,
                        return_stats=True)
    assert st["status"] == ENONFINITE and not st["stopped"]
    assert ctv.get_last_error() == ENONFINITE


def test_batched_marks_only_the_bad_image():
    B, m, n = 3, 64, 72
    b_np = np.stack([_image(m, n, seed=10 + i) for i in range(B)])
    b_np[1, 5, 70] = complex(math.inf, 1.0)
    b = torch.from_numpy(b_np).cuda()
    lams = torch.tensor([0.03, 0.05, 0.07], dtype=torch.float32, device="cuda")
    _, st = ctv.denoise(b, lams, "tv1_aniso", 16, ctv.Constraint(amp_max=1.0), return_stats=True)
    assert [s["status"] for s in st] == [0, ENONFINITE, 0]
    assert ctv.get_last_error() == ENONFINITE


def test_plan_marks_only_the_bad_image():
    shapes = [(64, 64), (70, 90), (33, 128), (128, 40)]
    ims = []
    for i, (m, n) in enumerate(shapes):
        bn = _image(m, n, seed=20 + i)
        if i == 2:
            bn[m - 1, n - 1] = complex(0.0, math.nan)
        bb = torch.from_numpy(bn).cuda()
        ims.append({"b": bb, "x": torch.empty_like(bb), "lam": 0.04, "tv": ("tv1_iso", "tv2_iso")[i % 2],
                    "C": ctv.Constraint(amp_max=1.0)})
    plan = ctv.Plan(ims, 12)
    plan.execute()
    st = plan.stats()
    assert [s["status"] for s in st] == [0, 0, ENONFINITE, 0]
    assert ctv.get_last_error() == ENONFINITE
    plan.close()


def _pr_inputs(m=64):
    M = 2 * m
    H = fresnel_tf(M, M, 532e-9, 2e-6, 5e-3).astype(np.complex64)
    x_gt = pr_object(m, m, seed=5, blur_sigma=2.0)
    y = simulate_intensity(x_gt, H.astype(np.complex128), seed=6, photons=1e4)
    return np.sqrt(y).astype(np.float32), H


@pytest.mark.parametrize("where", ["sqrt_y", "x0", "H"])
def test_pr_solve_reports_nonfinite_input(where):
    m = 64
    sy, H = _pr_inputs(m)
    x0 = np.full((m, m), 0.5 + 0.1j, dtype=np.complex64)
    if where == "sqrt_y":
        sy[3, 4] = math.nan
    elif where == "x0":
        x0[10, 60] = complex(math.inf, 0.0)
    else:
        H[100, 7] = complex(math.nan, 0.0)
    plan = ctv.PRPlan(m, m, 2 * m, 2 * m)
    args = (torch.from_numpy(x0).cuda(), torch.from_numpy(sy).cuda(), torch.from_numpy(H).cuda())
    plan.solve(*args, 0.01, 1.0, ctv.Constraint(amp_max=1.0), "tv1_aniso", 5, 3)
    assert ctv.get_last_error() == ENONFINITE
    # the gradient call alone reports it too
    plan.gradient(*args)
    assert ctv.get_last_error() == ENONFINITE
    # finite inputs afterwards: nothing reported
    sy2, H2 = _pr_inputs(m)
    plan.solve(torch.from_numpy(np.full((m, m), 0.5 + 0.1j, dtype=np.complex64)).cuda(),
               torch.from_numpy(sy2).cuda(), torch.from_numpy(H2).cuda(), 0.01, 1.0, ctv.Constraint(amp_max=1.0),
               "tv1_aniso", 5, 3)
    assert ctv.get_last_error() == 0
    plan.close()
