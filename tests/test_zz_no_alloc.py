"""ctv_denoise_noalloc: the denoiser for callers that cannot allocate device memory
(programs whose device memory all belongs to their own pool, plugin hosts whose
callbacks must not allocate, latency-critical loops). It keeps its scratch in a
fixed array inside the library instead of a caller workspace.

Checked through the C ABI against ctv_denoise on two calls in a row (different
sizes, TV types and constraints, so stale scratch from the first call would
show), within the parity tolerance of the other tests: once without a stopping
test, once with a call that stops early followed by one that must run all its
iterations (the stop flag lives in the shared array), and at the largest
accepted size. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2109_05496_gb300 as ctv
from paper_2109_05496_gb300 import _lib
from phantoms import noisy_phantom, support_rect, to_c64

pytestmark = pytest.mark.gpu

XTOL = 1e-4


def call_noalloc(lib, b, x, lam, C, tv, opts, stats):
    cc, keep = C.to_c()
    st = lib.ctv_denoise_noalloc(b.data_ptr(), x.data_ptr(), b.shape[0], b.shape[1], b.stride(0), float(lam),
                                 ctypes.byref(cc), ctv.api.tv_code(tv), ctypes.byref(opts),
                                 ctypes.byref(stats), torch.cuda.current_stream().cuda_stream)
    del keep
    return st


def test_noalloc_matches_ctv_denoise_twice():
    lib = _lib.load()
    cases = [
        (300, 410, 0.05, "tv1_iso", ctv.Constraint(amp_max=1.0, rect=support_rect(300, 410)), 60),
        (129, 77, 0.08, "tv2_aniso", ctv.Constraint(amp_max=1.0), 35),
    ]
    for i, (m, n, lam, tv, C, K) in enumerate(cases):
        _, noisy = noisy_phantom(m, n, 0.1, seed=70 + i)
        b = torch.from_numpy(to_c64(noisy)).cuda()
        x_ref, st_ref = ctv.denoise(b, lam, tv, K, C, 0.5, return_stats=True)
        x = torch.empty_like(b)
        opts = ctv.make_opts(K, alpha=0.5)
        st = _lib.CtvStats()
        status = call_noalloc(lib, b, x, lam, C, tv, opts, st)
        assert status == 0, lib.ctv_status_string(status)
        torch.cuda.synchronize()
        binf = float(b.abs().max())
        assert float((x - x_ref).abs().max()) <= XTOL * binf
        assert st.iters == st_ref["iters"] == K
        assert st.primal == pytest.approx(st_ref["primal"], rel=1e-6)
        assert st.gap == pytest.approx(st_ref["gap"], rel=1e-4, abs=1e-9 * st_ref["primal"])


def _compare(lib, m, n, lam, tv, C, K, seed, check_every=0, gap_tol=0.0):
    _, noisy = noisy_phantom(m, n, 0.1, seed=seed)
    b = torch.from_numpy(to_c64(noisy)).cuda()
    x_ref, st_ref = ctv.denoise(b, lam, tv, K, C, 0.5, check_every=check_every, gap_tol=gap_tol,
                                return_stats=True)
    x = torch.empty_like(b)
    opts = ctv.make_opts(K, check_every, gap_tol, 0.5)
    st = _lib.CtvStats()
    status = call_noalloc(lib, b, x, lam, C, tv, opts, st)
    assert status == 0, lib.ctv_status_string(status)
    torch.cuda.synchronize()
    assert float((x - x_ref).abs().max()) <= XTOL * float(b.abs().max())
    assert st.iters == st_ref["iters"] and bool(st.stopped) == st_ref["stopped"]
    assert st.primal == pytest.approx(st_ref["primal"], rel=1e-6)
    return st


def test_noalloc_stop_does_not_carry_into_the_next_call():
    lib = _lib.load()
    C = ctv.Constraint(amp_max=1.0)
    st = _compare(lib, 256, 256, 0.05, "tv1_iso", C, 200, 81, check_every=10, gap_tol=1e-4)
    assert st.stopped and st.iters < 200
    st = _compare(lib, 200, 180, 0.05, "tv1_aniso", C, 30, 82, check_every=10, gap_tol=0.0)
    assert not st.stopped and st.iters == 30


def test_noalloc_largest_accepted_size():
    lib = _lib.load()
    st = _compare(lib, 512, 512, 0.04, "tv2_iso", ctv.Constraint(amp_max=1.0, rect=support_rect(512, 512)), 24, 83)
    assert st.iters == 24


def test_noalloc_rejects_oversize_images():
    lib = _lib.load()
    m, n = 513, 512          # one row more than CTV_NOALLOC_MAX_PIXELS = 512 * 512
    b = torch.zeros(m, n, dtype=torch.complex64, device="cuda")
    x = torch.empty_like(b)
    st = _lib.CtvStats()
    status = call_noalloc(lib, b, x, 0.05, ctv.Constraint(amp_max=1.0), "tv1_iso", ctv.make_opts(10), st)
    assert status == 7      # CTV_ETOOBIG
    assert b"CTV_NOALLOC_MAX_PIXELS" in lib.ctv_status_string(status)
