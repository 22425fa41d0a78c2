"""The C-ABI library builds, loads and exports every function include/*.h
declares; the Python binding declares a signature for each (no GPU needed)."""
import glob
import os
import re

import pytest

from paper_2109_05496_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(ctv_[A-Za-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_functions():
    names = declared_functions()
    assert "ctv_denoise" in names and "ctv_denoise_batched" in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if getattr(lib, n, None) is None]
    assert not missing, missing


def test_binding_covers_every_symbol():
    missing = [n for n in declared_functions() if n not in _lib.SIGNATURES]
    assert not missing, missing


def test_host_only_queries(lib):
    assert lib.ctv_abi_version() >= 1
    assert lib.ctv_status_string(0) == b"ok"
    assert lib.ctv_status_string(1) == b"invalid argument"
    n = lib.ctv_num_configs()
    assert n >= 1
    # workspace: stats block + four float4 m x n buffers
    assert lib.ctv_denoise_workspace_size(1, 256, 256) >= 4 * 256 * 256 * 16
    assert lib.ctv_denoise_workspace_size(0, 256, 256) == 0


def test_null_arguments_rejected_before_any_launch(lib):
    # argument validation happens on the host and returns CTV_EINVAL (1)
    opts = _lib.CtvOpts(10, 0, 0.0, 0.5, 0, -1)
    st = lib.ctv_denoise(None, None, 8, 8, 8, 0.1, None, 0, opts, None, None, 0, None, None)
    assert st == 1


def test_tune_table_host_only(lib):
    import ctypes
    assert lib.ctv_size_class(1024, 1024) == 20
    assert lib.ctv_size_class(0, 5) == -1
    v = ctypes.c_int()
    assert lib.ctv_tune_get(20, 1, ctypes.byref(v)) == 0
    before = v.value
    assert lib.ctv_tune_set(20, 1, 3) == 0
    assert lib.ctv_tune_get(20, 1, ctypes.byref(v)) == 0 and v.value == 3
    assert lib.ctv_default_config(1024, 1024, 100, 1, None) == 3      # the tuned choice wins
    assert lib.ctv_tune_set(20, 1, before) == 0
    assert lib.ctv_tune_set(20, 9, 3) == 1 and lib.ctv_tune_set(99, 0, 3) == 1   # CTV_EINVAL
    assert lib.ctv_tune_set(20, 1, lib.ctv_num_configs()) == 1
    assert lib.ctv_default_config(2048, 2048, 1, 0, None) == 0        # a single iteration needs no blocking
    # a support rectangle changes the large-image choice (its outside tiles are cheap)
    from paper_2109_05496_gb300 import api
    rect, _ = api.Constraint(amp_max=1.0, rect=(256, 256, 1792, 1792)).to_c()
    amp, _ = api.Constraint(amp_max=1.0).to_c()
    assert lib.ctv_default_config(2048, 2048, 200, 0, ctypes.byref(rect)) == 18
    assert lib.ctv_default_config(2048, 2048, 200, 0, ctypes.byref(amp)) == 5


def test_config_table_matches_library(lib):
    import ctypes
    rows = build.config_table()
    assert len(rows) == lib.ctv_num_configs()
    for (cid, kind, T, A, B, C) in rows:
        t, w, h, nt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        assert lib.ctv_config_info(cid, ctypes.byref(t), ctypes.byref(w), ctypes.byref(h), ctypes.byref(nt)) == 0
        assert t.value == T
        if kind == 0:
            assert (w.value, h.value, nt.value) == (A, B, C)
        else:
            assert (w.value, h.value, nt.value) == (32 * A, B * C, 32 * A * B)


def test_default_configuration_by_size(lib):
    # the measured size rule of the untuned default (no tuned entry for these
    # classes in a fresh process): 32 x 32 regions for small images, 64 x 64
    # regions above, the depth and rows per thread depending on size and on
    # whether a support rectangle makes the outside tiles cheap
    import ctypes
    from paper_2109_05496_gb300 import api
    rect, _ = api.Constraint(amp_max=1.0, rect=(1, 1, 2, 2)).to_c()
    amp, _ = api.Constraint(amp_max=1.0).to_c()
    want = {256: (17, 17), 384: (16, 16), 512: (6, 18), 768: (6, 18), 1024: (5, 5), 1536: (18, 6), 2048: (18, 5),
            4096: (18, 5)}
    for side, (w_rect, w_amp) in want.items():
        assert lib.ctv_default_config(side, side, 200, 0, ctypes.byref(rect)) == w_rect, side
        assert lib.ctv_default_config(side, side, 200, 0, ctypes.byref(amp)) == w_amp, side
    assert lib.ctv_default_config(2048, 2048, 200, 0, None) == 5   # no constraint: as the amplitude bound
