"""Autotuning of the fused FGP pass configuration (C calls ctv_autotune_denoise,
ctv_tune_get / ctv_tune_set), with a JSON cache per GPU name.

The cache file is $CTV_TUNE_CACHE, else ~/.cache/ctv_tune.json; it maps a GPU
name to {"<size class>/<tv type>": config}.
"""
from __future__ import annotations

import ctypes as C
import json
import os
from typing import Dict, Optional

import torch

from . import _lib as L
from .api import NO_CONSTRAINT, Constraint, _check_image, _stream_ptr, make_opts, tv_code, workspace

NUM_CLASSES = 40


def cache_path() -> str:
    return os.environ.get("CTV_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ctv_tune.json"))


def autotune(b: torch.Tensor, lam: float, tv="tv1_iso", iters: int = 100, C_: Optional[Constraint] = Constraint(),
             alpha: float = 0.5, repeats: int = 2) -> Dict[str, object]:
    """Time every configuration on this image (iters iterations each) and make
    the fastest the default for its size class and TV type."""
    lib = L.load()
    _check_image(b, "b", 2)
    m, n = b.shape
    x = torch.empty_like(b)
    ws = workspace(1, m, n, b.device)
    cc, keep = (C_ or NO_CONSTRAINT).to_c()
    opts = make_opts(iters, alpha=alpha)
    ncfg = lib.ctv_num_configs()
    times = (C.c_float * ncfg)()
    best = C.c_int(-1)
    L.check("ctv_autotune_denoise", lib.ctv_autotune_denoise(
        b.data_ptr(), x.data_ptr(), m, n, b.stride(0), float(lam), C.byref(cc), tv_code(tv), C.byref(opts),
        ws.data_ptr(), ws.numel(), int(repeats), C.byref(best), times, _stream_ptr()))
    del keep
    return {"best": best.value, "times_ms": list(times), "size_class": lib.ctv_size_class(m, n)}


def table() -> Dict[str, int]:
    lib = L.load()
    out = {}
    v = C.c_int()
    for sc in range(NUM_CLASSES):
        for tv in range(4):
            L.check("ctv_tune_get", lib.ctv_tune_get(sc, tv, C.byref(v)))
            if v.value >= 0:
                out["%d/%d" % (sc, tv)] = v.value
    return out


def save(path: Optional[str] = None) -> str:
    path = path or cache_path()
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[torch.cuda.get_device_name()] = table()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    return path


def load(path: Optional[str] = None) -> int:
    """Install the cached choices for this GPU; returns how many were loaded."""
    lib = L.load()
    path = path or cache_path()
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        data = json.load(f).get(torch.cuda.get_device_name(), {})
    for key, cfg in data.items():
        sc, tv = (int(v) for v in key.split("/"))
        L.check("ctv_tune_set", lib.ctv_tune_set(sc, tv, int(cfg)))
    return len(data)
