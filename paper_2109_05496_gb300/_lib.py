"""ctypes binding of ``libctv.so`` (the C ABI declared in ``include/ctv.h``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels. Loading fails loudly when the library has not been built; there is no
fallback of any kind.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_int, c_float, c_double, c_size_t, c_void_p, c_longlong = C.c_int, C.c_float, C.c_double, C.c_size_t, C.c_void_p, C.c_longlong


class CtvConstraint(C.Structure):
    _fields_ = [("amp_bound", c_int), ("amp_max", c_float), ("support_kind", c_int),
                ("rect", c_int * 4), ("mask", c_void_p), ("mask_ld", c_int),
                ("box", c_int), ("box_re", c_float * 2), ("box_im", c_float * 2)]


class CtvOpts(C.Structure):
    _fields_ = [("max_iters", c_int), ("check_every", c_int), ("gap_tol", c_double),
                ("alpha", c_float), ("warm_start", c_int), ("config", c_int), ("plain_gp", c_int)]


class CtvStats(C.Structure):
    _fields_ = [("iters", c_int), ("stopped", c_int), ("primal", c_double), ("dual", c_double),
                ("gap", c_double), ("status", c_int)]

    def as_dict(self):
        return {"iters": self.iters, "stopped": bool(self.stopped), "primal": self.primal,
                "dual": self.dual, "gap": self.gap, "status": self.status}


class CtvImageDesc(C.Structure):
    _fields_ = [("b", c_void_p), ("x", c_void_p), ("m", c_int), ("n", c_int), ("ld", c_int),
                ("lam", c_float), ("alpha", c_float), ("tv_type", c_int), ("C", CtvConstraint)]


assert C.sizeof(CtvConstraint) == 64 and C.sizeof(CtvOpts) == 32 and C.sizeof(CtvStats) == 40


P = C.POINTER
# name -> (restype, argtypes); every symbol include/ctv.h declares
SIGNATURES = {
    "ctv_status_string": (C.c_char_p, [c_int]),
    "ctv_abi_version": (c_int, []),
    "ctv_get_last_error": (c_int, [c_void_p]),
    "ctv_num_configs": (c_int, []),
    "ctv_default_config": (c_int, [c_int, c_int, c_int, c_int, P(CtvConstraint)]),
    "ctv_config_info": (c_int, [c_int, P(c_int), P(c_int), P(c_int), P(c_int)]),
    "ctv_denoise_workspace_size": (c_size_t, [c_int, c_int, c_int]),
    "ctv_size_class": (c_int, [c_int, c_int]),
    "ctv_tune_get": (c_int, [c_int, c_int, P(c_int)]),
    "ctv_tune_set": (c_int, [c_int, c_int, c_int]),
    "ctv_autotune_denoise": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_float, P(CtvConstraint), c_int,
                                     P(CtvOpts), c_void_p, c_size_t, c_int, P(c_int), c_void_p, c_void_p]),
    "ctv_denoise": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_float, P(CtvConstraint), c_int,
                            P(CtvOpts), c_void_p, c_void_p, c_size_t, P(CtvStats), c_void_p]),
    "ctv_denoise_batched": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_longlong, c_void_p,
                                    P(CtvConstraint), c_int, P(CtvOpts), c_void_p, c_void_p, c_size_t,
                                    P(CtvStats), c_void_p]),
    "ctv_denoise_noalloc": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_float, P(CtvConstraint), c_int,
                                    P(CtvOpts), P(CtvStats), c_void_p]),
    "ctv_unrolled_workspace_size": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "ctv_unrolled_forward": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, P(CtvConstraint), c_int,
                                     P(CtvOpts), c_int, c_void_p, c_size_t, c_void_p]),
    "ctv_unrolled_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p,
                                      P(CtvConstraint), c_int, P(CtvOpts), c_int, c_void_p, c_size_t, c_void_p]),
    "ctv_plan_create": (c_int, [c_void_p, c_int, P(CtvOpts), P(c_void_p)]),
    "ctv_plan_execute": (c_int, [c_void_p, c_void_p]),
    "ctv_plan_stats": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ctv_plan_info": (c_int, [c_void_p, P(c_int), P(c_int), P(c_double), P(c_size_t)]),
    "ctv_plan_destroy": (None, [c_void_p]),
    "ctv_pr_plan_create": (c_int, [c_int, c_int, c_int, c_int, P(c_void_p)]),
    "ctv_pr_plan_destroy": (None, [c_void_p]),
    "ctv_pr_gradient": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ctv_pr_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_float, c_float, P(CtvConstraint), c_int,
                             P(CtvOpts), c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "ctv_pr_solve_ls": (c_int, [c_void_p, c_void_p, c_void_p, c_float, c_float, c_float, P(CtvConstraint), c_int,
                                P(CtvOpts), c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ctv_prox_grad_workspace_size": (c_size_t, [c_int, c_int]),
    "ctv_prox_grad_step": (c_int, [c_void_p, c_void_p, c_float, c_float, P(CtvConstraint), c_int, P(CtvOpts),
                                   c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_int, c_int, c_void_p,
                                   c_size_t, c_void_p]),
    "ctv_profile_enable": (c_int, [c_int]),
    "ctv_profile_read": (c_int, [P(c_double), P(C.c_longlong), P(c_double), P(C.c_longlong)]),
}


class CtvError(RuntimeError):
    def __init__(self, fn, status):
        lib = _lib
        msg = lib.ctv_status_string(status).decode() if lib is not None else str(status)
        super().__init__("%s failed: %s (status %d)" % (fn, msg, status))
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Return the loaded library, building it first when asked to."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path) or (build_if_missing and not _build.up_to_date()):
            if not build_if_missing:
                raise RuntimeError("libctv.so is not built (%s); run __graft_entry__.build() "
                                   "or python -m paper_2109_05496_gb300.build" % path)
            _build.build()
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(fn_name: str, status: int):
    if status != 0:
        raise CtvError(fn_name, status)
