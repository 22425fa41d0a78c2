"""Python entry points over the C ABI (argument marshalling only).

``ctv_denoise`` / ``ctv_denoise_batched`` mirror the C calls of the same names
on torch tensors; ``denoise`` is the convenience form. torch supplies device
memory and the current stream; all arithmetic runs in ``libctv.so``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple, Union

import torch

from . import _lib as L

TV_TYPES = {"tv1_iso": 0, "tv1_aniso": 1, "tv2_iso": 2, "tv2_aniso": 3}


def tv_code(tv: Union[str, int]) -> int:
    if isinstance(tv, str):
        if tv not in TV_TYPES:
            raise ValueError("unknown TV type %r (one of %s)" % (tv, ", ".join(TV_TYPES)))
        return TV_TYPES[tv]
    return int(tv)


@dataclass
class Constraint:
    """The set C of problem (1): |x| <= amp_max (None: no bound; Eq. (25) uses 1),
    or a box (re_lo, re_hi, im_lo, im_hi) on the real and imaginary parts (give
    amp_max=None with it), and an optional support rectangle (j0, k0, j1, k1)
    (half-open) or support mask (CUDA uint8/bool tensor, nonzero = inside)."""
    amp_max: Optional[float] = 1.0
    rect: Optional[Tuple[int, int, int, int]] = None
    mask: Optional[torch.Tensor] = None
    box: Optional[Tuple[float, float, float, float]] = None

    def to_c(self) -> Tuple[L.CtvConstraint, object]:
        c = L.CtvConstraint()
        if self.amp_max is not None:
            c.amp_bound, c.amp_max = 1, float(self.amp_max)
        if self.box is not None:
            c.box = 1
            c.box_re[0], c.box_re[1], c.box_im[0], c.box_im[1] = (float(v) for v in self.box)
        keep = None
        if self.rect is not None:
            c.support_kind = 1
            for i, v in enumerate(self.rect):
                c.rect[i] = int(v)
        elif self.mask is not None:
            mk = self.mask
            if mk.dtype == torch.bool:
                mk = mk.to(torch.uint8)
            if not mk.is_cuda or mk.dim() != 2 or mk.stride(1) != 1:
                raise ValueError("mask must be a 2-D CUDA tensor with unit column stride")
            c.support_kind, c.mask, c.mask_ld = 2, mk.data_ptr(), mk.stride(0)
            keep = mk
        return c, keep


NO_CONSTRAINT = Constraint(amp_max=None)


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def make_opts(iters: int, check_every: int = 0, gap_tol: float = 0.0, alpha: float = 0.5,
              warm_start: bool = False, config: int = -1, plain_gp: bool = False) -> L.CtvOpts:
    o = L.CtvOpts()
    o.max_iters, o.check_every, o.gap_tol = int(iters), int(check_every), float(gap_tol)
    o.alpha, o.warm_start, o.config = float(alpha), int(bool(warm_start)), int(config)
    o.plain_gp = int(bool(plain_gp))
    return o


def _check_image(t: torch.Tensor, name: str, ndim: int):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.complex64:
        raise ValueError("%s must be complex64" % name)
    if t.dim() != ndim or t.stride(-1) != 1:
        raise ValueError("%s must be %d-D with unit column stride" % (name, ndim))


def get_last_error(stream=None) -> int:
    """The C call ``ctv_get_last_error``: synchronises the stream and returns (and
    clears) the first asynchronous error recorded on the current device, e.g.
    CTV_ENONFINITE (5) for a NaN or infinity in an input image; 0 if none."""
    return int(L.load().ctv_get_last_error(_stream_ptr(stream)))


def workspace(batch: int, m: int, n: int, device) -> torch.Tensor:
    lib = L.load()
    nbytes = lib.ctv_denoise_workspace_size(batch, m, n)
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def ctv_denoise(b: torch.Tensor, x: torch.Tensor, lam: float, C: Optional[Constraint], tv_type,
                opts: L.CtvOpts, dual_state: Optional[torch.Tensor] = None,
                ws: Optional[torch.Tensor] = None, want_stats: bool = False, stream=None):
    """One image: the C call ``ctv_denoise`` on tensors. Returns a stats dict
    when want_stats (this synchronises the stream), else None."""
    lib = L.load()
    _check_image(b, "b", 2)
    _check_image(x, "x", 2)
    m, n = b.shape
    if x.shape != b.shape or x.stride(0) != b.stride(0):
        raise ValueError("x must have b's shape and row stride")
    if dual_state is not None and (dual_state.dtype != torch.float32 or not dual_state.is_contiguous()
                                   or dual_state.numel() != 4 * m * n):
        raise ValueError("dual_state must be a contiguous float32 tensor of 4*m*n values")
    if ws is None:
        ws = workspace(1, m, n, b.device)
    cc, keep = (C or NO_CONSTRAINT).to_c()
    st = L.CtvStats()
    status = lib.ctv_denoise(b.data_ptr(), x.data_ptr(), m, n, b.stride(0), float(lam), C_ref(cc),
                             tv_code(tv_type), C_ref(opts),
                             dual_state.data_ptr() if dual_state is not None else None,
                             ws.data_ptr(), ws.numel(), C_ref(st) if want_stats else None,
                             _stream_ptr(stream))
    L.check("ctv_denoise", status)
    del keep
    return st.as_dict() if want_stats else None


def ctv_denoise_batched(b: torch.Tensor, x: torch.Tensor, lams: torch.Tensor, C: Optional[Constraint],
                        tv_type, opts: L.CtvOpts, dual_state: Optional[torch.Tensor] = None,
                        ws: Optional[torch.Tensor] = None, want_stats: bool = False, stream=None):
    """Equally sized batch (B, m, n) with per-image lambda (CUDA float32 tensor
    of B values): the C call ``ctv_denoise_batched``."""
    lib = L.load()
    _check_image(b, "b", 3)
    _check_image(x, "x", 3)
    B, m, n = b.shape
    if x.shape != b.shape or x.stride() != b.stride():
        raise ValueError("x must have b's shape and strides")
    if not (lams.is_cuda and lams.dtype == torch.float32 and lams.numel() == B and lams.is_contiguous()):
        raise ValueError("lams must be a contiguous CUDA float32 tensor with one value per image")
    if dual_state is not None and (dual_state.dtype != torch.float32 or not dual_state.is_contiguous()
                                   or dual_state.numel() != 4 * B * m * n):
        raise ValueError("dual_state must be a contiguous float32 tensor of 4*B*m*n values")
    if ws is None:
        ws = workspace(B, m, n, b.device)
    cc, keep = (C or NO_CONSTRAINT).to_c()
    st = (L.CtvStats * B)()
    status = lib.ctv_denoise_batched(b.data_ptr(), x.data_ptr(), B, m, n, b.stride(1), b.stride(0),
                                     lams.data_ptr(), C_ref(cc), tv_code(tv_type), C_ref(opts),
                                     dual_state.data_ptr() if dual_state is not None else None,
                                     ws.data_ptr(), ws.numel(), st if want_stats else None,
                                     _stream_ptr(stream))
    L.check("ctv_denoise_batched", status)
    del keep
    return [s.as_dict() for s in st] if want_stats else None


def C_ref(obj):
    return C.byref(obj)


def denoise(b: torch.Tensor, lam, tv: Union[str, int] = "tv1_iso", iters: int = 100,
            C: Optional[Constraint] = Constraint(), alpha: float = 0.5, check_every: int = 0,
            gap_tol: float = 0.0, dual_state: Optional[torch.Tensor] = None, warm_start: bool = False,
            config: int = -1, return_stats: bool = False, out: Optional[torch.Tensor] = None,
            plain_gp: bool = False):
    """Solve problem (1) for one complex64 image (m, n) or a batch (B, m, n).

    lam: a float, or for a batch a float / CUDA float32 tensor of B values.
    plain_gp: run the gradient projection of Eq. (21) instead of Algorithm 2.
    Returns x (and the statistics when return_stats)."""
    opts = make_opts(iters, check_every, gap_tol, alpha, warm_start, config, plain_gp)
    x = out if out is not None else torch.empty_like(b)
    if b.dim() == 2:
        st = ctv_denoise(b, x, float(lam), C, tv, opts, dual_state, want_stats=return_stats)
    elif b.dim() == 3:
        if isinstance(lam, torch.Tensor):
            lams = lam.to(device=b.device, dtype=torch.float32).contiguous()
        else:
            lams = torch.full((b.shape[0],), float(lam), dtype=torch.float32, device=b.device)
        st = ctv_denoise_batched(b, x, lams, C, tv, opts, dual_state, want_stats=return_stats)
    else:
        raise ValueError("b must be (m, n) or (B, m, n)")
    return (x, st) if return_stats else x


def configs():
    lib = L.load()
    out = []
    for i in range(lib.ctv_num_configs()):
        T, W, H, NT = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        L.check("ctv_config_info", lib.ctv_config_info(i, C.byref(T), C.byref(W), C.byref(H), C.byref(NT)))
        out.append({"config": i, "iters_per_pass": T.value, "region_w": W.value, "region_h": H.value,
                    "threads": NT.value})
    return out


# ----------------------------------------------------------------------------- phase retrieval
class PRPlan:
    """cuFFT plan and device buffers for phase retrieval of an m x n object on an
    M x N padded grid (C calls ctv_pr_plan_create / ctv_pr_plan_destroy)."""

    def __init__(self, m: int, n: int, M: int, N: int):
        self._lib = L.load()
        h = C.c_void_p()
        L.check("ctv_pr_plan_create", self._lib.ctv_pr_plan_create(m, n, M, N, C.byref(h)))
        self.handle = h
        self.m, self.n, self.M, self.N = m, n, M, N

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.ctv_pr_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, z, sqrt_y, H):
        _check_image(z, "z", 2)
        if z.shape != (self.m, self.n) or not z.is_contiguous():
            raise ValueError("z must be a contiguous (m, n) complex64 CUDA tensor")
        if sqrt_y.shape != (self.m, self.n) or sqrt_y.dtype != torch.float32 or not sqrt_y.is_contiguous() \
                or not sqrt_y.is_cuda:
            raise ValueError("sqrt_y must be a contiguous (m, n) float32 CUDA tensor")
        if H.shape != (self.M, self.N) or H.dtype != torch.complex64 or not H.is_contiguous() or not H.is_cuda:
            raise ValueError("H must be a contiguous (M, N) complex64 CUDA tensor")

    def gradient(self, z: torch.Tensor, sqrt_y: torch.Tensor, H: torch.Tensor, stream=None):
        """grad F(z) of Eq. (27) and F(z) of Eq. (24) (ctv_pr_gradient)."""
        self._check(z, sqrt_y, H)
        g = torch.empty_like(z)
        loss = torch.zeros(1, dtype=torch.float64, device=z.device)
        L.check("ctv_pr_gradient", self._lib.ctv_pr_gradient(self.handle, z.data_ptr(), sqrt_y.data_ptr(),
                                                             H.data_ptr(), g.data_ptr(), loss.data_ptr(),
                                                             _stream_ptr(stream)))
        return g, loss

    def solve(self, x0: torch.Tensor, sqrt_y: torch.Tensor, H: torch.Tensor, tau: float, gamma: float = 1.0,
              C: Optional[Constraint] = Constraint(), tv: Union[str, int] = "tv1_aniso", inner_iters: int = 10,
              outer_iters: int = 300, alpha: float = 0.5, accelerate: bool = True, config: int = -1,
              return_loss: bool = False, out: Optional[torch.Tensor] = None, stream=None):
        """Algorithm 1 (or ISTA) from x0; returns x_K (and F(z_k) per outer iteration)."""
        self._check(x0, sqrt_y, H)
        x = out if out is not None else x0.clone()
        if out is not None:
            x.copy_(x0)
        hist = torch.zeros(max(outer_iters, 1), dtype=torch.float64, device=x0.device) if return_loss else None
        cc, keep = (C or NO_CONSTRAINT).to_c()
        opts = make_opts(inner_iters, 0, 0.0, alpha, False, config)
        L.check("ctv_pr_solve", self._lib.ctv_pr_solve(self.handle, sqrt_y.data_ptr(), H.data_ptr(), float(tau),
                                                       float(gamma), C_ref(cc),
                                                       tv_code(tv), C_ref(opts), int(outer_iters),
                                                       int(bool(accelerate)), x.data_ptr(),
                                                       hist.data_ptr() if hist is not None else None,
                                                       _stream_ptr(stream)))
        del keep
        return (x, hist[:outer_iters]) if return_loss else x

    solve_ls = None   # bound below


def _solve_ls(self, x0: torch.Tensor, sqrt_y: torch.Tensor, H: torch.Tensor, tau: float, gamma0: float = 1.0,
              eta: float = 0.5, C: Optional[Constraint] = Constraint(), tv: Union[str, int] = "tv1_aniso",
              inner_iters: int = 10, outer_iters: int = 300, alpha: float = 0.5, accelerate: bool = True,
              config: int = -1, stream=None):
    """Algorithm 1 (or ISTA) with backtracking on the step (C call ctv_pr_solve_ls).
    Returns (x_K, F(z_k) per outer iteration, accepted steps)."""
    self._check(x0, sqrt_y, H)
    x = x0.clone()
    hist = torch.zeros(max(outer_iters, 1), dtype=torch.float64, device=x0.device)
    gam = (L.c_float * max(outer_iters, 1))()
    cc, keep = (C or NO_CONSTRAINT).to_c()
    opts = make_opts(inner_iters, 0, 0.0, alpha, False, config)
    L.check("ctv_pr_solve_ls", self._lib.ctv_pr_solve_ls(
        self.handle, sqrt_y.data_ptr(), H.data_ptr(), float(tau), float(gamma0), float(eta), C_ref(cc),
        tv_code(tv), C_ref(opts), int(outer_iters), int(bool(accelerate)), x.data_ptr(), hist.data_ptr(), gam,
        _stream_ptr(stream)))
    del keep
    return x, hist[:outer_iters], list(gam)[:outer_iters]


def ip_solve(plan: "PRPlan", x0: torch.Tensor, sqrt_y: torch.Tensor, H: torch.Tensor, outer_iters: int,
             C: Optional[Constraint] = Constraint(), return_loss: bool = False):
    """The iterative-projection comparator of Sec. VI-A: x <- P_C(x - grad F(x))
    (for a unitary propagator this is P_C(A^*(sqrt(y) A x / |A x|)), alternating
    projections onto the measured modulus and onto C). It is ISTA with tau = 0 and
    gamma = 1, so it runs through ctv_pr_solve."""
    return plan.solve(x0, sqrt_y, H, 0.0, 1.0, C, "tv1_aniso", 1, outer_iters, accelerate=False,
                      return_loss=return_loss)


def ctv_prox_grad_step(z: torch.Tensor, grad: torch.Tensor, gamma: float, tau: float, C: Optional[Constraint],
                       tv_type, opts: L.CtvOpts, dual_state: Optional[torch.Tensor], x_prev: torch.Tensor,
                       x_out: torch.Tensor, z_next: torch.Tensor, beta: float, stream=None):
    """One proximal-gradient step of problem (2) with a caller-supplied gradient
    (C call ctv_prox_grad_step)."""
    lib = L.load()
    for t, nm in ((z, "z"), (grad, "grad"), (x_prev, "x_prev"), (x_out, "x_out"), (z_next, "z_next")):
        _check_image(t, nm, 2)
        if not t.is_contiguous() or t.shape != z.shape:
            raise ValueError("%s must be contiguous with z's shape" % nm)
    m, n = z.shape
    ws = torch.empty(max(int(lib.ctv_prox_grad_workspace_size(m, n)), 256), dtype=torch.uint8, device=z.device)
    cc, keep = (C or NO_CONSTRAINT).to_c()
    L.check("ctv_prox_grad_step", lib.ctv_prox_grad_step(
        z.data_ptr(), grad.data_ptr(), float(gamma), float(tau), C_ref(cc), tv_code(tv_type), C_ref(opts),
        dual_state.data_ptr() if dual_state is not None else None, x_prev.data_ptr(), x_out.data_ptr(),
        z_next.data_ptr(), float(beta), m, n, ws.data_ptr(), ws.numel(), _stream_ptr(stream)))
    del keep


# ----------------------------------------------------------------------------- batched plans
class Plan:
    """Batched denoising of images of uneven sizes in one graph replay
    (C calls ctv_plan_create / ctv_plan_execute / ctv_plan_stats).

    images: sequence of dicts with keys b (complex64 CUDA (m, n)), x (output,
    same shape and row stride), lam, and optionally tv, alpha, C."""

    def __init__(self, images: Sequence[dict], iters: int, check_every: int = 0, gap_tol: float = 0.0,
                 config: Union[int, str] = -1):
        # config: -1 the default, a plan configuration, or "auto" to time every plan
        # configuration on these images and keep the fastest (CTV_CONFIG_AUTOTUNE)
        if config == "auto":
            config = -2
        self._lib = L.load()
        n = len(images)
        arr = (L.CtvImageDesc * n)()
        self._keep = []
        for i, im in enumerate(images):
            b, x = im["b"], im["x"]
            _check_image(b, "b", 2)
            _check_image(x, "x", 2)
            if x.shape != b.shape or x.stride(0) != b.stride(0):
                raise ValueError("x must have b's shape and row stride")
            d = arr[i]
            d.b, d.x = b.data_ptr(), x.data_ptr()
            d.m, d.n, d.ld = b.shape[0], b.shape[1], b.stride(0)
            d.lam = float(im["lam"])
            d.alpha = float(im.get("alpha", 0.5))
            d.tv_type = tv_code(im.get("tv", "tv1_iso"))
            cc, keep = (im.get("C", Constraint()) or NO_CONSTRAINT).to_c()
            d.C = cc
            self._keep += [b, x, keep]
        opts = make_opts(iters, check_every, gap_tol, 0.5, False, config)
        h = C.c_void_p()
        L.check("ctv_plan_create", self._lib.ctv_plan_create(arr, n, C.byref(opts), C.byref(h)))
        self.handle = h
        self.count = n

    def execute(self, stream=None):
        L.check("ctv_plan_execute", self._lib.ctv_plan_execute(self.handle, _stream_ptr(stream)))

    def stats(self, stream=None):
        st = (L.CtvStats * self.count)()
        L.check("ctv_plan_stats", self._lib.ctv_plan_stats(self.handle, st, _stream_ptr(stream)))
        return [s.as_dict() for s in st]

    def info(self):
        cfg, nl, pi, nb = C.c_int(), C.c_int(), C.c_double(), C.c_size_t()
        L.check("ctv_plan_info", self._lib.ctv_plan_info(self.handle, C.byref(cfg), C.byref(nl), C.byref(pi),
                                                         C.byref(nb)))
        return {"config": cfg.value, "launches_per_execute": nl.value, "pixel_iters": pi.value,
                "device_bytes": nb.value}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.ctv_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- differentiation
def _unrolled_checks(b, lams):
    _check_image(b, "b", 3)
    if not b.is_contiguous():
        raise ValueError("b must be contiguous (B, m, n)")
    if not (lams.is_cuda and lams.dtype == torch.float32 and lams.numel() == b.shape[0] and lams.is_contiguous()):
        raise ValueError("lams must be a contiguous CUDA float32 tensor with one value per image")


class UnrolledFGP(torch.autograd.Function):
    """x = K unrolled iterations of Algorithm 2 followed by Eq. (18), for a batch
    (B, m, n) of complex64 images and per-image lambda, differentiable with
    respect to b and lambda through the library's adjoint kernels (C calls
    ctv_unrolled_forward / ctv_unrolled_backward). Gradients follow torch's
    convention for real losses of complex tensors: dL/dRe + i dL/dIm."""

    @staticmethod
    def forward(ctx, b, lams, tv, iters, C, alpha, ckpt_every, config):
        lib = L.load()
        b = b.contiguous()
        lams = lams.contiguous()
        _unrolled_checks(b, lams)
        B, m, n = b.shape
        nbytes = int(lib.ctv_unrolled_workspace_size(B, m, n, int(iters), int(ckpt_every)))
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=b.device)
        x = torch.empty_like(b)
        cc, keep = (C or NO_CONSTRAINT).to_c()
        opts = make_opts(iters, 0, 0.0, alpha, False, config)
        L.check("ctv_unrolled_forward", lib.ctv_unrolled_forward(
            b.data_ptr(), x.data_ptr(), B, m, n, lams.data_ptr(), C_ref(cc), tv_code(tv), C_ref(opts),
            int(ckpt_every), ws.data_ptr(), ws.numel(), _stream_ptr()))
        ctx.save_for_backward(b, lams)
        ctx.ws, ctx.keep, ctx.cc, ctx.opts = ws, keep, cc, opts
        ctx.meta = (tv_code(tv), int(ckpt_every))
        return x

    @staticmethod
    def backward(ctx, xbar):
        lib = L.load()
        b, lams = ctx.saved_tensors
        B, m, n = b.shape
        xbar = xbar.to(torch.complex64).contiguous()
        bbar = torch.empty_like(b)
        lbar = torch.empty(B, dtype=torch.float32, device=b.device)
        tv, ck = ctx.meta
        L.check("ctv_unrolled_backward", lib.ctv_unrolled_backward(
            b.data_ptr(), xbar.data_ptr(), bbar.data_ptr(), lbar.data_ptr(), B, m, n, lams.data_ptr(),
            C_ref(ctx.cc), tv, C_ref(ctx.opts), ck, ctx.ws.data_ptr(), ctx.ws.numel(), _stream_ptr()))
        return bbar, lbar, None, None, None, None, None, None


def denoise_unrolled(b: torch.Tensor, lams, tv: Union[str, int] = "tv1_iso", iters: int = 50,
                     C: Optional[Constraint] = Constraint(), alpha: float = 0.5, ckpt_every: int = 10,
                     config: int = -1) -> torch.Tensor:
    """Differentiable form of ``denoise`` for a batch (B, m, n) (or one (m, n) image)."""
    squeeze = b.dim() == 2
    bb = b.unsqueeze(0) if squeeze else b
    if not isinstance(lams, torch.Tensor):
        lams = torch.full((bb.shape[0],), float(lams), dtype=torch.float32, device=b.device)
    lams = lams.to(device=b.device, dtype=torch.float32).reshape(-1)
    x = UnrolledFGP.apply(bb, lams, tv, iters, C, alpha, ckpt_every, config)
    return x.squeeze(0) if squeeze else x


PRPlan.solve_ls = _solve_ls
