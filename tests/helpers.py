"""Shared test helpers: layout conversions between the library's padded dual
(float4 per pixel) and the oracle's paper-shaped dual, and oracle runners."""
from __future__ import annotations

import numpy as np
import torch

from oracle.fgp import fgp, primal_value
from oracle.ops import DT, Constraint as OConstraint, in_S

TV_NAMES = ["tv1_iso", "tv1_aniso", "tv2_iso", "tv2_aniso"]


def f32(v: float) -> float:
    """The FP32 value the GPU computes with, promoted back to FP64."""
    return float(np.float32(v))


def dual_to_paper(d: torch.Tensor, m: int, n: int):
    """(m*n*4) float32 (r1, s1, r2, s2) per pixel -> (r1, r2, s1, s2) in the paper's shapes."""
    d = d.detach().reshape(m, n, 4).to("cpu", torch.float64)
    return (d[:-1, :, 0].clone(), d[:, :-1, 2].clone(), d[:-1, :, 1].clone(), d[:, :-1, 3].clone())


def dual_from_paper(q, m: int, n: int) -> torch.Tensor:
    r1, r2, s1, s2 = q
    d = torch.zeros(m, n, 4, dtype=torch.float64)
    d[:-1, :, 0] = r1
    d[:-1, :, 1] = s1
    d[:, :-1, 2] = r2
    d[:, :-1, 3] = s2
    return d.to(torch.float32).reshape(-1)


def padded_slots_zero(d: torch.Tensor, m: int, n: int) -> bool:
    d = d.detach().reshape(m, n, 4).cpu()
    return bool((d[m - 1, :, 0:2] == 0).all()) and bool((d[:, n - 1, 2:4] == 0).all())


def oracle_constraint(amp_max=1.0, rect=None, mask=None):
    return OConstraint(amp_max=amp_max, rect=rect, mask=None if mask is None else torch.as_tensor(mask).bool().cpu())


def run_oracle(b_c64: np.ndarray, lam: float, K: int, tv: str, alpha: float, C, q0=None, **kw):
    """Oracle on the FP32-rounded input promoted to FP64."""
    bb = torch.as_tensor(np.asarray(b_c64).astype(np.complex64).astype(np.complex128))
    b = (bb.real.clone(), bb.imag.clone())
    res = fgp(b, f32(lam), K, tv, f32(alpha), C, q0=q0, **kw)
    return b, res


def objective(x_c: np.ndarray, b, lam, tv, alpha) -> float:
    xt = torch.as_tensor(np.asarray(x_c).astype(np.complex128))
    return float(primal_value((xt.real.clone(), xt.imag.clone()), b, f32(lam), tv, f32(alpha)))


def _oracle_x_job(args):
    """x_K of the oracle for one image (a process-pool job)."""
    b_c64, lam, K, tv, alpha, amp_max = args
    torch.set_num_threads(1)
    _, res = run_oracle(b_c64, lam, K, tv, alpha, oracle_constraint(amp_max))
    return (res.x[0] + 1j * res.x[1]).numpy()


def oracle_x_many(jobs, workers: int = 0):
    """The oracle's x_K for many small images, (b_c64, lam, K, tv, alpha, amp_max)
    each, in a pool of spawned processes (a forked child of a process that has
    used the GPU is not safe; spawned ones start clean)."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_oracle_x_job, jobs, chunksize=2))
