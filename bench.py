#!/usr/bin/env python
"""Throughput of complex constrained TV denoising (Algorithm 2) on GB300.

One step = the whole fused FGP path (passes + gap/finalize) for the four TV
types of Eq. (7)-(10) on one 2048 x 2048 complex64 phantom, 200 iterations each,
C = {|x| <= 1} with a rectangular support. Successive steps cycle through the
nine (sigma, lambda) pairs sigma in {0.05, 0.1, 0.2}, lambda in {0.02, 0.05, 0.1}.
Inputs are resident in HBM and every solve's working set (b, two dual buffer
pairs: ~288 MB) is larger than the 129 MB L2, so no flush is needed.

Prints one JSON line (rank 0). --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "complex-TV FGP Gpixel-iter/s, % HBM roofline, batched vs looped at tol"
UNIT = "Gpixel-iter/s"
M = N = 2048
ITERS = 200
SIGMAS = (0.05, 0.1, 0.2)
LAMS = (0.02, 0.05, 0.1)
TVS = ("tv1_iso", "tv1_aniso", "tv2_iso", "tv2_aniso")
ALGO_BYTES_PER_PX_IT = 72   # b 8 + r 16 + q_prev 16 read, q 16 + r' 16 written
WORKLOAD = ("2048x2048 complex64 phantoms (12 rectangles/disks, CN noise), 4 TV types x "
            "9 (sigma, lambda) pairs, 200 FGP iterations per solve (gap stopping off), "
            "C = |x|<=1 + rect support [m/8,7m/8)x[n/8,7n/8)")


def combos():
    return [(s, l) for s in SIGMAS for l in LAMS]


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in ("paper_2109_05496_gb300/csrc/ctv_device.cuh", "paper_2109_05496_gb300/csrc/pass_tv.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(cfg_geom: str, units_per_launch: float):
    """DRAM bytes per launch of the fused pass from the committed ncu summaries,
    scaled to this launch's pixel-iterations; None if the kernel source or the
    configuration's geometry changed since the counters were taken."""
    import glob
    want = kernel_source_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for ln in open(path).read().splitlines():
            if not ln.startswith("bench-traffic:"):
                continue
            kv = dict(p.split("=", 1) for p in ln.split()[1:])
            if kv.get("kernel_sha") != want or kv.get("geometry") != cfg_geom:
                continue
            per_unit = float(kv["dram_bytes_per_launch"]) / float(kv["pixel_iters_per_launch"])
            return per_unit * units_per_launch
    return None


def config_geometry(lib, cfg: int) -> str:
    import ctypes
    v = [ctypes.c_int() for _ in range(4)]
    lib.ctv_config_info(cfg, *[ctypes.byref(x) for x in v])
    return "T%d-%dx%d-%d" % tuple(x.value for x in v)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------- inputs
def make_inputs(rank: int):
    import numpy as np
    from phantoms import noisy_phantom, support_rect, to_c64
    imgs = []
    for i, (sigma, _) in enumerate(combos()):
        _, noisy = noisy_phantom(M, N, sigma, seed=1000 + 97 * rank + i)
        imgs.append(to_c64(noisy))
    return imgs, support_rect(M, N)


# ----------------------------------------------------------------------------- CPU oracle sample
def oracle_sample(imgs, rect, step: int, crop: int):
    """The oracle on a crop x crop window of one step's image and one TV type.
    Returns (pixel-iterations, seconds, threads)."""
    import numpy as np
    import torch
    from oracle.fgp import fgp
    from oracle.ops import Constraint as OC
    ci = step % len(imgs)
    sigma, lam = combos()[ci]
    tv = TVS[step % 4]
    j0 = (M - crop) // 2
    b = imgs[ci][j0:j0 + crop, j0:j0 + crop].astype(np.complex128)
    wr = (max(rect[0] - j0, 0), max(rect[1] - j0, 0), min(rect[2] - j0, crop), min(rect[3] - j0, crop))
    bt = torch.as_tensor(b)
    t0 = time.perf_counter()
    fgp((bt.real.clone(), bt.imag.clone()), float(np.float32(lam)), ITERS, tv, 0.5, OC(amp_max=1.0, rect=wr))
    dt = time.perf_counter() - t0
    return crop * crop * ITERS, dt, torch.get_num_threads()


# ----------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=18)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--config", type=int, default=-1, help="fused-pass configuration (-1: library default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-crop", type=int, default=512)
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the short runs of the other workloads after the headline")
    ap.add_argument("--workload", default="denoise2048",
                    choices=("denoise2048", "denoise2048_stop", "denoise256", "batched", "pr", "backward",
                             "pr_paper"),
                    help="denoise2048 is the headline line; the others measure the remaining workloads")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload != "denoise2048":
        return run_other_workload(args, world, rank, local)

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_05496_gb300 as ctv
    from paper_2109_05496_gb300 import _lib

    lib = _lib.load()
    dev = torch.device("cuda", local)
    imgs_np, rect = make_inputs(rank)
    imgs = [torch.from_numpy(a).to(dev) for a in imgs_np]
    xs = [torch.empty(M, N, dtype=torch.complex64, device=dev) for _ in TVS]
    ws = ctv.workspace(1, M, N, dev)
    C = ctv.Constraint(amp_max=1.0, rect=rect)
    opts = [ctv.make_opts(ITERS, 0, 0.0, 0.5, False, args.config) for _ in TVS]
    lams = [l for (_, l) in combos()]
    stream = torch.cuda.current_stream()

    def step(i, b=None, outs=None):
        ci = i % len(imgs)
        bb = imgs[ci] if b is None else b
        for t, tv in enumerate(TVS):
            ctv.ctv_denoise(bb, xs[t] if outs is None else outs[t], lams[ci], C, tv, opts[t], ws=ws)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    import ctypes
    lib.ctv_profile_enable(0)   # resets the launch counter; no timing events in the timed steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    sampler.stop()
    ms = e0.elapsed_time(e1)
    pass_ms, pass_n, units, all_n = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_longlong()
    lib.ctv_profile_read(ctypes.byref(pass_ms), ctypes.byref(pass_n), ctypes.byref(units), ctypes.byref(all_n))
    # the same steps again with each solve's run of fused-pass launches bracketed by two CUDA
    # events on its stream (the passes inside a run keep their back-to-back overlap), for the
    # roofline's kernel time per launch (kept out of the timed steps above)
    lib.ctv_profile_enable(2)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for i in range(args.steps):
        step(i)
    p1.record(stream)
    torch.cuda.synchronize()
    ms_profiled = p0.elapsed_time(p1)
    launches_timed = ctypes.c_longlong()
    lib.ctv_profile_read(ctypes.byref(pass_ms), ctypes.byref(pass_n), ctypes.byref(units),
                         ctypes.byref(launches_timed))
    lib.ctv_profile_enable(0)
    from paper_2109_05496_gb300 import dist as pdist
    ms = pdist.max_over_ranks(ms)
    px_it_step = len(TVS) * M * N * ITERS
    value = pdist.weak_scaling_value(args.steps * px_it_step, ms, world) / 1e9

    # end to end through the public API: pinned host input in, result back to pinned host, every step
    e2e = None
    if not args.no_e2e:
        # Copies run on their own stream, double-buffered: the input of step i + 1 goes up while
        # step i computes, and step i's results come down while step i + 1 computes.
        host_in = [torch.from_numpy(a).pin_memory() for a in imgs_np]
        host_out = [torch.empty(M, N, dtype=torch.complex64).pin_memory() for _ in TVS]
        din = [torch.empty(M, N, dtype=torch.complex64, device=dev) for _ in range(2)]
        dout = [[torch.empty(M, N, dtype=torch.complex64, device=dev) for _ in TVS] for _ in range(2)]
        cstream = torch.cuda.Stream(device=dev)
        done = [torch.cuda.Event() for _ in range(2)]      # step using slot s finished computing
        copied_in = [torch.cuda.Event() for _ in range(2)]
        copied_out = [torch.cuda.Event() for _ in range(2)]
        for e in done + copied_out:
            e.record(stream)

        def upload(i):
            sl = i % 2
            cstream.wait_event(done[sl])
            with torch.cuda.stream(cstream):
                din[sl].copy_(host_in[i % len(host_in)], non_blocking=True)
            copied_in[sl].record(cstream)

        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        upload(0)
        for i in range(args.steps):
            sl = i % 2
            if i + 1 < args.steps:
                upload(i + 1)
            stream.wait_event(copied_in[sl])
            stream.wait_event(copied_out[sl])
            step(i, b=din[sl], outs=dout[sl])
            done[sl].record(stream)
            cstream.wait_event(done[sl])
            with torch.cuda.stream(cstream):
                for t in range(len(TVS)):
                    host_out[t].copy_(dout[sl][t], non_blocking=True)
            copied_out[sl].record(cstream)
        stream.wait_stream(cstream)
        f1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = pdist.max_over_ranks(f0.elapsed_time(f1))
        e2e = {"value": pdist.weak_scaling_value(args.steps * px_it_step, ems, world) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": M * N * 8, "d2h_bytes_per_step": len(TVS) * M * N * 8}

    peak, peak_kind = read_peaks()
    per_launch_units = units.value / max(pass_n.value, 1)
    achieved = ALGO_BYTES_PER_PX_IT * units.value / (pass_ms.value * 1e-3) / 1e9 if pass_ms.value > 0 else None
    cfg_used = args.config if args.config >= 0 else default_config_id(lib, rect)
    traffic = profiled_traffic(config_geometry(lib, cfg_used), per_launch_units)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "kernel": "fgp_pass_kernel", "peak_source": peak_kind + " (hbm_gbs, copy)",
            "algorithmic_bytes_per_pixel_iter": ALGO_BYTES_PER_PX_IT,
            "pixel_iters_per_launch": per_launch_units,
            "avg_launch_us": pass_ms.value * 1e3 / max(pass_n.value, 1),
            "timing": "CUDA events around each solve's run of back-to-back pass launches (one run of "
                      "%d launches per solve), in a second pass over the timed steps" %
                      (pass_n.value // max(args.steps * len(TVS), 1)),
            "kernel_ms_per_step": pass_ms.value / args.steps,
            "kernel_share_of_step": pass_ms.value / ms_profiled if ms_profiled > 0 else None,
            "traffic_note": "ncu DRAM bytes per launch averaged over consecutive launches with "
                            "--cache-control none (a launch's dirty L2 lines are written back during the "
                            "next one)"}

    # the other workloads of the metric (batched vs looped; 256^2 latency; gap stopping;
    # phase retrieval; backward), each briefly, on rank 0 of a single-GPU run
    workloads = None
    if rank == 0 and world == 1 and not args.no_workloads:
        workloads = {}
        wl_steps = 5
        workloads["amp_only"] = measure_amp_only(ctv, dev, 10, 3, args.config)
        workloads["batched"] = measure_batched(ctv, dev, wl_steps, 3)
        workloads["denoise256"] = measure_denoise256(ctv, dev, 50, 3, [default_config_small(lib)])
        workloads["denoise2048_stop"] = measure_stop(ctv, dev, 2)
        workloads["pr"] = measure_pr(ctv, dev, 1)
        workloads["backward"] = measure_backward(ctv, dev, wl_steps, 3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        pxit, dt, threads = 0, 0.0, 1
        s = 0
        while dt < 10.0 and s < 8:
            a, b_, threads = oracle_sample(imgs_np, rect, s, args.cpu_crop)
            pxit += a
            dt += b_
            s += 1
        cpu = {"value": pxit / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d oracle solves of a %dx%d crop of the step images, 200 iterations each, "
                         "TV type cycling, FP64 PyTorch CPU" % (s, args.cpu_crop, args.cpu_crop)}
        # the same oracle on one host thread
        nt = torch.get_num_threads()
        torch.set_num_threads(1)
        a, b_, _ = oracle_sample(imgs_np, rect, 0, 128)
        torch.set_num_threads(nt)
        cpu["single_thread_value"] = a / b_ / 1e9
        cpu["single_thread_sample"] = "one oracle solve of a 128x128 crop, 200 iterations, TV1 iso, 1 thread"

    clocks = sampler.summary()
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD, "m": M, "n": N, "iters": ITERS, "tv_types": list(TVS),
                          "solves_per_step": len(TVS), "fused_pass_config": cfg_used,
                          "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if world > 1 else "single"},
               "e2e": e2e, "gpu_launches": int(all_n.value), "roofline": roof, "cpu_baseline": cpu,
               "clocks": clocks}
        if workloads is not None:
            bt = workloads["batched"]
            out["batched"] = {"value": bt["value"], "looped_value": bt["looped_value"],
                              "speedup_vs_loop": bt["speedup_vs_loop"],
                              "speedup_vs_loop_same_config": bt["speedup_vs_loop_same_config"],
                              "unit": UNIT, "accuracy": bt["accuracy"],
                              "workload": "512 complex64 images, sides log-uniform in [64, 1024], lambda ~ "
                                          "U[0.01, 0.1], mixed TV types, 100 iterations: one plan graph replay "
                                          "vs a per-image loop of ctv_denoise"}
            out["workloads"] = workloads
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def default_config_id(lib, rect) -> int:
    import ctypes
    from paper_2109_05496_gb300 import api
    cc, _ = api.Constraint(amp_max=1.0, rect=rect).to_c()
    return int(lib.ctv_default_config(M, N, ITERS, 0, ctypes.byref(cc)))


def default_config_small(lib) -> int:
    import ctypes
    from paper_2109_05496_gb300 import api
    cc, _ = api.Constraint(amp_max=1.0).to_c()
    return int(lib.ctv_default_config(256, 256, 100, 0, ctypes.byref(cc)))


# ----------------------------------------------------------------------------- other workloads
def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure_denoise256(ctv, dev, steps, warmup, configs):
    """C1: 256^2 phantom, sigma 0.1, lambda 0.05, |x| <= 1, TV1 iso, 100 iterations;
    plain calls and a CUDA graph, per configuration."""
    import torch
    from phantoms import noisy_phantom, to_c64
    _, noisy = noisy_phantom(256, 256, 0.1, seed=1)
    b = torch.from_numpy(to_c64(noisy)).to(dev)
    x = torch.empty_like(b)
    ws = ctv.workspace(1, 256, 256, dev)
    C = ctv.Constraint(amp_max=1.0)
    res = {}
    for cfg in configs:
        opts = ctv.make_opts(100, config=cfg)
        for _ in range(warmup):
            ctv.ctv_denoise(b, x, 0.05, C, "tv1_iso", opts, ws=ws)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        for _ in range(steps):
            ctv.ctv_denoise(b, x, 0.05, C, "tv1_iso", opts, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        plain_us = e0.elapsed_time(e1) * 1e3 / steps
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ctv.ctv_denoise(b, x, 0.05, C, "tv1_iso", opts, ws=ws)
        for _ in range(warmup):
            g.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_us = e0.elapsed_time(e1) * 1e3 / steps
        res[cfg] = {"us_per_solve": plain_us, "us_per_solve_graph": graph_us,
                    "gpx_it_s_graph": 256 * 256 * 100 / (graph_us * 1e-6) / 1e9}
    best = min(res, key=lambda c: res[c]["us_per_solve_graph"])
    return {"metric": "FGP 256x256 solve time (100 iterations)", "value": res[best]["us_per_solve_graph"],
            "unit": "us/solve", "higher_is_better": False, "configs": res, "best_config": best}


def measure_batched(ctv, dev, steps, warmup, config=-1):
    """C4: 512 images, sides log-uniform in [64, 1024], lambda ~ U[0.01, 0.1], mixed TV
    types, 100 iterations: one graph replay of a plan against a per-image loop of
    ctv_denoise. Equal accuracy: the same 100 iterations on every image; the loop
    with the plan's configuration reproduces the plan's x bit for bit, and the
    loop with each image's default configuration agrees with it within 1e-4 ||b||_inf."""
    import torch
    from phantoms import batch_params, batch_shapes, noisy_phantom, to_c64
    shapes = batch_shapes(512, 64, 1024, seed=2021)
    lams, types = batch_params(512, seed=2022)
    ims = []
    for i, (m, n) in enumerate(shapes):
        _, noisy = noisy_phantom(m, n, 0.1, seed=2021000 + i)
        bb = torch.from_numpy(to_c64(noisy)).to(dev)
        ims.append({"b": bb, "x": torch.empty_like(bb), "lam": float(lams[i]), "tv": TVS[int(types[i])],
                    "alpha": 0.5, "C": ctv.Constraint(amp_max=1.0)})
    plan = ctv.Plan(ims, 100, config=config)
    info = plan.info()
    for _ in range(warmup):
        plan.execute()
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    for _ in range(steps):
        plan.execute()
    e1.record()
    torch.cuda.synchronize()
    ms_plan = e0.elapsed_time(e1) / steps
    x_plan = [im["x"].clone() for im in ims]
    wss = {}
    for im in ims:
        key = tuple(im["b"].shape)
        if key not in wss:
            wss[key] = ctv.workspace(1, key[0], key[1], dev)

    def loop(opts):
        for im in ims:
            ctv.ctv_denoise(im["b"], im["x"], im["lam"], im["C"], im["tv"], opts, ws=wss[tuple(im["b"].shape)])

    def time_loop(opts, reps):
        loop(opts)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            loop(opts)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(1, steps // 3)
    # the loop a user writes: every image with the library's default configuration for its size
    ms_loop = time_loop(ctv.make_opts(100), reps)
    worst = 0.0
    for im, xp in zip(ims, x_plan):
        worst = max(worst, float((im["x"] - xp).abs().max()) / max(float(im["b"].abs().max()), 1e-30))
    # and the loop with the plan's own configuration
    ms_loop_same = time_loop(ctv.make_opts(100, config=info["config"]), reps)
    same_bits = all(torch.equal(im["x"], xp) for im, xp in zip(ims, x_plan))
    pxit = info["pixel_iters"]
    return {"metric": "batched FGP Gpixel-iter/s (512 uneven images, one graph replay) vs per-image loop",
            "value": pxit / (ms_plan * 1e-3) / 1e9, "unit": "Gpixel-iter/s", "higher_is_better": True,
            "ms_per_batch": ms_plan, "looped_ms_per_batch": ms_loop,
            "looped_value": pxit / (ms_loop * 1e-3) / 1e9, "speedup_vs_loop": ms_loop / ms_plan,
            "looped_same_config_ms_per_batch": ms_loop_same,
            "speedup_vs_loop_same_config": ms_loop_same / ms_plan,
            "accuracy": {"iterations": 100, "loop_same_config_bit_identical": same_bits,
                         "loop_default_config_max_dx_over_binf": worst, "tol": 1e-4},
            "plan": info, "images": 512, "megapixels": pxit / 100 / 1e6}


def measure_pr(ctv, dev, warmup):
    """C3: 1024^2 object, Fresnel TF (532 nm, 2 um, 5 mm), 2x padding, Poisson 1e4 photons,
    300 outer x 10 inner iterations, tau 0.01."""
    import ctypes
    import numpy as np
    import torch
    from paper_2109_05496_gb300 import _lib
    from phantoms import fresnel_tf, pr_object, simulate_intensity
    m = n = 1024
    Mp = Np = 2048
    H = fresnel_tf(Mp, Np, 532e-9, 2e-6, 5e-3).astype(np.complex64)
    x_gt = pr_object(m, n, seed=11)
    y = simulate_intensity(x_gt, H.astype(np.complex128), seed=12, photons=1e4)
    sqrt_y = torch.from_numpy(np.sqrt(y).astype(np.float32)).to(dev)
    Hg = torch.from_numpy(H).to(dev)
    plan = ctv.PRPlan(m, n, Mp, Np)
    x0 = torch.empty(m, n, dtype=torch.complex64, device=dev)
    g, _ = plan.gradient(torch.zeros_like(x0), sqrt_y, Hg)
    x0.copy_(-g)                    # A^* sqrt(y): the gradient at 0 is -A^*(sqrt(y))
    outer = 300
    C = ctv.Constraint(amp_max=1.0)
    # warm-up: full solves, long enough for the clocks to settle
    for _ in range(warmup):
        plan.solve(x0, sqrt_y, Hg, 0.01, 1.0, C, "tv1_aniso", 10, outer)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    xk, hist = plan.solve(x0, sqrt_y, Hg, 0.01, 1.0, C, "tv1_aniso", 10, outer, return_loss=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    xg = xk.cpu().numpy()
    ph = np.angle(xg * np.conj(x_gt))
    ph = np.angle(np.exp(1j * (ph - np.angle(np.exp(1j * ph).mean()))))
    ph0 = np.angle(x0.cpu().numpy() * np.conj(x_gt))
    ph0 = np.angle(np.exp(1j * (ph0 - np.angle(np.exp(1j * ph0).mean()))))
    h = hist.cpu().numpy()
    # where the time goes: the fused FGP pass runs (timed per run of passes in a second solve)
    # and one gradient evaluation (two 2048^2 FFT pairs, the fused residual and the adjoint crop)
    lib = _lib.load()
    lib.ctv_profile_enable(2)
    plan.solve(x0, sqrt_y, Hg, 0.01, 1.0, C, "tv1_aniso", 10, outer)
    pass_ms, pass_n, units, all_n = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_longlong()
    lib.ctv_profile_read(ctypes.byref(pass_ms), ctypes.byref(pass_n), ctypes.byref(units), ctypes.byref(all_n))
    lib.ctv_profile_enable(0)
    reps = 50
    g0, g1 = _events()
    g0.record()
    for _ in range(reps):
        plan.gradient(x0, sqrt_y, Hg)
    g1.record()
    torch.cuda.synchronize()
    grad_ms = g0.elapsed_time(g1) / reps
    return {"metric": "phase retrieval outer iterations/s (1024^2 object, 2048^2 FFTs, 10 FGP iterations each)",
            "value": outer / (ms * 1e-3), "unit": "outer-iter/s", "higher_is_better": True,
            "ms_total": ms, "fgp_pixel_iters": outer * 10 * m * n,
            "fgp_pass_ms_total": pass_ms.value,
            "fgp_pass_gpx_it_s": units.value / (pass_ms.value * 1e-3) / 1e9 if pass_ms.value > 0 else None,
            "gradient_ms_per_outer": grad_ms, "gradient_share": grad_ms * outer / ms,
            "fgp_pass_share": pass_ms.value / ms,
            "loss_first": float(h[0]), "loss_last": float(h[-1]),
            "phase_rmse_initial": float(np.sqrt((ph0 ** 2).mean())),
            "phase_rmse_final": float(np.sqrt((ph ** 2).mean()))}


def measure_stop(ctv, dev, steps, config=-1):
    """C2 with stopping: the 36 solves of the headline workload with the duality-gap
    test on (checked every 10 iterations, stop at gap <= 1e-6 P, at most 200
    iterations): iterations to stop and time per solve."""
    import numpy as np
    import torch
    imgs_np, rect = make_inputs(0)
    hm, hn = imgs_np[0].shape
    C = ctv.Constraint(amp_max=1.0, rect=rect)
    ws = ctv.workspace(1, hm, hn, dev)
    x = torch.empty(hm, hn, dtype=torch.complex64, device=dev)
    solves, tot_ms, tot_pxit = [], 0.0, 0.0
    for ci, (sigma, lam) in enumerate(combos()):
        b = torch.from_numpy(imgs_np[ci]).to(dev)
        for tv in TVS:
            opts = ctv.make_opts(ITERS, 10, 1e-6, 0.5, False, config)
            st = ctv.ctv_denoise(b, x, lam, C, tv, opts, ws=ws, want_stats=True)
            ctv.ctv_denoise(b, x, lam, C, tv, opts, ws=ws)   # the library builds its stop graph here
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record()
            for _ in range(steps):
                ctv.ctv_denoise(b, x, lam, C, tv, opts, ws=ws)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / steps
            solves.append({"sigma": sigma, "lambda": lam, "tv": tv, "k_stop": st["iters"],
                           "stopped": st["stopped"], "gap_rel": st["gap"] / max(st["primal"], 1e-30),
                           "ms": t})
            tot_ms += t
            tot_pxit += st["iters"] * hm * hn
    ks = [r["k_stop"] for r in solves]
    return {"metric": "2048^2 solves with duality-gap stopping (gap <= 1e-6 P, checked every 10)",
            "value": tot_ms / len(solves), "unit": "ms/solve", "higher_is_better": False,
            "k_stop_mean": float(np.mean(ks)), "k_stop_min": int(min(ks)), "k_stop_max": int(max(ks)),
            "stopped_before_200": int(sum(1 for r in solves if r["stopped"])),
            "gpx_it_s_effective": tot_pxit / (tot_ms * 1e-3) / 1e9, "solves": solves}


def measure_amp_only(ctv, dev, steps, warmup, config=-1):
    """The headline solves with C = {|x| <= 1} alone (no support rectangle): the
    same 4 TV types x 9 (sigma, lambda) images and 200 iterations, every tile
    running the full stencil (with the rectangle, tiles entirely outside it take
    the neighbour-free path where x = 0)."""
    import torch
    imgs_np, _ = make_inputs(0)
    imgs = [torch.from_numpy(a).to(dev) for a in imgs_np]
    xs = [torch.empty(M, N, dtype=torch.complex64, device=dev) for _ in TVS]
    ws = ctv.workspace(1, M, N, dev)
    C = ctv.Constraint(amp_max=1.0)
    opts = ctv.make_opts(ITERS, 0, 0.0, 0.5, False, config)
    lams = [l for (_, l) in combos()]

    def step(i):
        ci = i % len(imgs)
        for t, tv in enumerate(TVS):
            ctv.ctv_denoise(imgs[ci], xs[t], lams[ci], C, tv, opts, ws=ws)

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    for i in range(steps):
        step(i)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"metric": "headline solves with the amplitude bound only (no support rectangle)",
            "value": len(TVS) * M * N * ITERS / (ms * 1e-3) / 1e9, "unit": UNIT, "higher_is_better": True,
            "ms_per_step": ms}


def measure_backward(ctv, dev, steps, warmup, config=-1):
    """C5: 8 x 1024^2, 50 unrolled iterations, checkpoints every 10, loss ||x - x_gt||^2:
    backward / forward time."""
    import numpy as np
    import torch
    from phantoms import noisy_phantom, to_c64
    Bn, m, n, K = 8, 1024, 1024, 50
    cl, nz = [], []
    for i in range(Bn):
        c_, z_ = noisy_phantom(m, n, 0.1, seed=700 + i)
        cl.append(to_c64(c_))
        nz.append(to_c64(z_))
    b = torch.from_numpy(np.stack(nz)).to(dev).requires_grad_(True)
    gt = torch.from_numpy(np.stack(cl)).to(dev)
    lam = torch.linspace(0.02, 0.09, Bn, device=dev).requires_grad_(True)
    C = ctv.Constraint(amp_max=1.0)

    def fwd():
        return ctv.denoise_unrolled(b, lam, "tv1_iso", K, C, 0.5, 10, config)

    for _ in range(warmup):
        loss = ((fwd() - gt).abs() ** 2).sum()
        loss.backward()
    torch.cuda.synchronize()
    tf = tb = 0.0
    for _ in range(steps):
        e0, e1 = _events()
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record()
        x = fwd()
        e1.record()
        loss = ((x - gt).abs() ** 2).sum()
        e3 = torch.cuda.Event(enable_timing=True)
        e3.record()
        loss.backward()
        e2.record()
        torch.cuda.synchronize()
        tf += e0.elapsed_time(e1)
        tb += e3.elapsed_time(e2)
    tf /= steps
    tb /= steps
    return {"metric": "unrolled FGP backward/forward time ratio (8 x 1024^2, 50 iterations, ckpt 10)",
            "value": tb / tf, "unit": "ratio", "higher_is_better": False, "forward_ms": tf,
            "backward_ms": tb, "forward_gpx_it_s": Bn * m * n * K / (tf * 1e-3) / 1e9}


def measure_pr_paper(ctv, dev):
    """The paper's simulated setting (Sec. VI-A): 256^2 pure phase object (phase in [0, pi]),
    angular spectrum at 500 nm, 5 um pixels, 5 mm, 10% Gaussian intensity noise,
    back-propagated start, type-I anisotropic TV, 10 FGP iterations per outer
    iteration; IP vs TV (C = C^n) vs CTV."""
    import numpy as np
    import torch
    from phantoms import angular_spectrum_tf, intensity_with_gaussian_noise, phase_object, phase_rmse
    m = n = 256
    H = angular_spectrum_tf(m, n, 500e-9, 5e-6, 5e-3).astype(np.complex64)
    x_gt = phase_object(m, n, seed=31)
    y = intensity_with_gaussian_noise(x_gt, H.astype(np.complex128), 0.1, seed=32)
    sqrt_y = torch.from_numpy(np.sqrt(y).astype(np.float32)).to(dev)
    Hg = torch.from_numpy(H).to(dev)
    plan = ctv.PRPlan(m, n, m, n)
    g0, _ = plan.gradient(torch.zeros(m, n, dtype=torch.complex64, device=dev), sqrt_y, Hg)
    x0 = (-g0).contiguous()
    tau = 0.005
    curves = {}
    t0 = time.perf_counter()
    for name in ("IP", "TV", "CTV"):
        rm = []
        for K in range(10, 151, 10):      # the state after K outer iterations, from x_0 each time
            if name == "IP":
                x = ctv.api.ip_solve(plan, x0, sqrt_y, Hg, K, ctv.Constraint(amp_max=1.0))
            else:
                C = ctv.Constraint(amp_max=1.0) if name == "CTV" else ctv.NO_CONSTRAINT
                x = plan.solve(x0, sqrt_y, Hg, tau, 1.0, C, "tv1_aniso", 10, K)
            rm.append(phase_rmse(x.cpu().numpy(), x_gt))
        curves[name] = rm
    dt = time.perf_counter() - t0
    return {"metric": "phase RMSE (rad) after 50/100/150 outer iterations, paper's simulated setting",
            "value": curves["CTV"][-1], "unit": "rad", "higher_is_better": False,
            "rmse_initial": phase_rmse(x0.cpu().numpy(), x_gt),
            "rmse_at_50_100_150": {k: [v[4], v[9], v[14]] for k, v in curves.items()},
            "curves_every_10": curves, "tau": tau, "wall_s": dt}


def run_other_workload(args, world, rank, local):
    """Secondary measurements, one JSON line each (single GPU)."""
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_05496_gb300 as ctv
    dev = torch.device("cuda", local)
    out = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "data": "synthetic", "dtype": "f32",
           "workload": args.workload}
    if args.workload == "denoise256":
        cfgs = [args.config] if args.config >= 0 else list(range(ctv._lib.load().ctv_num_configs()))
        out.update(measure_denoise256(ctv, dev, args.steps, args.warmup, cfgs))
    elif args.workload == "batched":
        out.update(measure_batched(ctv, dev, args.steps, args.warmup, args.config if args.config >= 0 else -1))
    elif args.workload == "pr":
        out.update(measure_pr(ctv, dev, args.warmup))
    elif args.workload == "denoise2048_stop":
        out.update(measure_stop(ctv, dev, args.steps, args.config))
    elif args.workload == "pr_paper":
        out.update(measure_pr_paper(ctv, dev))
    elif args.workload == "backward":
        out.update(measure_backward(ctv, dev, args.steps, args.warmup, args.config if args.config >= 0 else -1))
    print(json.dumps(out))


def run_reference(args, world, rank):
    if rank != 0:
        return
    imgs_np, rect = make_inputs(0)
    for i in range(args.warmup):
        oracle_sample(imgs_np, rect, i, 128)
    pxit, dt, threads = 0, 0.0, 1
    for i in range(args.steps):
        a, b_, threads = oracle_sample(imgs_np, rect, i, 192)
        pxit += a
        dt += b_
    value = pxit / dt / 1e9
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "m": M, "n": N, "iters": ITERS,
                      "sample": "each step: one oracle solve of a 192x192 crop, 200 iterations"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": "one 192x192 crop solve (200 iterations) per step"}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
