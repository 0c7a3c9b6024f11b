#!/usr/bin/env python3
"""Benchmark of the NFFT nonlocal-denoising hot path (one JSON line).

A step is one pass of the whole path over one synthetic image: patch
features, the plan (torus map, sort by cell with the points' cell offsets,
multiplier tables, degrees), and a deflated Jacobi-PCG solve of
(alpha I + L) u = alpha f to relative residual 1e-6 in the mixed form
(FP32-NFFT inner solves, FP64-accurate refinement residuals).  The default
workload is the 2048 x 2048 image with 5x5 patches (9 windows, M = 64,
n_os = 128, m = 6) at sigma = 0.2; sigma = 0.1 and 0.4 are solved beside it.
The metric is NFFT matvec throughput in Gpts/s: point-windows (N * L per
matvec) pushed through the NFFT per second, over the whole step; the
seconds-to-solve of the mixed and the FP64-accurate forms are reported
beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (launched by torchrun): --shard windows (default) gives every rank a
contiguous range of the windows (Sec. 3: the ANOVA kernel is a mean of
independent per-window Gauss transforms); each matvec sums the ranks'
shares of Gamma_full x with one NCCL all-reduce and the Krylov scalars are
computed redundantly ("scaling": "strong").  --shard replicas runs N
independent replicas ("scaling": "weak").
--impl reference times the CPU FP64 oracle (direct O(N^2) sums) on the host
cores on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2407_06834_gb300.inputs import WORKLOADS  # noqa: E402

METRIC = "NFFT kernel matvec Gpts/s (whole features+plan+solve step, mixed form)"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
CSRC = os.path.join(ROOT, "paper_2407_06834_gb300", "csrc")
# Non-tensor ALU peaks derived from unit counts and the 2070 MHz max clock:
# FP32: 152 SMs x 128 FMA lanes x 2 flop; FP64: GB300 nominal 1.25 TFLOP/s.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = 1.25
# Inner tolerance of the mixed solves: 0 = the library's automatic policy
# (the first FP32 inner solve aims at the outer tolerance; a step the
# FP64-accurate residual does not certify is followed by a short one).
INNER_TOL = 0.0
# FP32 operations of one double-float stencil update (see roofline())
DF32_OPS_PER_UPDATE = 12
# DRAM bytes (read + write) per launch of the NFFT kernels, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the 2048 x 2048
# workload per coordinate mode (stored cell offsets, or recomputed from the
# image), keyed by a hash of the kernel sources at capture time: when the
# sources change, the figures no longer describe the kernels and the bench
# reports traffic null.
NCU_TRAFFIC = {"sources_sha16": "444583fc392f26ea", "workload": "img2048",
               "bytes_per_launch": {
                   "stored": {"spread32": 780996352, "interp32": 725467136,
                              "spread_df32": 1431011584, "interp_df32": 1294031104},
                   "image": {"spread32": 840602624, "interp32": 430556672,
                             "spread_df32": 1062125824, "interp_df32": 738703872}}}


def kernel_sources_sha16() -> str:
    """Hash of the sources the NFFT kernels are compiled from."""
    h = hashlib.sha256()
    for name in ("nfft.cu", "window.cuh", "common.cuh", "df32.cuh"):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    """The measured copy bandwidth and bf16 rate of the GB300s
    (MEASURED_PEAKS.json), else the profiling fallback (6.8 TB/s)."""
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s (no measured peaks file)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="img2048", choices=sorted(WORKLOADS))
    ap.add_argument("--shard", choices=["windows", "replicas"], default="windows",
                    help="N > 1: windows over ranks (one all-reduce per matvec) or replicas")
    ap.add_argument("--coords", choices=["stored", "image"], default="stored",
                    help="plans store each point's cell offsets (default) or recompute "
                         "the coordinates from the image")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=0, help="oracle row sample (0 = auto)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-form leg")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the side legs (512^2 line, learned, MIS, sweep)")
    ap.add_argument("--learned-triples", type=int, default=512,
                    help="training triples at 256x256 for the learned leg")
    ap.add_argument("--learned-steps", type=int, default=1000, help="Adam steps (batch 16)")
    ap.add_argument("--learned-eval", type=int, default=4, help="(sigma, alpha) draws at 1024x1024")
    ap.add_argument("--bilevel", action="store_true",
                    help="learn alpha by the bilevel problem on 8 pairs of 256x256 images")
    ap.add_argument("--sweep", action="store_true",
                    help="batched bilevel sweep only: 64 (sigma, alpha) solves on 8 uneven images")
    ap.add_argument("--matvec-case", action="store_true",
                    help="profiling case: one plan of --workload, then 2 matvecs per NFFT "
                         "arithmetic; no JSON")
    ap.add_argument("--net-case", action="store_true",
                    help="profiling case: 2 x (forward + loss/gradient) of the network on 16 "
                         "images of 256x256; no JSON")
    ap.add_argument("--net-engine", type=int, default=1,
                    help="--net-case convolution engine: 1 tcgen05, 0 mma.sync")
    ap.add_argument("--mis-case", action="store_true",
                    help="profiling case: window selection by mutual information, 2048x2048, "
                         "5x5 patches, 4 calls; no JSON")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def describe(wl):
    p = 2 * wl.radius + 1
    return ("%s: %dx%d image (N=%d), %dx%d %s patches -> L=%d windows of 3 dims, sigma=%g, "
            "alpha=%g, M=%d, n_os=%d, m=%d, tol=%g"
            % (wl.name, wl.n1, wl.n2, wl.N, p, p, wl.pad, wl.L, wl.sigma, wl.alpha, wl.M,
               wl.n_os, wl.m, wl.tol))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle baseline
def oracle_rows_baseline(wl, rows: int, seed: int = 99):
    """Direct O(N^2) oracle sums on a row sample; Gpts/s = rows * L / t.  The
    full-N direct matvec time is extrapolated from the sample (N / rows x t)."""
    from oracle import oracle as orc
    img = wl.image()
    coords = orc.image_coords(img, wl.radius, wl.windows, wl.pad)
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(wl.N)
    r = np.sort(rng.choice(wl.N, rows, replace=False))
    t0 = time.perf_counter()
    orc.gamma_full_rows(coords, wl.sigma, v, r)
    dt = time.perf_counter() - t0
    return {"value": rows * wl.L / dt / 1e9, "unit": "Gpts/s", "cores": orc.num_threads(),
            "kind": "oracle", "seconds": dt,
            "full_matvec_seconds_extrapolated": dt * wl.N / rows,
            "sample": "%d random rows of the direct FP64 sum Gamma_full v on %s (N=%d, L=%d); "
                      "full-N matvec time extrapolated (N / rows x sample time)"
                      % (rows, wl.name, wl.N, wl.L)}


def auto_rows(wl, target_s=12.0):
    from oracle import oracle as orc
    probe = oracle_rows_baseline(wl, 16)
    per_row = probe["seconds"] / 16
    return int(max(16, min(wl.N, target_s / max(per_row, 1e-9)))), orc.num_threads()


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    rows = args.cpu_rows or max(16, auto_rows(wl, target_s=8.0)[0] // max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_rows_baseline(wl, max(4, rows // 8))
    times = []
    for k in range(args.steps):
        b = oracle_rows_baseline(wl, rows, seed=100 + k)
        times.append(b["seconds"])
    total = sum(times)
    value = rows * wl.L * args.steps / total / 1e9
    cpu = {"value": value, "unit": "Gpts/s", "cores": b["cores"], "kind": "oracle",
           "sample": b["sample"] + "; per step"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gpts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(wl), "sample_rows": rows},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def combine_ranks(total_ms: float, pts: float, device, sum_work: bool = True) -> float:
    """Whole-job Gpts/s: the point-windows all ranks processed (summed over
    ranks for replicas; the one solve's for window sharding) divided by the
    slowest rank's timed region (max over ranks)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    p = torch.tensor([pts], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if sum_work:
            dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(p.item()) / (float(t.item()) * 1e-3) / 1e9


KERNEL_CLASSES = ["spread64", "spread32", "conv64", "conv32", "interp64", "interp32", "epilogue",
                  "krylov", "plan", "spread_df32", "interp_df32"]


def read_profile(lib):
    import ctypes as C
    prof = {}
    for c, nm in enumerate(KERNEL_CLASSES):
        cl, cm = C.c_int64(0), C.c_double(0)
        lib.nlh_profile_read(c, C.byref(cl), C.byref(cm))
        if cl.value:
            prof[nm] = {"launches": cl.value, "ms": cm.value}
    lib.nlh_profile_reset()
    return prof


def roofline(prof, wl, coords="stored"):
    """The dominant NFFT kernel class of the timed region against its
    rooflines.  Method work per point-window and direction: (2m)^3 stencil
    multiply-adds (2m window points per dim), 2 FLOP each, in the kernel's
    arithmetic (double-float and FP32 kernels run on the FP32 pipes; their
    peak is the FP32 one).  Algorithmic bytes per launch: half of the
    per-matvec N * 20 + N * L * 8 (image or coordinates, input, output,
    permutation)."""
    nfft = {k: v for k, v in prof.items() if k.startswith(("spread", "interp"))}
    if not nfft:
        return None
    dom = max(nfft, key=lambda k: nfft[k]["ms"])
    avg_s = nfft[dom]["ms"] / nfft[dom]["launches"] * 1e-3
    W2 = 2 * wl.m
    flops = 2.0 * float(wl.N * wl.L) * W2 ** 3
    ach = flops / avg_s / 1e12
    if dom.endswith("64"):
        peak, src = FP64_PEAK_TFLOPS, "GB300 nominal FP64 1.25 TFLOP/s"
    else:
        peak = FP32_PEAK_TFLOPS
        src = ("derived FP32: 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz" +
               ("; the kernel computes FP64-accurate double-float values on the FP32 pipes "
                "(~6 packed FP32 instructions per stencil update), counted here as 2 FLOP per "
                "update" if dom.endswith("df32") else ""))
    hbm_peak, hbm_src = measured_peaks()
    alg_bytes = 0.5 * (wl.N * 20.0 + wl.N * wl.L * 8.0)
    # what these kernels read with the plan's data: the permutation entry and
    # the stored cell offsets per point-window (12 B FP32, + 12 B low parts
    # for FP64 and double-float; the image per pixel instead when the
    # coordinates are recomputed from it), the input or output per pixel,
    # the grid
    parts = 2 if dom.endswith(("64", "df32")) else 1
    gbytes = 8 if dom.endswith(("64", "df32")) else 4
    per_pw = 4.0 + (0.0 if coords == "image" else 12.0 * parts)
    data_bytes = (wl.N * wl.L * per_pw + wl.N * 8.0 + (wl.N * 8.0 if coords == "image" else 0.0)
                  + wl.L * wl.n_os ** 3 * float(gbytes))
    traffic, tnote = None, None
    sha = kernel_sources_sha16()
    if NCU_TRAFFIC.get("sources_sha16") == sha and NCU_TRAFFIC.get("workload") == wl.name:
        traffic = NCU_TRAFFIC["bytes_per_launch"].get(coords, {}).get(dom)
        tnote = "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, same kernel sources"
    else:
        tnote = ("no ncu capture of the current kernel sources for this workload "
                 "(sources %s)" % sha)
    out = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
           "frac": ach / peak, "traffic": traffic, "traffic_note": tnote,
            "mean_launch_ms": avg_s * 1e3, "launches": nfft[dom]["launches"],
            "work": "2 x (2m)^3 FLOP per point-window, N L = %d point-windows per launch"
                    % (wl.N * wl.L),
            "peak_source": src,
            "hbm": {"algorithmic_bytes": alg_bytes, "achieved_gbs": alg_bytes / avg_s / 1e9,
                    "peak_gbs": hbm_peak, "frac": alg_bytes / avg_s / 1e9 / hbm_peak,
                    "kernel_data_bytes": data_bytes,
                    "kernel_data_gbs": data_bytes / avg_s / 1e9,
                    "peak_source": hbm_src}}
    if dom.endswith("df32"):
        # a double-float stencil update is 12 FP32 operations (exact product
        # with cross terms 4, TwoSum 6, low-word adds 2) for the method's 2
        # FLOP, so even a fully busy FP32 pipe reaches 2/12 of its peak in
        # method FLOP
        ceil = peak * 2.0 / DF32_OPS_PER_UPDATE
        out["arithmetic_ceiling"] = {"tflops": ceil, "frac": ach / ceil,
                                     "fp32_ops_per_update": DF32_OPS_PER_UPDATE}
    return out


def time_steps(step, args, dev, world, lib, stream, flush, steps, warmup, barrier):
    import torch
    infos = []
    for _ in range(warmup):
        infos.append(step())
    torch.cuda.synchronize()
    lib.nlh_profile_reset()
    launches0 = lib.nlh_kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    barrier()
    lib.nlh_profile_enable(1)
    step_infos = []
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        step_infos.append(step())
        ev[k][1].record(stream)
    lib.nlh_profile_enable(0)
    barrier()
    launches = lib.nlh_kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    return step_infos, step_ms, launches


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2407_06834_gb300 import nlh, shard

    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo",
                                init_method="env://")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    lib = nlh.load()
    wl = WORKLOADS[args.workload]
    img_np = wl.image()
    img = torch.as_tensor(img_np, device=dev)
    N, L = wl.N, wl.L
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    sharded = world > 1 and args.shard == "windows"
    wrange = shard.window_range(L, world, rank) if sharded else None

    def make_plan(image, sigma, precision=6, autotune=True):
        kw = {}
        if sharded:
            kw = {"window_range": wrange, "reduce": shard.allreduce_sum}
            autotune = False
        return nlh.Plan.from_image(image, wl.radius, wl.windows, sigma, pad=wl.pad, M=wl.M,
                                   n_os=wl.n_os, m=wl.m, precision=precision,
                                   autotune=autotune, coords_from_image=args.coords == "image",
                                   **kw)

    def step_on(image, u):
        P = make_plan(image, wl.sigma)
        b = image.reshape(-1) * wl.alpha
        res = P.solve(wl.alpha, b, tol=wl.tol, arith=nlh.SOLVE_MIXED, inner_tol=INNER_TOL, u=u)
        P.close()
        return res.info

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    u = torch.empty(N, dtype=torch.float64, device=dev)
    with ClockSampler(local_rank) as clk:
        step_infos, step_ms, launches = time_steps(lambda: step_on(img, u), args, dev, world,
                                                   lib, stream, flush, args.steps, args.warmup,
                                                   barrier)
    prof = read_profile(lib)
    total_ms = sum(step_ms)
    # degree matvecs of the plan (FP32 and double-float) + the solve's matvecs
    mv = [i["matvecs_fp64"] + i["matvecs_fp32"] + 2 for i in step_infos]
    pts = float(N * L * sum(mv))
    value = combine_ranks(total_ms, pts, dev, sum_work=not sharded)
    roof = roofline(prof, wl, args.coords) if not sharded else None

    # ---- end to end through the public API with host buffers
    img_h = torch.empty((wl.n1, wl.n2), dtype=torch.float64, pin_memory=True)
    img_h.copy_(torch.as_tensor(img_np))
    u_h = torch.empty(N, dtype=torch.float64, pin_memory=True)
    img_d = torch.empty_like(img)
    e2e_ms = []
    barrier()
    for k in range(max(3, args.steps // 2)):
        flush.zero_()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        img_d.copy_(img_h, non_blocking=True)
        info = step_on(img_d, u)
        u_h.copy_(u, non_blocking=True)
        b_.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b_))
        mv_e = info["matvecs_fp64"] + info["matvecs_fp32"] + 2
    e2e_val = N * L * mv_e / (statistics.mean(e2e_ms) * 1e-3) / 1e9

    # ---- seconds to 1e-6 per sigma of the workload (plan prebuilt)
    solve_s = {}
    for sg in (wl.sigmas or [wl.sigma]):
        P = make_plan(img, sg)
        bvec = img.reshape(-1) * wl.alpha
        row = {}
        for nm, ar, it in (("mixed", nlh.SOLVE_MIXED, INNER_TOL),
                           ("mixed_inner_1e-3", nlh.SOLVE_MIXED, 1e-3),
                           ("df32", nlh.SOLVE_DF32, INNER_TOL)):
            P.solve(wl.alpha, bvec, tol=wl.tol, arith=ar, inner_tol=it)
            r = P.solve(wl.alpha, bvec, tol=wl.tol, arith=ar, inner_tol=it)
            row[nm] = {"seconds": r.info["seconds"], "iters": r.info["iters"],
                       "outer": r.info["outer"], "rel_res_fp64": r.info["rel_res_true"]}
        P.close()
        solve_s["sigma=%g" % sg] = row
    # plan creation alone
    t0 = time.perf_counter()
    for _ in range(2):
        Q = make_plan(img, wl.sigma)
        Q.close()
    torch.cuda.synchronize()
    solve_s["plan_seconds"] = (time.perf_counter() - t0) / 2
    # kernel-only matvec throughput
    P = make_plan(img, wl.sigma)
    x = torch.randn(N, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    mv_gpts = {}
    for nm, prec in (("df32", nlh.NLH_DF32), ("fp32", nlh.NLH_FP32)):
        for _ in range(3):
            P.matvec(x, op=2, precision=prec, alpha=wl.alpha, out=y)
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(5):
            P.matvec(x, op=2, precision=prec, alpha=wl.alpha, out=y)
        b_.record(stream)
        torch.cuda.synchronize()
        mv_gpts[nm] = {"gpts": N * L / (a.elapsed_time(b_) / 5 * 1e-3) / 1e9,
                       "ms": a.elapsed_time(b_) / 5}
    pinfo = P.info()
    P.close()

    side = {}
    if not args.no_side and world == 1:
        side["img512"] = small_line(args, dev, lib, flush)
        side["sweep"] = sweep_leg(args)
        if not args.no_learned:
            side["learned"] = learned_leg(args, dev)
        side["mis_windows"] = mis_leg(dev)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rows = args.cpu_rows or auto_rows(wl)[0]
        cpu = oracle_rows_baseline(wl, rows)
        cpu.pop("seconds", None)
    line = {
        "metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": "f32 + df32 (FP32 NFFT inner solves; double-float NFFT for degrees and refinement residuals; FP64 Krylov vectors and dots)",
        "data": "synthetic (seeded piecewise-constant image + N(0,0.1^2) noise)",
        "config": {"workload": describe(wl),
                   "l2": "flushed between steps (256 MB write); the plan's data (~1 GB) exceeds L2",
                   "parallelism": ("windows %s per rank, one NCCL all-reduce per matvec" % (wrange,)
                                   if sharded else ("replicas" if world > 1 else "single GPU")),
                   "torus_fill": pinfo["torus_fill"], "work_items": pinfo["n_items"],
                   "plan_device_bytes": pinfo["device_bytes"],
                   "tiling": {"max_items_pts": pinfo["max_items_pts"],
                              "unit_points": pinfo["unit_points"], "units": pinfo["n_units"],
                              "team_fp64_fp32_df32": pinfo["team"]},
                   "coordinates": ("recomputed from the image" if args.coords == "image"
                                   else "stored cell offsets per point-window")},
        "solve_seconds": solve_s,
        "matvec_kernel_only": mv_gpts,
        "iters_per_step": statistics.mean(i["iters"] for i in step_infos),
        "matvecs_per_step": statistics.mean(mv),
        "e2e": {"value": e2e_val, "unit": "Gpts/s", "h2d_bytes_per_step": N * 8,
                "d2h_bytes_per_step": N * 8},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "roofline": roof,
        "kernel_ms": prof,
        "cpu_baseline": cpu,
    }
    line.update(side)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def small_line(args, dev, lib, flush):
    """The same step on the 512 x 512 workload (3x3 patches, L = 3, M = 32,
    n_os = 64, m = 4): Gpts/s over the step, the roofline of its dominant
    NFFT kernel, and FP64 / double-float / mixed solves to 1e-6."""
    import torch

    from paper_2407_06834_gb300 import nlh
    wl = WORKLOADS["img512"]
    img = torch.as_tensor(wl.image(), device=dev)
    stream = torch.cuda.current_stream()
    u = torch.empty(wl.N, dtype=torch.float64, device=dev)

    def step():
        P = nlh.Plan.from_image(img, wl.radius, wl.windows, wl.sigma, pad=wl.pad, M=wl.M,
                                n_os=wl.n_os, m=wl.m, precision=6, autotune=True)
        r = P.solve(wl.alpha, img.reshape(-1) * wl.alpha, tol=wl.tol, arith=nlh.SOLVE_MIXED,
                    inner_tol=INNER_TOL, u=u)
        P.close()
        return r.info

    infos, ms, launches = time_steps(step, args, dev, 1, lib, stream, flush, 10, 3,
                                     torch.cuda.synchronize)
    prof = read_profile(lib)
    mv = [i["matvecs_fp64"] + i["matvecs_fp32"] + 2 for i in infos]
    out = {"workload": describe(wl), "value": wl.N * wl.L * sum(mv) / (sum(ms) * 1e-3) / 1e9,
           "unit": "Gpts/s", "ms_per_step": sum(ms) / len(ms), "gpu_launches": int(launches),
           "roofline": roofline(prof, wl), "kernel_ms": prof}
    P = nlh.Plan.from_image(img, wl.radius, wl.windows, wl.sigma, pad=wl.pad, M=wl.M,
                            n_os=wl.n_os, m=wl.m, precision=7)
    b = img.reshape(-1) * wl.alpha
    sv = {}
    for nm, ar, it in (("fp64", nlh.SOLVE_FP64, INNER_TOL), ("df32", nlh.SOLVE_DF32, INNER_TOL),
                       ("mixed", nlh.SOLVE_MIXED, INNER_TOL),
                       ("mixed_inner_1e-3", nlh.SOLVE_MIXED, 1e-3)):
        P.solve(wl.alpha, b, tol=wl.tol, arith=ar, inner_tol=it)
        r = P.solve(wl.alpha, b, tol=wl.tol, arith=ar, inner_tol=it)
        sv[nm] = {"seconds": r.info["seconds"], "iters": r.info["iters"],
                  "outer": r.info["outer"], "rel_res_fp64": r.info["rel_res_true"]}
    P.close()
    out["solve_seconds"] = sv
    return out


def net_flops_per_image(net, H, W):
    """Tensor-core FLOPs of one forward pass (3x3 layers; the head is not a GEMM)."""
    fl = 0.0
    names = []
    L = net.levels
    for l in range(L):
        names += [l, l]
    for l in range(L - 2, -1, -1):
        names += [l, l]
    for (cin, cout, k), lv in zip(net.layers[:-1], names):
        cinp = (cin + 31) // 32 * 32
        fl += 2.0 * 9 * cinp * cout * (H >> lv) * (W >> lv)
    return fl


def learned_leg(args, dev):
    """Train the network on method-generated 256x256 triples with the
    library's kernels, then time plain vs learned mixed solves to 1e-6 on
    1024x1024 images (the learned time includes the network's forward)."""
    import torch

    from paper_2407_06834_gb300 import learned, nlh
    from paper_2407_06834_gb300.inputs import learned_draws, synthetic_image
    out = {}
    net = learned.new_net(seed=0)
    data = learned.make_triples(args.learned_triples, 256, 256, seed=0, per_image=4, net=net,
                                workers=min(16, os.cpu_count() or 1))
    out["triples"] = {"count": data.count, "size": "256x256", "seconds": data.seconds,
                      "worst_rel_res_fp64": data.worst_rel_res,
                      "plain_iters_mean": float(data.iters.mean())}
    batch = 16
    epochs = args.learned_steps * batch / data.count
    log = learned.train(net, data, epochs=epochs, batch=batch, lr=1e-3, beta=0.25,
                        beta_from=0.5, log_every=100)
    fl = 3.0 * net_flops_per_image(net, 256, 256) * batch * log.steps
    out["training"] = {"steps": log.steps, "batch": batch, "seconds": log.seconds,
                       "snapshot_refresh_seconds": log.refresh_seconds,
                       "tensor_tflops": fl / log.seconds / 1e12,
                       "loss_first": log.losses[0][2], "loss_last": log.losses[-1][2]}
    rows = []
    for k, (_, sg, al) in enumerate(learned_draws(args.learned_eval, 99)):
        img = torch.as_tensor(synthetic_image(1024, 1024, 5000 + k)[1], device=dev)
        # precision 7: the FP64 path too, for the plain FP64 solve
        P = learned._plan(img, sg, precision=7)
        b = img.reshape(-1) * al
        for _ in range(2):
            pl = P.solve(al, b, tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=1e-3)
            p64 = P.solve(al, b, tol=1e-6, arith=nlh.SOLVE_FP64)
            t0 = time.perf_counter()
            lr_, t_net = learned.learned_solve(net, P, img, sg, al)
            t_l = time.perf_counter() - t0
        rows.append({"sigma": sg, "alpha": al, "plain_iters": pl.info["iters"],
                     "plain_seconds": pl.info["seconds"],
                     "plain_fp64_iters": p64.info["iters"],
                     "plain_fp64_seconds": p64.info["seconds"],
                     "plain_fp64_rel_res": p64.info["rel_res_true"],
                     "learned_iters": lr_.info["iters"],
                     "learned_seconds": t_l, "net_forward_seconds": t_net,
                     "x0_rejected": lr_.info["x0_rejected"],
                     "used_fallback": lr_.info["used_fallback"],
                     "learned_rel_res_fp64": lr_.info["rel_res_true"]})
        P.close()
    out["eval_1024"] = rows
    out["time_ratio_learned_over_plain"] = (sum(r["learned_seconds"] for r in rows)
                                            / sum(r["plain_seconds"] for r in rows))
    # the stated target: the learned + mixed form against the plain FP64 solve
    out["time_ratio_learned_over_plain_fp64"] = (sum(r["learned_seconds"] for r in rows)
                                                 / sum(r["plain_fp64_seconds"] for r in rows))
    out["net_forward_tflops_1024"] = (net_flops_per_image(net, 1024, 1024)
                                      / statistics.mean(r["net_forward_seconds"] for r in rows)
                                      / 1e12)
    net.close()
    return out


def mis_leg(dev):
    """Window selection by mutual information (Sec. 5), a setup step once
    per image: device time of nlh_mis_windows (64 bins, reflect padding) at
    512^2 with 3x3 patches and 2048^2 with 5x5 patches, the oracle timed on
    the 512^2 case on the host, and whether the windows agree there."""
    import torch

    from oracle import mis as omis
    from paper_2407_06834_gb300 import nlh
    from paper_2407_06834_gb300.inputs import synthetic_image
    out = {}
    for n, rho in ((512, 1), (2048, 2)):
        img_h = synthetic_image(n, n, 0)[1]
        img = torch.as_tensor(img_h, device=dev)
        for _ in range(3):
            nlh.mis_windows(img, rho, "reflect", 64)
        stream = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(20):
            _, w, _ = nlh.mis_windows(img, rho, "reflect", 64)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 20
        D = (2 * rho + 1) ** 2
        row = {"ms": ms, "gfeatures_per_s": n * n * D / ms / 1e6, "windows": w.tolist()}
        if n == 512:
            t0 = time.perf_counter()
            _, w_ref = omis.mis_windows(img_h, rho, "reflect", 64)
            row["oracle_seconds"] = time.perf_counter() - t0
            row["oracle_kind"] = "oracle/mis.py: numpy, one thread (patch extraction OpenMP)"
            row["windows_match_oracle"] = bool((w == w_ref).all())
        out["%dx%d_%dx%d" % (n, n, 2 * rho + 1, 2 * rho + 1)] = row
    return out


def matvec_case(args):
    """Small profiling case: one plan of --workload with the FP32 and
    double-float arithmetics in the default tiling and launch shapes, then
    2 matvecs per arithmetic."""
    import torch

    from paper_2407_06834_gb300 import nlh
    wl = WORKLOADS[args.workload]
    img = torch.as_tensor(wl.image(), device="cuda")
    P = nlh.Plan.from_image(img, wl.radius, wl.windows, wl.sigma, pad=wl.pad, M=wl.M,
                            n_os=wl.n_os, m=wl.m, precision=6,
                            coords_from_image=args.coords == "image")
    x = torch.randn(wl.N, dtype=torch.float64, device="cuda")
    for prec in (nlh.NLH_FP32, nlh.NLH_DF32):
        for _ in range(2):
            P.matvec(x, op=2, precision=prec, alpha=wl.alpha)
    torch.cuda.synchronize()
    P.close()


def net_case(args):
    """Small profiling case of the learned leg's network: 2 x (forward +
    loss and gradient) on 16 synthetic 256x256 images."""
    import torch

    from paper_2407_06834_gb300 import learned
    from paper_2407_06834_gb300.inputs import synthetic_image
    net = learned.new_net(seed=0)
    net.engine = args.net_engine
    B = 16
    f = torch.as_tensor(np.stack([synthetic_image(256, 256, i)[1] for i in range(B)]),
                        device="cuda")
    sig, alp = [0.2] * B, [0.5] * B
    ustar, deg = f.clone(), torch.full_like(f, 2.0)
    for _ in range(2):
        net.forward(f, sig, alp)
        net.loss_grad(f, sig, alp, ustar, deg=deg, want_loss=False)
    net.check()
    net.close()


def mis_case(args):
    """Small profiling case: 4 calls of nlh_mis_windows on a 2048x2048 image
    with 5x5 reflect-padded patches and 64 bins."""
    import torch

    from paper_2407_06834_gb300 import nlh
    from paper_2407_06834_gb300.inputs import synthetic_image
    img = torch.as_tensor(synthetic_image(2048, 2048, 0)[1], device="cuda")
    for _ in range(4):
        nlh.mis_windows(img, 2, "reflect", 64)
    torch.cuda.synchronize()


def sweep_leg(args):
    """64 solves over a log grid of sigma in [0.05, 1] x alpha in [0.01, 10] on 8
    synthetic images of uneven sizes (pair (i, j) -> image (i + j) mod 8), each
    with its own plan (NFFT parameters chosen for a 1e-7 per-dim error).
    Times one batched call against a loop of single solves."""
    import torch

    from paper_2407_06834_gb300 import nlh
    from paper_2407_06834_gb300.inputs import SWEEP_SIZES, raster_windows, sweep_pairs, synthetic_image
    dev = torch.device("cuda", 0)
    imgs = [torch.as_tensor(synthetic_image(n, n, 1 + k)[1], device=dev)
            for k, n in enumerate(SWEEP_SIZES)]
    pairs = sweep_pairs()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # autotuned tiling and launch shapes (cached per problem class; the first
    # plan of a class pays the tuning inside plans_seconds)
    plans = [nlh.Plan.from_image(imgs[i], 1, raster_windows(1), s, precision=6, nfft_eps=1e-7,
                                 m=0, autotune=True) for i, s, a in pairs]
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    bs = [imgs[i].reshape(-1) * a for i, s, a in pairs]
    alphas = [a for i, s, a in pairs]
    us = [torch.empty_like(b) for b in bs]
    # warm up: graphs instantiated once per plan
    nlh.solve_batched(plans, alphas, bs, us, tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=INNER_TOL)
    for P, a, b, u in zip(plans, alphas, bs, us):
        P.solve(a, b, tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=INNER_TOL, u=u)
    torch.cuda.synchronize()
    reps = max(1, args.steps // 5)
    t0 = time.perf_counter()
    for _ in range(reps):
        for P, a, b, u in zip(plans, alphas, bs, us):
            P.solve(a, b, tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=INNER_TOL, u=u)
    torch.cuda.synchronize()
    t_loop = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        _, infos = nlh.solve_batched(plans, alphas, bs, us, tol=1e-6, arith=nlh.SOLVE_MIXED,
                                     inner_tol=INNER_TOL)
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) / reps
    worst = max(i["rel_res_true"] for i in infos)
    px = sum(P.N for P in plans)
    out = {
        "metric": "batched bilevel sweep, solves/s (64 mixed-precision solves to 1e-6)",
        "value": len(plans) / t_batch, "unit": "solves/s", "higher_is_better": True,
        "loop_of_single_solves": len(plans) / t_loop, "speedup_vs_loop": t_loop / t_batch,
        "plans_seconds": t_plan, "batch_seconds": t_batch, "loop_seconds": t_loop,
        "worst_rel_res_fp64": worst, "pixels_per_sweep": px,
        "iters": [i["iters"] for i in infos], "outer": [i["outer"] for i in infos],
        "nfft": [{"M": P.info()["M"], "n_os": P.info()["n_os"], "m": P.info()["m"],
                  "fill": P.info()["torus_fill"]} for P in plans[:8]],
        "config": {"workload": "8 images %s, 64 (sigma, alpha) pairs" % SWEEP_SIZES,
                   "reps": reps}}
    for P in plans:
        P.close()
    return out


def run_sweep(args):
    print(json.dumps(sweep_leg(args)), flush=True)


def run_bilevel(args):
    """Sec. 5.5's learning experiment on synthetic pairs: alpha by Brent's
    method on j(alpha) = mean ||u_c - u(alpha)||^2 over 8 pairs of 256x256
    images (sigma = 0.2, Lambda = [1e-2, 1e6]); each evaluation is one
    batched call of 8 mixed-precision lower-level solves to 1e-8."""
    import torch

    from paper_2407_06834_gb300 import bilevel
    from paper_2407_06834_gb300.inputs import synthetic_image
    pairs = [synthetic_image(256, 256, s) for s in range(1, 9)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = bilevel.Bilevel(pairs, 0.2, tol=1e-8)
    torch.cuda.synchronize()
    t_plans = time.perf_counter() - t0
    res = B.learn(bounds=(1e-2, 1e6), xatol=1e-3)
    j0 = float(np.mean([np.sum((c - n) ** 2) for c, n in pairs]))
    _, g = B.objective_and_gradient(res.alpha)
    joint = B.learn_alpha_theta(res.alpha, 0.2, bounds_alpha=(1e-2, 1e6),
                                bounds_sigma=(0.1, 0.4))
    joint.pop("history")
    B.close()
    print(json.dumps({
        "metric": "bilevel learning of alpha: seconds (8 pairs of 256x256, Brent, mixed solves)",
        "value": res.seconds, "unit": "s", "higher_is_better": False,
        "alpha": res.alpha, "j": res.j, "j_noisy": j0, "evaluations": res.evaluations,
        "lower_level_solves": res.solves, "cg_iters_per_solve": res.cg_iters_mean,
        "gradient_at_alpha": g, "plans_seconds": t_plans,
        "joint_alpha_theta": joint,
        "history": res.history,
        "config": {"workload": "8 synthetic pairs (seeds 1-8) 256x256, 3x3 reflect patches, "
                               "L=3, sigma=0.2, Lambda=[1e-2, 1e6], tol 1e-8"}}), flush=True)


def main():
    args = parse()
    if args.bilevel:
        run_bilevel(args)
    elif args.sweep:
        run_sweep(args)
    elif args.matvec_case:
        matvec_case(args)
    elif args.net_case:
        net_case(args)
    elif args.mis_case:
        mis_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
