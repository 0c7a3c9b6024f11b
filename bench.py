#!/usr/bin/env python3
"""Benchmark of the NFFT nonlocal-denoising hot path (one JSON line).

A step is one pass of the whole path over one synthetic image: patch
features, the plan (torus map, sort by cell, weights, tables, degrees), and
a deflated Jacobi-PCG solve of (alpha I + L) u = alpha f to relative
residual 1e-6 in the mixed form (FP32-NFFT inner solves, FP64 refinement
residuals).  The metric is NFFT matvec throughput in Gpts/s: point-windows
(N * L per matvec) pushed through the NFFT per second, over the whole step;
the seconds-to-solve of the FP64 and mixed forms are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per rank, launched by torchrun): the
path has no exchange step, so there is no data collective; the ranks only
meet at the timing barriers and the max-over-ranks of the step time.
--impl reference times the CPU FP64 oracle (direct O(N^2) sums) on the host
cores on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
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
# Non-tensor ALU peaks derived from unit counts and the 2070 MHz max clock:
# FP32: 152 SMs x 128 FMA lanes x 2 flop; FP64: GB300 nominal 1.25 TFLOP/s.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = 1.25
# FP32 FLOPs of one double-float stencil multiply-add: TwoProduct by FMA with
# the two cross terms (1 mul + 3 FMA = 7 FLOP) and TwoSum into the high word
# with the low word accumulated (8 add/sub) -- 12 instructions, 15 FLOP.
DF32_FLOP_PER_UPDATE = 15
# DRAM bytes (read + write) per launch from the ncu capture summarised in
# profiles/k_nfft_fp32_df32_img512.md (512 x 512 workload); None elsewhere.
NCU_TRAFFIC_IMG512 = {"spread32": 80.39e6, "interp32": 81.26e6,
                      "spread_df32": 160.22e6, "interp_df32": 159.31e6}


def measured_hbm_gbs():
    """The measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the
    profiling fallback of 6.8 TB/s."""
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="img512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=0, help="oracle row sample (0 = auto)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-form leg")
    ap.add_argument("--learned-triples", type=int, default=512,
                    help="training triples at 256x256 for the learned leg")
    ap.add_argument("--learned-steps", type=int, default=1000, help="Adam steps (batch 16)")
    ap.add_argument("--learned-eval", type=int, default=4, help="(sigma, alpha) draws at 1024x1024")
    ap.add_argument("--bilevel", action="store_true",
                    help="learn alpha by the bilevel problem on 8 pairs of 256x256 images")
    ap.add_argument("--sweep", action="store_true",
                    help="batched bilevel sweep: 64 (sigma, alpha) solves on 8 uneven images")
    ap.add_argument("--matvec-case", action="store_true",
                    help="profiling case: one plan, then 2 matvecs per NFFT precision; no JSON")
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
    """Direct O(N^2) oracle sums on a row sample; Gpts/s = rows * L / t."""
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
            "sample": "%d random rows of the direct FP64 sum Gamma_full v on %s (N=%d, L=%d)"
                      % (rows, wl.name, wl.N, wl.L)}


def auto_rows(wl, target_s=12.0):
    from oracle import oracle as orc
    probe = oracle_rows_baseline(wl, 64)
    per_row = probe["seconds"] / 64
    return int(max(64, min(wl.N, target_s / max(per_row, 1e-9)))), orc.num_threads()


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    rows = args.cpu_rows or max(64, auto_rows(wl, target_s=8.0)[0] // max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_rows_baseline(wl, max(16, rows // 8))
    times, vals = [], []
    for k in range(args.steps):
        b = oracle_rows_baseline(wl, rows, seed=100 + k)
        times.append(b["seconds"])
        vals.append(b["value"])
    total = sum(times)
    value = rows * wl.L * args.steps / total / 1e9
    cpu = {"value": value, "unit": "Gpts/s", "cores": b["cores"], "kind": "oracle",
           "sample": b["sample"] + " per step"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gpts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%s: %dx%d synthetic image, 3x3 reflect patches, L=%d, "
                                   "sigma=%g" % (wl.name, wl.n1, wl.n2, wl.L, wl.sigma),
                       "sample_rows": rows},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def combine_ranks(total_ms: float, pts: float, device) -> float:
    """Replicas: whole-job Gpts/s = the point-windows all ranks processed
    divided by the slowest rank's timed region (max over ranks)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    p = torch.tensor([pts], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(p.item()) / (float(t.item()) * 1e-3) / 1e9


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2407_06834_gb300 import nlh

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

    def step(image, u):
        P = nlh.Plan.from_image(image, wl.radius, wl.windows, wl.sigma, pad=wl.pad, M=wl.M,
                                n_os=wl.n_os, m=wl.m, precision=6, autotune=True)
        b = image.reshape(-1) * wl.alpha
        res = P.solve(wl.alpha, b, tol=wl.tol, arith=nlh.SOLVE_MIXED, inner_tol=1e-3, u=u)
        P.close()
        return res

    u = torch.empty(N, dtype=torch.float64, device=dev)
    infos = []
    for _ in range(args.warmup):
        infos.append(step(img, u).info)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region (device-resident inputs)
    lib.nlh_profile_reset()
    launches0 = lib.nlh_kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        barrier()
        lib.nlh_profile_enable(1)
        step_infos = []
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step_infos.append(step(img, u).info)
            ev[k][1].record(stream)
        lib.nlh_profile_enable(0)
        barrier()
    launches = lib.nlh_kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    # 2 degree matvecs per plan (double-float and FP32) + the solve's matvecs
    mv = [i["matvecs_fp64"] + i["matvecs_fp32"] + 2 for i in step_infos]
    pts = float(N * L * sum(mv))
    value = combine_ranks(total_ms, pts, dev)

    # per-kernel-class device time inside the timed region
    prof = {}
    names = ["spread64", "spread32", "conv64", "conv32", "interp64", "interp32", "epilogue",
             "krylov", "plan", "spread_df32", "interp_df32"]
    import ctypes as C
    for c, nm in enumerate(names):
        cl, cm = C.c_int64(0), C.c_double(0)
        lib.nlh_profile_read(c, C.byref(cl), C.byref(cm))
        if cl.value:
            prof[nm] = {"launches": cl.value, "ms": cm.value}
    lib.nlh_profile_reset()
    dom = max(prof, key=lambda k: prof[k]["ms"]) if prof else None
    W2 = 2 * wl.m
    updates = float(N * L * W2 ** 3)          # (2m)^3 stencil updates per point-window
    roof = None
    if dom and dom.startswith(("spread", "interp")):
        avg_s = prof[dom]["ms"] / prof[dom]["launches"] * 1e-3
        traffic = NCU_TRAFFIC_IMG512.get(dom) if wl.name == "img512" else None
        if dom.endswith("df32"):
            ach = DF32_FLOP_PER_UPDATE * updates / avg_s / 1e12
            peak = FP32_PEAK_TFLOPS
            src = ("derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz; achieved = 15 FP32 FLOP "
                   "per double-float stencil update (TwoProduct + TwoSum) x (2m)^3 N L / launch "
                   "time; FP64-accurate rate %.2f TFLOP/s vs FP64 nominal 1.25"
                   % (2.0 * updates / avg_s / 1e12))
        elif dom.endswith("64"):
            ach, peak = 2.0 * updates / avg_s / 1e12, FP64_PEAK_TFLOPS
            src = "GB300 nominal FP64 1.25 TFLOP/s"
        else:
            ach, peak = 2.0 * updates / avg_s / 1e12, FP32_PEAK_TFLOPS
            src = "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"
        # the same launch against the HBM roofline: algorithmic bytes per
        # point-window = one weight record + one permutation entry + one FP64
        # value (interpolation output / spreading input of the FP64-side
        # vectors); 108 B FP32, 204 B double-float at m = 4, as ncu measures
        rec_bytes = 3 * W2 * (8 if dom.endswith(("64", "df32")) else 4)
        alg_bytes = float(N * L) * (((rec_bytes + 15) // 16) * 16 + 4 + 8)
        hbm_peak = measured_hbm_gbs()
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic,
                "traffic_note": "ncu DRAM read+write bytes per launch, 512x512 capture"
                if traffic else None,
                "mean_launch_ms": avg_s * 1e3, "peak_source": src,
                "hbm": {"algorithmic_bytes": alg_bytes, "achieved_gbs": alg_bytes / avg_s / 1e9,
                        "peak_gbs": hbm_peak,
                        "frac": (alg_bytes / avg_s / 1e9 / hbm_peak) if hbm_peak else None,
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}}
    elif dom:
        roof = {"bound": "hbm", "kernel": dom, "achieved": None, "peak": None, "unit": "GB/s",
                "frac": None, "traffic": None}

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
        info = step(img_d, u).info
        u_h.copy_(u, non_blocking=True)
        b_.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b_))
        mv_e = info["matvecs_fp64"] + info["matvecs_fp32"] + 2
    e2e_val = N * L * mv_e / (statistics.mean(e2e_ms) * 1e-3) / 1e9

    # ---- seconds to 1e-6, FP64 form vs mixed form (plan prebuilt)
    P = nlh.Plan.from_image(img, wl.radius, wl.windows, wl.sigma, pad=wl.pad, M=wl.M,
                            n_os=wl.n_os, m=wl.m, precision=7)
    bvec = img.reshape(-1) * wl.alpha
    solve_s = {}
    t0 = time.perf_counter()
    for _ in range(3):
        Q = nlh.Plan.from_image(img, wl.radius, wl.windows, wl.sigma, pad=wl.pad, M=wl.M,
                                n_os=wl.n_os, m=wl.m, precision=6)
        Q.close()
    torch.cuda.synchronize()
    solve_s["plan_seconds"] = (time.perf_counter() - t0) / 3
    for nm, ar, pc in (("fp64", nlh.SOLVE_FP64, 0), ("df32", nlh.SOLVE_DF32, 0),
                       ("mixed", nlh.SOLVE_MIXED, 0), ("mixed_pb", nlh.SOLVE_MIXED, 1)):
        P.solve(wl.alpha, bvec, tol=wl.tol, arith=ar, inner_tol=1e-3, precond=pc)
        r = P.solve(wl.alpha, bvec, tol=wl.tol, arith=ar, inner_tol=1e-3, precond=pc)
        solve_s[nm] = {"seconds": r.info["seconds"], "iters": r.info["iters"],
                       "rel_res_fp64": r.info["rel_res_true"]}
    # kernel-only matvec throughput
    x = torch.randn(N, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    mv_gpts = {}
    for nm, prec in (("fp64", nlh.NLH_FP64), ("df32", nlh.NLH_DF32), ("fp32", nlh.NLH_FP32)):
        for _ in range(3):
            P.matvec(x, op=2, precision=prec, alpha=wl.alpha, out=y)
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(10):
            P.matvec(x, op=2, precision=prec, alpha=wl.alpha, out=y)
        b_.record(stream)
        torch.cuda.synchronize()
        mv_gpts[nm] = N * L / (a.elapsed_time(b_) / 10 * 1e-3) / 1e9
    pinfo = P.info()
    P.close()
    learned_out = None if args.no_learned or world > 1 else learned_leg(args, dev)
    mis_out = None if world > 1 or rank != 0 else mis_leg(dev)

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
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 + df32 (FP32 NFFT inner solves; double-float NFFT for degrees and refinement residuals; FP64 Krylov vectors and dots)",
        "data": "synthetic (seeded piecewise-constant image + N(0,0.1^2) noise)",
        "config": {"workload": "%s: %dx%d image (N=%d), %dx%d %s patches -> L=%d windows "
                               "of 3 dims, sigma=%g, alpha=%g, M=%d, n_os=%d, m=%d, "
                               "tol=%g" % (wl.name, wl.n1, wl.n2, N, 2 * wl.radius + 1,
                                            2 * wl.radius + 1, wl.pad, L, wl.sigma, wl.alpha,
                                            wl.M, wl.n_os, wl.m, wl.tol),
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "torus_fill": pinfo["torus_fill"], "work_items": pinfo["n_items"]},
        "solve_seconds": solve_s,
        "matvec_gpts_kernel_only": mv_gpts,
        "iters_per_step": statistics.mean(i["iters"] for i in step_infos),
        "matvecs_per_step": statistics.mean(mv),
        "e2e": {"value": e2e_val, "unit": "Gpts/s", "h2d_bytes_per_step": N * 8,
                "d2h_bytes_per_step": N * 8},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "roofline": roof,
        "kernel_ms": prof,
        "learned": learned_out,
        "mis_windows": mis_out,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


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
    """Small profiling case: one 512x512 plan with all three arithmetics and
    the autotuned launch shapes of the bench step (FP32: default; double-
    float: 2 warps x 4 teams), then 2 matvecs per arithmetic."""
    import torch

    from paper_2407_06834_gb300 import nlh
    wl = WORKLOADS[args.workload]
    img = torch.as_tensor(wl.image(), device="cuda")
    P = nlh.Plan.from_image(img, wl.radius, wl.windows, wl.sigma, pad=wl.pad, M=wl.M,
                            n_os=wl.n_os, m=wl.m, precision=7, max_items_pts=128,
                            unit_points=512, team=(0, 0, 2))
    x = torch.randn(wl.N, dtype=torch.float64, device="cuda")
    for prec in (nlh.NLH_FP64, nlh.NLH_FP32, nlh.NLH_DF32):
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


def run_sweep(args):
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
    nlh.solve_batched(plans, alphas, bs, us, tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=1e-3)
    for P, a, b, u in zip(plans, alphas, bs, us):
        P.solve(a, b, tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=1e-3, u=u)
    torch.cuda.synchronize()
    reps = max(1, args.steps // 5)
    t0 = time.perf_counter()
    for _ in range(reps):
        for P, a, b, u in zip(plans, alphas, bs, us):
            P.solve(a, b, tol=1e-6, arith=nlh.SOLVE_MIXED, inner_tol=1e-3, u=u)
    torch.cuda.synchronize()
    t_loop = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        _, infos = nlh.solve_batched(plans, alphas, bs, us, tol=1e-6, arith=nlh.SOLVE_MIXED,
                                     inner_tol=1e-3)
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) / reps
    worst = max(i["rel_res_true"] for i in infos)
    px = sum(P.N for P in plans)
    print(json.dumps({
        "metric": "batched bilevel sweep, solves/s (64 mixed-precision solves to 1e-6)",
        "value": len(plans) / t_batch, "unit": "solves/s", "higher_is_better": True,
        "loop_of_single_solves": len(plans) / t_loop, "speedup_vs_loop": t_loop / t_batch,
        "plans_seconds": t_plan, "batch_seconds": t_batch, "loop_seconds": t_loop,
        "worst_rel_res_fp64": worst, "pixels_per_sweep": px,
        "iters": [i["iters"] for i in infos], "outer": [i["outer"] for i in infos],
        "nfft": [{"M": P.info()["M"], "n_os": P.info()["n_os"], "m": P.info()["m"],
                  "fill": P.info()["torus_fill"]} for P in plans[:8]],
        "config": {"workload": "8 images %s, 64 (sigma, alpha) pairs" % SWEEP_SIZES,
                   "reps": reps}}), flush=True)


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
