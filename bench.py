#!/usr/bin/env python
"""Throughput benchmark of the accelerated FBP (IIR ramp filter + fast Hough transform
back projection) on GB300.

One step = the whole method (recursive filtering, resampling fused with the first Hough
pass, second Hough pass fused with the quarter sum) over a stack of 64 slices of N = 2048
(K = 3072 angles, M = 2897 bins) per GPU, synthetic noisy ten-ellipse phantoms, with the
sinograms already resident in HBM.  The stack (2.28 GB of sinograms) is larger than L2, so
no flush is needed between steps.

Printed (rank 0, one JSON line): slices/s of the whole job, the event-timed roofline of
the dominant kernel, the end-to-end number through the host-memory entry point, the
direct GPU FBP comparator, the RMSE against the float64 direct reconstruction at sampled
pixels, the SM clocks seen during the timed region and the CPU oracle baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 run it under torch.distributed.run: every rank reconstructs its own stack
(independent slices, no collective on the data path), timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "slices/s at N=2048 (IIR+FHT vs direct GPU FBP), %HBM roofline, RMSE vs FP64"
UNIT = "slices/s"
BASE_SEED = 2021
I0 = 1e5


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--N", type=int, default=2048)
    ap.add_argument("--slices", type=int, default=64, help="slices per GPU per step")
    ap.add_argument("--order", type=int, default=3, help="recursive filter order Q = Mb")
    ap.add_argument("--direct-slices", type=int, default=2)
    ap.add_argument("--chunk", type=int, default=0, help="slices per launch (0 = library default)")
    ap.add_argument("--sample-pixels", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=("stack", "ragged", "adjoint", "corrector", "sirt"),
                    default="stack",
                    help="stack: the N = 2048 64-slice stack (default); ragged: a volume of "
                         "--ragged-slices slices with N drawn uniformly from 256..2048; "
                         "adjoint: forward and adjoint (gradient) passes on a batch of 32 "
                         "slices of N = 512; corrector: the learned CNN corrector, trained on "
                         "N = 512 pairs, inference on 16 slices of N = 2048; sirt: "
                         "algebraic reconstruction on the fast Hough operators, 16 slices of "
                         "N = 512, 10 iterations per step")
    ap.add_argument("--ragged-slices", type=int, default=512)
    ap.add_argument("--train-pairs", type=int, default=20000,
                    help="corrector: N = 512 (fast, direct) training pairs")
    ap.add_argument("--train-steps", type=int, default=1250,
                    help="corrector: Adam steps of batch 16 (1250 = one pass over 20000 pairs)")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- topology
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard(rank: int, slices_per_rank: int):
    """Global slice indices and phantom seeds of this rank's stack (weak scaling: every
    rank owns a disjoint block of slices_per_rank consecutive slices)."""
    first = rank * slices_per_rank
    idx = list(range(first, first + slices_per_rank))
    return idx, [BASE_SEED + g for g in idx]


def reduce_max(value: float, world: int, device=None) -> float:
    """Max over ranks (identity at world size 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- model
def g_needed_floats(N: int, n1: int) -> int:
    """Floats of the first-pass output that the second pass reads, per quarter:
    sum over blocks bi and slopes tau of (N + (tau + 1) bi) columns."""
    R1 = 1 << n1
    nb = N // R1
    if nb == 1:
        return N * N
    return N * N + (R1 * (R1 + 1) // 2) * (nb * (nb - 1) // 2)


def byte_model(N: int, K: int, M: int, n1: int) -> dict:
    """Algorithmic bytes per slice.  S, Lin, Img as in the pass-plan model
    B_model = 3S + (2P+1) Lin + Img with P = ceil(log2 N / 6); per kernel, each kernel's
    inputs read once and outputs written once."""
    S = 4 * K * M
    Lin = 32 * N * N
    Img = 4 * N * N
    P = math.ceil(math.log2(N) / 6)
    G = 4 * 4 * g_needed_floats(N, n1)
    # charge_8d: the pass plan's per-step bytes assigned to the kernels that fuse those
    # steps -- filter 2S; resampling (S + Lin) plus the first Hough pass (2 Lin) for pass 1;
    # the last Hough pass (Lin + Lin/2) and the quarter sum (Lin/2 + Img) split between the
    # two second-pass launches, the image write charged to the v launch.
    charge_8d = dict(iir=2 * S, pass1_resample=S + (2 * (P - 1) + 1) * Lin,
                     pass2=Lin + Img, pass2_h=Lin)
    return dict(S=S, Lin=Lin, Img=Img, P=P, B_model=3 * S + (2 * P + 1) * Lin + Img,
                compulsory=S + Img, iir=2 * S, pass1_resample=S + G, pass2=G // 2 + Img,
                pass2_h=G // 2 + 2 * Img, G=G, charge_8d=charge_8d)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = list(csv.reader(io.StringIO(open(self.path).read())))
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [v.strip() for v in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle leg
def oracle_sample(sino64, N, b, a, taus_per_quarter, ys=None, xs=None, rows=None):
    """Time the CPU oracle, as it stands, on a bounded sample of one slice and extrapolate
    to seconds per slice: float64 recursive filtering of `rows` projection rows (all if
    None), float64 linogram of all four quarters, float64 dyadic-pattern back projection of
    `taus_per_quarter` slope rows per quarter.  Optionally also evaluates the float64 fast
    and direct reconstructions at pixels (ys, xs) for the quality figures."""
    import numpy as np

    import oracle
    K, M = sino64.shape
    out = {}
    sel = sino64 if rows is None else sino64[:rows]
    t0 = time.perf_counter()
    pt = oracle.iir_filter(sel, b, a)
    t_iir = (time.perf_counter() - t0) * (K / sel.shape[0])
    if rows is not None:
        pt = np.concatenate([pt, np.zeros((K - sel.shape[0], M))])   # timing only
    t0 = time.perf_counter()
    L = oracle.linogram(pt, N)
    t_lin = time.perf_counter() - t0
    taus = np.linspace(0, N - 1, taus_per_quarter).astype(int)
    t0 = time.perf_counter()
    for q in range(4):
        oracle.pattern_backproject(L[q], taus)
    t_bp = (time.perf_counter() - t0) * (N / taus_per_quarter)
    del L
    out["sec_per_slice"] = t_iir + t_lin + t_bp
    out["work_sec"] = None
    if ys is not None:
        full_pt = pt if rows is None else oracle.iir_filter(sino64, b, a)
        out["fast64"] = oracle.fast_fbp_pixels(sino64, N, b, a, ys, xs, pt=full_pt)
        out["direct64"] = oracle.direct_fbp_pixels(sino64, N, ys, xs)
    return out


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def _oracle_sample_worker(job):
    path, N, b, a, taus = job
    import numpy as np
    s64 = np.array(np.load(path, mmap_mode="r"))
    return oracle_sample(s64, N, np.array(b), np.array(a), taus_per_quarter=taus)["sec_per_slice"]


def oracle_all_cores(s64, N, b, a, taus):
    """The bounded oracle sample on every core at once, one slice per spawned process:
    returns (slices/s of all processes together, processes, wall seconds)."""
    import multiprocessing as mp

    import numpy as np
    cores = cpu_cores()
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    np.save(path, s64)
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    try:
        for k in saved:
            os.environ[k] = "1"                    # one thread per process
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(cores) as pool:
            secs = pool.map(_oracle_sample_worker, [(path, N, list(b), list(a), taus)] * cores)
        wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        os.unlink(path)
    return sum(1.0 / t for t in secs), cores, wall


# ----------------------------------------------------------------------------- traffic
def traffic_for(kernel: str, slices_per_launch: int):
    """ncu DRAM bytes per launch recorded in profiles/traffic.json for `kernel`, or None if
    absent, taken at another number of slices per launch, or if the kernel source changed
    since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec or rec.get("slices_per_launch") != slices_per_launch:
        return None
    src = os.path.join(ROOT, "paper_2007_06289_gb300", "csrc", rec["source"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return rec["bytes_per_launch"] if sha == rec["source_sha256_16"] else None


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    import phantoms
    from paper_2007_06289_gb300 import binding as fbp
    from paper_2007_06289_gb300 import build, iir_fit

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    fbp.load_library()

    N, S = args.N, args.slices
    K, M = phantoms.geometry_for(N)
    b, a = iir_fit.coefficients(N, args.order)
    idx, seeds = shard(rank, S)
    sino = torch.empty((S, K, M), dtype=torch.float32, device=dev)
    for j, sd in enumerate(seeds):
        sino[j] = phantoms.ellipse_sinogram_torch(phantoms.random_ellipses(sd), N, K, M, dev,
                                                  I0, sd * 7919 + 1).float()
    plan = fbp.fbp_plan(N, K, M, S, (list(b), list(a)))
    if args.chunk:
        fbp.fbp_set_chunk(plan, args.chunk)
    img = torch.empty(plan.img_shape, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        fbp.fbp_reconstruct(plan, sino, img)
    torch.cuda.synchronize(dev)

    # ---- timed region: K steps, per-kernel CUDA events recorded by the library
    fbp.fbp_profile_enable(plan, True)
    fbp.fbp_profile_reset(plan)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        fbp.fbp_reconstruct(plan, sino, img)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    ms_step = reduce_max(e0.elapsed_time(e1) / args.steps, world, dev)
    prof = fbp.fbp_profile_read(plan)
    fbp.fbp_profile_enable(plan, False)
    launches = sum(n for _, n in prof.values())

    # ---- end to end through the host-memory entry point (pinned buffers)
    h_sino = sino.cpu().pin_memory()
    h_img = torch.empty(plan.img_shape, dtype=torch.float32, pin_memory=True)
    fbp.fbp_reconstruct_host(plan, h_sino, h_img)
    torch.cuda.synchronize(dev)
    fbp.fbp_reconstruct_host(plan, h_sino, h_img)
    torch.cuda.synchronize(dev)
    # The copies bound this path (~210 GB/s host to device on this machine) and their rate
    # varies with what else the host is doing (single runs at twice the time): five timed
    # runs, the median reported.
    e2e_steps = max(1, min(args.steps, 10))
    e2e_runs = []
    for _ in range(5):
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(e2e_steps):
            fbp.fbp_reconstruct_host(plan, h_sino, h_img)
        f1.record(stream)
        f1.synchronize()
        e2e_runs.append(reduce_max(f0.elapsed_time(f1) / e2e_steps, world, dev))
    ms_e2e = statistics.median(e2e_runs)
    same = bool(torch.equal(h_img, img.cpu()))

    # ---- direct GPU FBP comparator on a few slices of the same stack
    D = args.direct_slices
    dplan = fbp.fbp_plan(N, K, M, D)
    dimg = torch.empty(dplan.img_shape, device=dev)
    dsino = sino[:D].contiguous()
    fbp.fbp_direct_reconstruct(dplan, dsino, dimg)
    torch.cuda.synchronize(dev)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(2):
        fbp.fbp_direct_reconstruct(dplan, dsino, dimg)
    g1.record(stream)
    g1.synchronize()
    ms_direct = g0.elapsed_time(g1) / 2
    dev_err = fbp.fbp_last_device_error(plan)

    if rank != 0:
        if world > 1:
            dist.barrier()
        return None

    # ---- numbers
    total_slices = S * world
    value = total_slices / (ms_step / 1e3)
    model = byte_model(N, K, M, plan.fuse_k)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    per_launch_slices = plan.chunk
    kern = {}
    for name in ("iir", "pass1_resample", "pass2", "pass2_h"):
        ms, n = prof[name]
        if n:
            sec = ms / n / 1e3
            rec = dict(ms_per_launch=ms / n, launches=n,
                       charge_8d_bytes=model["charge_8d"][name] * per_launch_slices,
                       own_bytes=model[name] * per_launch_slices,
                       traffic=traffic_for(name, plan.chunk))
            rec["frac_8d"] = rec["charge_8d_bytes"] / sec / 1e9 / hbm
            rec["frac_own"] = rec["own_bytes"] / sec / 1e9 / hbm
            rec["traffic_frac"] = None if rec["traffic"] is None else rec["traffic"] / sec / 1e9 / hbm
            kern[name] = rec
    dom = max(kern, key=lambda k: kern[k]["ms_per_launch"] * kern[k]["launches"])
    dk = kern[dom]
    achieved = dk["charge_8d_bytes"] / (dk["ms_per_launch"] / 1e3) / 1e9
    rnd = lambda v, d=4: None if v is None else round(v, d)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": dk["traffic"],
                "peak_source": peak_src,
                "achieved_basis": "pass-plan bytes of the steps the kernel fuses (x slices per launch)",
                "traffic_frac": rnd(dk["traffic_frac"]), "frac_own_bytes": rnd(dk["frac_own"]),
                "kernels": {k: {"ms_per_launch": round(v["ms_per_launch"], 5),
                                "launches": v["launches"],
                                "frac_8d": rnd(v["frac_8d"]),
                                "frac_own_bytes": rnd(v["frac_own"]),
                                "traffic_bytes": v["traffic"],
                                "traffic_frac": rnd(v["traffic_frac"])}
                            for k, v in kern.items()}}
    t_slice = ms_step / 1e3 / S
    pipeline = {"B_model_bytes_per_slice": model["B_model"],
                "frac_B_model_of_peak": round(model["B_model"] / (hbm * 1e9) / t_slice, 4),
                "compulsory_bytes_per_slice": model["compulsory"],
                "frac_compulsory_of_peak": round(model["compulsory"] / (hbm * 1e9) / t_slice, 4)}

    # the same stack with the order-6 filter of the default table (3x lower RMSE than the
    # paper's order 3 at N = 2048): its throughput and quality, beside the headline
    b6, a6 = iir_fit.coefficients(N, 6)
    plan6 = fbp.fbp_plan(N, K, M, S, (list(b6), list(a6)))
    if args.chunk:
        fbp.fbp_set_chunk(plan6, args.chunk)
    img6 = torch.empty(plan6.img_shape, device=dev)
    for _ in range(args.warmup):
        fbp.fbp_reconstruct(plan6, sino, img6)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    steps6 = max(1, min(args.steps, 10))
    for _ in range(steps6):
        fbp.fbp_reconstruct(plan6, sino, img6)
    h1.record(stream)
    h1.synchronize()
    ms6 = reduce_max(h0.elapsed_time(h1) / steps6, world, dev)

    # quality at sampled pixels of slice 0, and the CPU oracle baseline (one leg)
    rng = np.random.default_rng(0)
    P = args.sample_pixels
    ys, xs = rng.integers(0, N, P), rng.integers(0, N, P)
    fast_img = img[0].cpu().numpy()
    dir_img = dimg[0].cpu().numpy()
    truth = phantoms.ellipse_image(phantoms.random_ellipses(seeds[0]), N)
    img6_0 = img6[0].cpu().numpy()
    quality = {"pixels": P,
               "rmse_fast_vs_phantom": float(np.sqrt(np.mean((fast_img - truth) ** 2))),
               "rmse_direct_vs_phantom": float(np.sqrt(np.mean((dir_img - truth) ** 2))),
               "iir_order6": {"slices_per_s": round(total_slices / (ms6 / 1e3), 2),
                              "rmse_vs_phantom": float(np.sqrt(np.mean((img6_0 - truth) ** 2)))}}
    cpu_baseline = None
    if not args.no_cpu_baseline:
        s64 = sino[0].cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        res = oracle_sample(s64, N, b, a, taus_per_quarter=8, ys=ys, xs=xs)
        work = time.perf_counter() - t0
        f64, d64 = res["fast64"], res["direct64"]
        rng_img = float(fast_img.max() - fast_img.min())
        quality["iir_order6"]["rmse_vs_fp64_direct"] = float(np.sqrt(np.mean((img6_0[ys, xs] - d64) ** 2)))
        quality.update({
            "rmse_fast_vs_fp64_direct": float(np.sqrt(np.mean((fast_img[ys, xs] - d64) ** 2))),
            "rmse_direct_gpu_vs_fp64_direct": float(np.sqrt(np.mean((dir_img[ys, xs] - d64) ** 2))),
            "rmse_fp64_fast_vs_fp64_direct": float(np.sqrt(np.mean((f64 - d64) ** 2))),
            "max_abs_vs_fp64_fast_over_range": float(np.abs(fast_img[ys, xs] - f64).max() / rng_img),
        })
        v_all, cores_all, wall_all = oracle_all_cores(s64, N, b, a, 8)
        cpu_baseline = {"value": round(1.0 / res["sec_per_slice"], 6), "unit": UNIT,
                        "cores": 1, "kind": "oracle",
                        "sample": (f"one N={N} slice: float64 recursive filter of all {K} rows, "
                                   "float64 linogram of all four quarters, float64 dyadic-pattern "
                                   f"back projection of 8 of {N} slopes per quarter (scaled "
                                   f"x{N / 8:g}); single-threaded numpy; value_all: the same "
                                   "sample on every core at once, one slice per process"),
                        "work_seconds": round(work, 1),
                        "value_all": round(v_all, 6), "cores_all": cores_all,
                        "wall_seconds_all": round(wall_all, 1), "cpu_model": cpu_model()}

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded ten-ellipse phantoms, closed-form Radon transform, Poisson noise I0=1e5",
        "config": {"workload": f"N={N} K={K} M={M} stack of {S} noisy ellipse-phantom slices per GPU",
                   "N": N, "K": K, "M": M, "slices_per_gpu": S, "iir_order": args.order,
                   "fuse_k": plan.fuse_k, "chunk": plan.chunk,
                   "l2": "no flush: the per-step sinogram stack (%.2f GB) is larger than L2"
                         % (S * K * M * 4 / 1e9)},
        "voxels_per_s": round(value * N * N, 1),
        "roofline": roofline,
        "pipeline_roofline": pipeline,
        "e2e": {"value": round(total_slices / (ms_e2e / 1e3), 2), "unit": UNIT,
                "h2d_bytes_per_step": S * K * M * 4, "d2h_bytes_per_step": S * N * N * 4,
                "api": "fbp_reconstruct_host (pinned host buffers)", "matches_device_result": same,
                "ms_per_step_runs": [round(v, 3) for v in e2e_runs]},
        "gpu_launches": launches,
        "direct_gpu": {"value": round(D / (ms_direct / 1e3), 3), "unit": UNIT, "slices": D,
                       "speedup_fast_over_direct": round((S / ms_step) / (D / ms_direct), 1)},
        "quality": quality,
        "clocks": clocks,
        "cpu_baseline": cpu_baseline,
        "device_status": dev_err,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
    return line


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle as the reference arm: each step times a bounded sample of one slice
    of the same workload (float64 recursive filter of 192 of the K rows, float64 linogram,
    dyadic-pattern back projection of 2 slopes per quarter) and extrapolates to slices/s."""
    import numpy as np

    import phantoms
    from paper_2007_06289_gb300 import iir_fit

    rank, world, _ = dist_env()
    if rank != 0:
        return None
    N = args.N
    K, M = phantoms.geometry_for(N)
    b, a = iir_fit.coefficients(N, args.order)
    sd = BASE_SEED
    s64 = phantoms.ellipse_sinogram(phantoms.random_ellipses(sd), N, K, M, I0, sd * 7919 + 1)
    for _ in range(args.warmup):
        oracle_sample(s64, N, b, a, taus_per_quarter=2, rows=192)
    secs = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        secs.append(oracle_sample(s64, N, b, a, taus_per_quarter=2, rows=192)["sec_per_slice"])
    wall = time.perf_counter() - t0
    v = 1.0 / statistics.mean(secs)
    rows = min(192, K)
    sample = (f"per step, one N={N} slice: float64 recursive filter of {rows} of {K} rows "
              f"(x{K / rows:g}), float64 linogram of all four quarters, float64 dyadic-pattern "
              f"back projection of 2 of {N} slopes per quarter (x{N / 2:g})")
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(wall / args.steps * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"N={N} K={K} M={M} noisy ellipse-phantom slices", "N": N,
                       "K": K, "M": M, "iir_order": args.order},
            "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


# ----------------------------------------------------------------------------- ragged volume
RAGGED_SIZES = (256, 512, 1024, 2048)
RAGGED_SEED = 2022
RAGGED_DISTINCT = 4           # distinct phantoms per size, replicated over that size's slices


def run_ragged(args):
    """A volume of slices of mixed sizes in one fbp_volume_run (graph-captured, autotuned
    outside the timed region).  Slice i has N drawn uniformly from RAGGED_SIZES with seed
    RAGGED_SEED; each size's slices cycle through RAGGED_DISTINCT seeded noisy phantoms
    (every slice in its own buffers).  One step = one run over the whole volume."""
    import numpy as np
    import torch

    import phantoms
    from paper_2007_06289_gb300 import binding as fbp

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(RAGGED_SEED + rank)
    sizes = rng.choice(RAGGED_SIZES, size=args.ragged_slices)
    proto = {}
    for N in RAGGED_SIZES:
        proto[N] = phantoms.phantom_stack_torch(int(N), RAGGED_DISTINCT, RAGGED_SEED * 10 + N,
                                                dev, noise_i0=I0)
    items, seen = [], {N: 0 for N in RAGGED_SIZES}
    for N in sizes:
        N = int(N)
        sino = proto[N][seen[N] % RAGGED_DISTINCT].clone()
        seen[N] += 1
        items.append((N, sino, torch.empty((N, N), device=dev)))
    stream = torch.cuda.Stream(dev)
    vol = fbp.fbp_volume_create(items, order=args.order, graph=True)
    choices = vol.tune(stream)
    for _ in range(max(3, args.warmup)):
        vol.run(stream)
    stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        vol.run(stream)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, world, dev)
    groups = [vol.group(g) for g in range(vol.info()["groups"])]
    total = args.ragged_slices * world
    voxels = sum(int(N) * int(N) for N in sizes) * world
    line = {"metric": "slices/s of a ragged volume (N uniform in {256,512,1024,2048})",
            "value": round(total / (ms / 1e3), 2), "unit": "slices/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": f"synthetic: {RAGGED_DISTINCT} seeded noisy ellipse phantoms per size, "
                    "replicated; every slice in its own buffers",
            "config": {"workload": f"ragged volume of {args.ragged_slices} slices per GPU",
                       "slices_per_size": {str(N): int((sizes == N).sum()) for N in RAGGED_SIZES},
                       "graph": True,
                       "groups": [{k: g[k] for k in ("N", "items", "fuse_k", "chunk")}
                                  for g in groups],
                       "l2": "no flush: the volume's sinograms (GBs) exceed L2"},
            "voxels_per_s": round(voxels / (ms / 1e3), 1),
            "tuned": [list(c) for c in choices],
            "clocks": clocks,
            "gpu_launches": args.steps * sum(
                -(-g["items"] // g["chunk"]) * (4 if g["N"] > 64 else 3) for g in groups)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return line


def run_adjoint(args):
    """Forward reconstruction and its adjoint (the gradient with respect to the sinograms)
    on a batch of 32 noisy phantom slices of N = 512 (K = 768, M = 725).  One step = one
    adjoint pass over the batch; the forward pass is timed the same way beside it."""
    import torch

    import phantoms
    from paper_2007_06289_gb300 import binding as fbp

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    N, B = 512, 32
    K, M = phantoms.geometry_for(N)
    sino = phantoms.phantom_stack_torch(N, B, 2023 + rank * B, dev, noise_i0=I0)
    plan = fbp.fbp_plan(N, K, M, B)
    img = torch.empty(plan.img_shape, device=dev)
    grad = torch.empty(plan.sino_shape, device=dev)
    w = torch.randn(plan.img_shape, device=dev, generator=torch.Generator(device=dev).manual_seed(3))
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return reduce_max(e0.elapsed_time(e1) / args.steps, world, dev)

    sampler = ClockSampler(local)
    sampler.start()
    ms_fwd = timed(lambda: fbp.fbp_reconstruct(plan, sino, img))
    ms_adj = timed(lambda: fbp.fbp_reconstruct_adjoint(plan, w, grad))
    clocks = sampler.stop()
    n = plan.N.bit_length() - 1
    line = {"metric": "slices/s of the adjoint (sinogram gradient) at N=512, batch 32",
            "value": round(B * world / (ms_adj / 1e3), 2), "unit": "slices/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms_adj, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded noisy ellipse phantoms (gradient: seeded normal image)",
            "config": {"workload": "adjoint of the fast FBP, N=512 K=768 M=725, batch 32",
                       "N": N, "K": K, "M": M, "batch": B, "chunk": plan.chunk,
                       "l2": "no flush: per-step buffers (sinogram gradients, linogram-"
                             "sized ping-pong buffers) exceed L2"},
            "forward": {"value": round(B * world / (ms_fwd / 1e3), 2), "unit": "slices/s",
                        "ms_per_step": round(ms_fwd, 4)},
            "clocks": clocks,
            # per chunk: ceil(n / 5) fused transposed-stage launches, the resampling
            # adjoint, the filter
            "gpu_launches": args.steps * -(-B // plan.chunk) * (-(-n // 5) + 1 + 1)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return line


def run_corrector(args):
    """The learned corrector, and the quality of every form of the reconstruction.

    Training (outside the timed region): --train-pairs (fast FBP, direct GPU FBP) pairs of
    N = 512 seeded noisy phantoms, generated on the GPU by the library's own kernels, and
    --train-steps Adam steps of batch 16 through the library's forward and backward kernels.
    Timed: inference over 16 fast reconstructions of N = 2048 (one step = one fbp_cnn_forward
    over the batch); beside it the throughput of every form.  Quality at N = 2048 (the first
    --direct-slices slices): RMSE against the phantom (whole images) and against the float64
    direct FBP (--sample-pixels pixels of slice 0, CPU oracle) of the fast reconstruction with
    the default filter table, with the table fitted against the direct FBP, with the paper's
    impulse-response-MSE fit, with the exact FIR filter (which isolates the dyadic lines'
    share of the error), the corrected fast reconstructions (one corrector trained on the
    order-3 images, one on the order-6 images, both against the direct FBP) and the direct GPU
    FBP.  The
    dominant kernel is the bf16 tensor-core 3x3 convolution (5 of the 6 layers: the four
    32 -> 32 layers and the 32 -> 1 layer)."""
    import numpy as np
    import torch

    import oracle
    import phantoms
    from paper_2007_06289_gb300 import binding as fbp
    from paper_2007_06289_gb300 import corrector, iir_fit, iir_fit_direct

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    fbp.load_library()

    def rmse(a, b):
        return float(torch.sqrt(torch.mean((a.double() - b.double()) ** 2)))

    # ---- training pairs, generated in chunks on the GPU
    t0 = time.perf_counter()
    Nt, P, held = 512, args.train_pairs, 32
    Kt, Mt = phantoms.geometry_for(Nt)
    fast512 = torch.empty(P + held, Nt, Nt, device=dev)          # order-3 filter (the paper's)
    fast512_6 = torch.empty(P + held, Nt, Nt, device=dev)        # order-6 filter
    direct512 = torch.empty(P + held, Nt, Nt, device=dev)
    chunk = 500
    fplan = fbp.fbp_plan(Nt, Kt, Mt, chunk)
    b6, a6 = iir_fit.coefficients(Nt, 6)
    fplan6 = fbp.fbp_plan(Nt, Kt, Mt, chunk, (list(b6), list(a6)))
    dplan = fbp.fbp_plan(Nt, Kt, Mt, chunk)
    for c0 in range(0, P + held, chunk):
        n = min(chunk, P + held - c0)
        sino = phantoms.phantom_stack_torch(Nt, chunk, 4000 + rank * (P + held) + c0, dev, noise_i0=I0)
        fout = torch.empty(chunk, Nt, Nt, device=dev)
        dout = torch.empty(chunk, Nt, Nt, device=dev)
        fbp.fbp_reconstruct(fplan, sino, fout)
        fast512[c0:c0 + n] = fout[:n]
        fbp.fbp_reconstruct(fplan6, sino, fout)
        fast512_6[c0:c0 + n] = fout[:n]
        fbp.fbp_direct_reconstruct(dplan, sino, dout)
        direct512[c0:c0 + n] = dout[:n]
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, losses = corrector.train(fast512[:P], direct512[:P], steps=args.train_steps, batch=16,
                                     lr=2e-3, seed=0)
    params6, losses6 = corrector.train(fast512_6[:P], direct512[:P], steps=args.train_steps,
                                       batch=16, lr=2e-3, seed=0)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    hs = slice(P, P + held)
    q512 = {"rmse_fast_vs_direct": rmse(fast512[hs], direct512[hs]),
            "rmse_corrected_vs_direct": rmse(corrector.infer(params, fast512[hs].contiguous()),
                                              direct512[hs]),
            "rmse_fast_order6_vs_direct": rmse(fast512_6[hs], direct512[hs]),
            "rmse_corrected_order6_vs_direct": rmse(corrector.infer(params6, fast512_6[hs].contiguous()),
                                                     direct512[hs])}
    del fast512, fast512_6, direct512

    # ---- the forms at N = 2048
    N, B = 2048, min(16, args.slices)
    K, M = phantoms.geometry_for(N)
    base = 2025 + rank * B
    sino = phantoms.phantom_stack_torch(N, B, base, dev, noise_i0=I0)
    D = min(args.direct_slices, B)
    forms = {
        "fast": iir_fit.coefficients(N, 3),
        "fast_direct_fit": iir_fit_direct.direct_coefficients(N, 3),
        "fast_order6": iir_fit.coefficients(N, 6),
        "fast_order6_direct_fit": iir_fit_direct.direct_coefficients(N, 6),
        "fast_paper_mse_fit": iir_fit.mse_coefficients(N),
    }
    plans = {k: fbp.fbp_plan(N, K, M, B, (list(b), list(a))) for k, (b, a) in forms.items()}
    shared_ws = torch.empty(fbp.fbp_workspace_bytes(plans["fast"]), dtype=torch.uint8, device=dev)
    for pl in plans.values():
        fbp.fbp_set_workspace(pl, shared_ws)
    imgs = {k: torch.empty(B, N, N, device=dev) for k in plans}
    for k, pl in plans.items():
        fbp.fbp_reconstruct(pl, sino, imgs[k])
    # the exact FIR filter, then the fast back projection (the dyadic lines' share of the
    # error; the paper's own FHT-with-FIR configuration)
    filt = torch.empty(B, K, M, device=dev)
    lin = torch.empty(plans["fast"].lin_shape, device=dev)
    fir_fast = torch.empty(B, N, N, device=dev)

    def fir_form():
        fbp.fbp_filter_fir(plans["fast"], sino, filt)
        fbp.fbp_resample_st(plans["fast"], filt, lin)
        fbp.fbp_fht_backproject(plans["fast"], lin, fir_fast)

    fir_form()
    ws = torch.empty(fbp.fbp_cnn_workspace_bytes(N, B, False), dtype=torch.uint8, device=dev)
    corrected = torch.empty(B, N, N, device=dev)
    fbp.fbp_cnn_forward(params, imgs["fast"], corrected, ws)
    corrected6 = torch.empty(B, N, N, device=dev)
    fbp.fbp_cnn_forward(params6, imgs["fast_order6"], corrected6, ws)
    direct = torch.empty(D, N, N, device=dev)
    dplan2 = fbp.fbp_plan(N, K, M, D)
    fbp.fbp_direct_reconstruct(dplan2, sino[:D].contiguous(), direct)
    torch.cuda.synchronize(dev)
    cnn_status = fbp.fbp_cnn_last_error()

    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return reduce_max(e0.elapsed_time(e1) / steps, world, dev)

    sampler = ClockSampler(local)
    sampler.start()
    ms_inf = timed(lambda: fbp.fbp_cnn_forward(params, imgs["fast"], corrected, ws), args.steps)
    ms_form = {k: timed(lambda k=k: fbp.fbp_reconstruct(plans[k], sino, imgs[k]), args.steps)
               for k in plans}
    ms_fast = ms_form["fast"]
    ms_fir = timed(fir_form, 3)
    ms_direct = timed(lambda: fbp.fbp_direct_reconstruct(dplan2, sino[:D].contiguous(), direct), 2)
    xt = imgs["fast"][:4].contiguous()
    tt = imgs["fast"][:4].contiguous()
    pt = params.clone().requires_grad_(True)

    def train_step():
        loss = torch.mean((corrector.correct(pt, xt) - tt) ** 2)
        loss.backward()
        pt.grad = None

    ms_train = timed(train_step, max(3, args.steps // 3))
    clocks = sampler.stop()

    # quality: against the phantoms (whole images of the first D slices) and against the
    # float64 direct FBP (sampled pixels of slice 0)
    truth = torch.stack([torch.from_numpy(phantoms.ellipse_image(phantoms.random_ellipses(base + i), N))
                         for i in range(D)]).to(dev)
    rng = np.random.default_rng(0)
    ys, xs = rng.integers(0, N, args.sample_pixels), rng.integers(0, N, args.sample_pixels)
    d64 = oracle.direct_fbp_pixels(sino[0].cpu().numpy().astype(np.float64), N, ys, xs)

    def q(img):
        at = img[0].cpu().numpy()[ys, xs].astype(np.float64)
        return {"rmse_vs_phantom": round(rmse(img[:D], truth), 6),
                "rmse_vs_fp64_direct": round(float(np.sqrt(np.mean((at - d64) ** 2))), 6)}

    quality = {k: q(v) for k, v in imgs.items()}
    quality["fast_exact_fir_filter"] = q(fir_fast)
    quality["corrected"] = q(corrected)
    quality["corrected_order6"] = q(corrected6)
    quality["direct_gpu"] = q(direct)
    sps = lambda ms, n: round(n * world / (ms / 1e3), 2)
    throughput = {k: sps(v, B) for k, v in ms_form.items()}
    throughput.update({"fast_exact_fir_filter": sps(ms_fir, B),
                       "corrected": sps(ms_fast + ms_inf, B),
                       "corrected_order6": sps(ms_form["fast_order6"] + ms_inf, B),
                       "direct_gpu": sps(ms_direct, D)})
    flops_px = 2 * (32 * 9) + 4 * 2 * (32 * 32 * 9) + 2 * (32 * 9)
    tflops = B * N * N * flops_px / (ms_inf / 1e3) / 1e12
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    pk = json.load(open(peaks)) if os.path.exists(peaks) else {}
    peak = pk.get("bf16_tflops_sustained") or 1700.0
    line = {"metric": "slices/s of the learned corrector (inference) at N=2048",
            "value": round(B * world / (ms_inf / 1e3), 2), "unit": "slices/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms_inf, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic: seeded noisy ellipse phantoms; corrector weights trained in this "
                    "run on N=512 (fast, direct GPU FBP) pairs made by the library",
            "config": {"workload": f"CNN corrector, 6 layers 3x3, 32 channels, N=2048 batch {B}",
                       "training": f"{args.train_steps} Adam steps, batch 16, lr 2e-3, "
                                   f"{P} N=512 pairs (+{held} held out)",
                       "l2": "no flush: bf16 activations of the batch exceed L2"},
            "roofline": {"bound": "tensor", "kernel": "whole corrector (5 tensor-core layers + "
                                                      "1 fp32 layer)",
                         "achieved": round(tflops, 1), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(tflops / peak, 4), "traffic": None,
                         "peak_source": "measured bf16, sustained (timed inside a long step)"},
            "quality_N2048": quality,
            "throughput_N2048_slices_per_s": throughput,
            "quality_N512_held_out_32": q512,
            "training": {"loss_first_last": [round(losses[0], 6), round(losses[-1], 6)],
                         "loss_first_last_order6": [round(losses6[0], 6), round(losses6[-1], 6)],
                         "pair_generation_seconds": round(gen_s, 1),
                         "train_seconds": round(train_s, 1)},
            "training_step_ms_N2048_batch4": round(ms_train, 3),
            "clocks": clocks, "cnn_status": cnn_status,
            "gpu_launches": args.steps * 11}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return line


def run_sirt(args):
    """Algebraic reconstruction (SIRT on the fast Hough operators) of 16 noisy phantom slices
    of N = 512 (K = 768, M = 725), started from the fast FBP image.  One step = 10 SIRT
    iterations over the batch; metric slice-iterations/s.  Quality: RMSE to the phantom of
    the fast FBP and of SIRT after 10 and 50 iterations from it (first 2 slices)."""
    import numpy as np
    import torch

    import phantoms
    from paper_2007_06289_gb300 import binding as fbp

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    N, B, IT, LAM = 512, 16, 10, 1.0
    K, M = phantoms.geometry_for(N)
    seed = 2025 + rank * B
    sino = phantoms.phantom_stack_torch(N, B, seed, dev, noise_i0=I0)
    plan = fbp.fbp_plan(N, K, M, B)
    data = torch.empty(plan.lin_shape, device=dev)
    fbp.fbp_hough_data(plan, sino, data)
    img0 = torch.empty(plan.img_shape, device=dev)
    fbp.fbp_reconstruct(plan, sino, img0)
    img = img0.clone()
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        fbp.fbp_sirt(plan, data, img, IT, LAM)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        fbp.fbp_sirt(plan, data, img, IT, LAM)
    e1.record(stream)
    e1.synchronize()
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, world, dev)
    # the fast Radon transform of the same batch (image -> (theta, r) sinogram), timed alike
    rsino = torch.empty(plan.sino_shape, device=dev)
    for _ in range(max(3, args.warmup)):
        fbp.fbp_radon(plan, img0, rsino)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.steps):
        fbp.fbp_radon(plan, img0, rsino)
    e1.record(stream)
    e1.synchronize()
    ms_radon = reduce_max(e0.elapsed_time(e1) / args.steps, world, dev)
    clocks = sampler.stop()
    # quality on the first two slices
    truth = np.stack([phantoms.ellipse_image(phantoms.random_ellipses(seed + s), N) for s in range(2)])

    def rmse(x):
        return float(np.sqrt(np.mean((x[:2].cpu().numpy().astype(np.float64) - truth) ** 2)))

    q = {"rmse_fast_fbp": rmse(img0)}
    img = img0.clone()
    fbp.fbp_sirt(plan, data, img, 10, LAM)
    q["rmse_sirt_10_from_fbp"] = rmse(img)
    fbp.fbp_sirt(plan, data, img, 40, LAM)
    q["rmse_sirt_50_from_fbp"] = rmse(img)
    n = N.bit_length() - 1
    # per chunk and iteration: the fused projection launches (the last one forms the
    # residual), the two or three back-projection passes, the update
    per_iter = -(-n // 5) + 2 + (1 if plan.fuse_k < n else 0) + 1
    line = {"metric": "slice-iterations/s of SIRT on the fast Hough operators at N=512, batch 16",
            "value": round(B * IT * world / (ms / 1e3), 1), "unit": "slice-iterations/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded noisy ellipse phantoms (Poisson, I0 = 1e5), Hough-space data",
            "config": {"workload": "SIRT, N=512 K=768 M=725, batch 16, 10 iterations per step, "
                                   "lambda 1, started from the fast FBP", "N": N, "K": K, "M": M,
                       "batch": B, "iterations_per_step": IT,
                       "l2": "no flush: per-step buffers (data and linogram-sized work arrays, "
                             "134 MB each) exceed L2"},
            "ms_per_iteration_per_slice": round(ms / IT / B, 5),
            "quality": q,
            "fast_radon": {"value": round(B * world / (ms_radon / 1e3), 1), "unit": "slices/s",
                           "ms_per_step": round(ms_radon, 4),
                           "what": "fbp_radon of the 16 images (not in the timed SIRT steps)"},
            "clocks": clocks,
            "gpu_launches": args.steps * IT * -(-B // plan.chunk) * per_iter}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return line


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ragged":
        run_ragged(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "corrector":
        run_corrector(args)
    elif args.workload == "sirt":
        run_sirt(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
