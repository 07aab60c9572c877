#!/usr/bin/env python
"""Benchmark of the GB300 smooth-and-clip library (one JSON line on stdout).

Metric: S+C voxel*kernels/s, i.e. cube voxels x kernel pairs processed per
second, for plain float32 S+C on a WALLABY-shaped synthetic cube
(1200 x 1200 x 1024, spatial {0,3,6} x spectral {0,3,7,15}, t = 3.5, MAD
noise, replacement 2.0), cube resident in HBM, sigma copied to the host every
step. The cube (5.9 GB) is larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas, one cube per rank (weak
scaling; S+C of one cube needs no exchange between GPUs). --impl reference
times the FP64 CPU oracle on bounded samples of the same workload.
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

METRIC = "S+C voxel·kernels/s on 1 GB300 (FP32 plain vs batched/BF16), % HBM roofline"
UNIT = "voxel·kernels/s"
SMOOTH_BYTES_PER_VOXEL = 4.0 + 4.0 + 1.0 / 8.0  # read C, write S, read the 1-bit mask
STORE_BYTES_PER_VOXEL = SMOOTH_BYTES_PER_VOXEL + 8.0  # the same, also writing the int64 spatial sums P'
SHARED_BYTES_PER_VOXEL = 8.0 + 4.0  # read P', write S (the correction lists add ~0.1 %)
WORKLOADS = ("wallaby", "medium", "small", "batch64", "small-bf16", "small-fp16", "wallaby-bf16", "wallaby-fp16",
             "stream512", "wallaby-noisescale", "medium-noisescale", "wallaby-link", "wallaby-autoflag",
             "wallaby-gauss", "medium-gauss", "wallaby-noisescale-gauss", "wallaby-autoflag-gauss",
             "wallaby-sampled", "medium-sampled", "small-sampled", "medium-fp16", "medium-bf16")
FLAG_METRIC = "auto-flagger voxels/s on 1 GB300 (channel and pixel MAD noise, k = 4)"
LINK_METRIC = "linker voxels/s on 1 GB300 (friends-of-friends, radius 2, minimum sizes 8 px / 5 ch)"
NOISE_SCALE_METRIC = "local noise normalisation voxels/s on 1 GB300 (31-voxel windows, 16-voxel cells)"


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x, pg, device=None):
    """The maximum of x over all ranks (x itself without a process group).
    Works with gloo (CPU tensors) and NCCL (tensors on `device`)."""
    if pg is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(voxels_per_rank, n_pairs, steps, world, seconds):
    """Whole-job S+C throughput: every rank runs its own cube (replicas), so
    the job processes world x voxels x pairs per step in the slowest rank's time."""
    return voxels_per_rank * n_pairs * steps * world / seconds


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


SMOOTH_SOURCES = ("sc_smooth.cu", "sc_smooth_ws.cu", "sc_smooth_ws.cuh", "sc_smooth_fir.cu", "sc_smooth_ws16.cu", "sc_smooth_tile.cu",
                  "sc_smooth_z.cu", "sc_smooth_p.cu", "sc_tile_common.cuh",
                  "sc_device.cuh")  # the smoothing kernels' code (declarations elsewhere do not change their traffic)


def smooth_source_hash():
    """First 16 hex digits of the SHA-256 of the smoothing kernels' sources."""
    h = hashlib.sha256()
    for name in SMOOTH_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_15789_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def smooth_traffic_record():
    """DRAM bytes per voxel of each smoothing kernel from the committed ncu
    summary, if it was taken on the current kernel sources (else None)."""
    rec = os.path.join(ROOT, "profiles", "smooth_traffic.json")
    try:
        with open(rec) as f:
            r = json.load(f)
        return r if r.get("source_sha256_16") == smooth_source_hash() else None
    except Exception:
        return None


TRAFFIC_WORKLOAD_VOXELS = 512 ** 3  # the medium workload, whose every smoothing launch covers the whole cube


def record_traffic(specs, command):
    """Write profiles/smooth_traffic.json from one-kernel ncu captures of the
    medium workload: specs are "key=path" pairs, each path an ncu --csv log of
    dram__bytes_read.sum and dram__bytes_write.sum for a few launches of the
    kernel named key (as pair_kernels names it). The record holds the mean
    DRAM bytes per output voxel of each, keyed by the current smoothing-source
    hash."""
    import csv

    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    per_key = {}  # key -> {(path, launch id): bytes}; a key may be given several captures
    for spec in specs:
        key, path = spec.split("=", 1)
        per_launch = per_key.setdefault(key, {})
        with open(path) as f:
            rows = [r for r in csv.reader(f) if len(r) >= 15]
        head = rows[0]
        ci = {k: head.index(k) for k in ("ID", "Metric Name", "Metric Unit", "Metric Value")}
        for r in rows[1:]:
            if r[ci["Metric Name"]] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                continue
            b = float(r[ci["Metric Value"]].replace(",", "")) * scale[r[ci["Metric Unit"]]]
            lid = (path, r[ci["ID"]])
            per_launch[lid] = per_launch.get(lid, 0.0) + b
    kernels = {k: round(sum(v.values()) / len(v) / TRAFFIC_WORKLOAD_VOXELS, 3) for k, v in per_key.items()}
    launches = {k: len(v) for k, v in per_key.items()}
    rec = {"source_sha256_16": smooth_source_hash(),
           "what": "DRAM bytes (read + write) per output voxel of one launch, mean over the captured launches, from "
                   "one-kernel ncu captures (dram__bytes_read.sum + dram__bytes_write.sum, a few launches each) of "
                   "the medium 512^3 workload (larger than L2); traffic is proportional to voxels, so the bench "
                   "scales it to the launch's voxels",
           "command": command, "kernels": kernels, "launches": launches}
    with open(os.path.join(ROOT, "profiles", "smooth_traffic.json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec["kernels"]))
    return 0


def smoothing_kernel_name(sc, pair, code, sampled=False):
    """Name of the smoothing kernel a pair ran on, from the SC_KERNEL_* code
    the library reports for it and the pair's cascade widths (or, for the
    sampled Gaussian, its FWHM)."""
    fwhm, _ = pair
    w = tuple(sc.sc_cascade_widths(fwhm)) if fwhm > 0 else (1, 1, 1)
    if sampled and fwhm > 0:
        names = {sc.SC_KERNEL_Z: "k_smooth_z", getattr(sc, "SC_KERNEL_FIR", -1): "k_smooth_ws<sampled %g px>" % fwhm,
                 sc.SC_KERNEL_SHARED: "k_smooth_p<sampled %g px>" % fwhm, sc.SC_KERNEL_GENERIC: "k_smooth_generic"}
        return names.get(code, "unknown")
    names = {sc.SC_KERNEL_NONE: "none", sc.SC_KERNEL_IDENTITY: "k_identity", sc.SC_KERNEL_Z: "k_smooth_z",
             sc.SC_KERNEL_WS32: "k_smooth_ws<%d,%d,%d>" % w, sc.SC_KERNEL_WS16: "k_smooth_ws<%d,%d,%d>/16" % w,
             sc.SC_KERNEL_TILE: "k_smooth_tile<%d,%d,%d>" % w, sc.SC_KERNEL_GENERIC: "k_smooth_generic",
             sc.SC_KERNEL_SHARED: "k_smooth_p<%d,%d,%d>" % w,
             getattr(sc, "SC_KERNEL_FIR", -1): "k_smooth_ws<sampled %g px>" % fwhm}
    return names.get(code, "unknown")


class ClockSampler:
    """nvidia-smi clock / throttle samples of one GPU while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
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
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def make_workload(name: str, rank: int, device: str):
    import torch

    from synth.cubes import SMALL, WALLABY, CubeSpec, make_cube

    if name == "wallaby":
        spec = WALLABY
    elif name == "medium":
        spec = CubeSpec(nx=512, ny=512, nz=512, seed=WALLABY.seed, n_gal=300, snr=WALLABY.snr, snr_log=True,
                        fwhm_xy=WALLABY.fwhm_xy, fwhm_z=WALLABY.fwhm_z, ripple=0.1, nan_border=16,
                        name="medium-512x512x512")
    else:
        spec = SMALL
    if rank:
        spec = CubeSpec(**{**spec.__dict__, "seed": spec.seed + 1000 * rank})
    with torch.no_grad():
        cube = make_cube(spec, device=device)
    return spec, cube


SUB_SHAPE = (256, 192, 192)  # (z, y, x) of one oracle sub-cube


def interior_subcubes(shape, count, border=16, sub=SUB_SHAPE):
    """Corners (z, y, x) of `count` disjoint sub-cubes of shape `sub` inside
    the cube, clear of a NaN border of `border` voxels in x and y, in z-major
    order (fewer if the cube holds fewer)."""
    nz, ny, nx = shape
    sz, sy, sx = min(sub[0], nz), min(sub[1], max(1, ny - 2 * border)), min(sub[2], max(1, nx - 2 * border))
    by0 = border if ny > 2 * border else 0
    bx0 = border if nx > 2 * border else 0
    out = []
    for z in range(0, nz - sz + 1, sz):
        for y in range(by0, ny - by0 - sy + 1, sy):
            for x in range(bx0, nx - bx0 - sx + 1, sx):
                out.append((z, y, x))
                if len(out) == count:
                    return out, (sz, sy, sx)
    return out, (sz, sy, sx)


def _oracle_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_job(job):
    """One pool worker: S+C of one sub-cube with the oracle, timed after all
    workers have their data (the barrier), one thread."""
    sub, kernels, t, n_repl, mode, spatial = job
    from oracle.sc_oracle import sc_filter

    _BARRIER.wait()
    t0 = time.perf_counter()
    sc_filter(sub, kernels, t, mode, n_repl, spatial=spatial)
    return time.perf_counter() - t0


def oracle_pool(subs, kernels, t, n_repl, mode, rounds=1, spatial="cascade"):
    """The oracle on the host cores: one spawned process per sub-cube, each
    single-threaded, all starting together; per round, the aggregate
    voxel*kernels/s is the sub-cubes' voxels x pairs over the slowest worker's
    time. Returns (rates per round, seconds per round)."""
    import multiprocessing as mp

    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")  # never fork a process that holds a CUDA context
        barrier = ctx.Barrier(len(subs))
        rates, secs = [], []
        with ctx.Pool(len(subs), initializer=_oracle_init, initargs=(barrier,)) as pool:
            for _ in range(rounds):
                times = pool.map(_oracle_job, [(x, kernels, t, n_repl, mode, spatial) for x in subs], chunksize=1)
                secs.append(max(times))
                rates.append(sum(x.size for x in subs) * len(kernels) / max(times))
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return rates, secs


def oracle_workers():
    return max(1, min(os.cpu_count() or 1, 64))


def cpu_baseline(cube_dev, kernels, t, n_repl, mode="mad", spatial="cascade"):
    """The FP64 oracle as it stands on all host cores (up to 64 processes):
    one interior 192 x 192 x 256 sub-cube of the same cube per process; plus
    the same sub-cube size on one thread for reference."""
    n = oracle_workers()
    corners, (sz, sy, sx) = interior_subcubes(tuple(cube_dev.shape), n)
    subs = [cube_dev[z:z + sz, y:y + sy, x:x + sx].float().cpu().numpy() for z, y, x in corners]
    rates, secs = oracle_pool(subs, kernels, t, n_repl, mode, spatial=spatial)
    rate1, secs1 = oracle_pool(subs[:1], kernels, t, n_repl, mode, spatial=spatial)
    return {"value": rates[0], "unit": UNIT, "cores": len(subs), "kind": "oracle",
            "value_one_thread": rate1[0],
            "sample": f"{len(subs)} disjoint interior {sx}x{sy}x{sz} sub-cubes of the same cube (one per host process, "
                      f"os.cpu_count() = {os.cpu_count()}), {len(kernels)} pairs each, numpy float64, "
                      f"{secs[0]:.1f} s; one sub-cube on one thread: {secs1[0]:.1f} s"}


def run_reference(args, rank, world):
    """The oracle on the host cores: each step is one round of the CPU
    baseline's sample (interior sub-cubes of the same WALLABY-shaped cube, one
    process per core)."""
    if rank != 0:
        return 0
    import torch

    from synth.cubes import KERNELS_12, SC_REPLACEMENT, SC_THRESHOLD, SMALL, WALLABY, make_cube

    mode = "gauss" if args.workload.endswith("-gauss") else "mad"
    dev = "cuda" if torch.cuda.is_available() else "cpu"  # the input generator only; S+C runs on the host
    with torch.no_grad():
        cube = make_cube(WALLABY if args.ref_cube == "wallaby" else SMALL, device=dev)
    n = oracle_workers()
    corners, (sz, sy, sx) = interior_subcubes(tuple(cube.shape), n)
    subs = [cube[z:z + sz, y:y + sy, x:x + sx].float().cpu().numpy() for z, y, x in corners]
    del cube
    rates, secs = oracle_pool(subs, KERNELS_12, SC_THRESHOLD, SC_REPLACEMENT, mode, rounds=args.warmup + args.steps)
    rates, secs = rates[args.warmup:], secs[args.warmup:]
    total = sum(secs)
    value = sum(x.size for x in subs) * len(KERNELS_12) * len(secs) / total
    sample = (f"{len(subs)} disjoint interior {sx}x{sy}x{sz} sub-cubes of the {args.ref_cube} cube per step (one "
              f"host process each, os.cpu_count() = {os.cpu_count()}), {len(KERNELS_12)} pairs, numpy float64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args.workload, KERNELS_12, mode),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": len(subs), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_dict(workload, kernels, mode="mad"):
    from synth.cubes import SC_REPLACEMENT, SC_THRESHOLD

    names = {"wallaby": "wallaby-1200x1200x1024", "medium": "medium-512x512x512", "small": "small-64x64x128",
             "small-bf16": "small-64x64x128 stored as BF16 + per-channel float32 scales",
             "small-fp16": "small-64x64x128 stored as FP16 + per-channel float32 scales",
             "wallaby-bf16": "wallaby-1200x1200x1024 stored as BF16 + per-channel float32 scales",
             "wallaby-fp16": "wallaby-1200x1200x1024 stored as FP16 + per-channel float32 scales",
             "medium-bf16": "medium-512x512x512 stored as BF16 + per-channel float32 scales",
             "medium-fp16": "medium-512x512x512 stored as FP16 + per-channel float32 scales",
             "batch64": "batch-64-subcubes-x,y~logU[128,512]-z~logU[256,1024]"}
    workload = workload.removesuffix("-gauss")
    sampled = workload.endswith("-sampled")
    workload = workload.removesuffix("-sampled")
    half = workload.endswith(("-bf16", "-fp16"))
    precision = ("%s cube + per-channel float32 scales, read as 16-bit values by the kernels, exact fixed-point "
                 "smoothing" % workload.split("-")[-1].upper()) if half else "float32 cube, exact fixed-point smoothing"
    big = workload in ("wallaby", "wallaby-bf16", "wallaby-fp16")
    return {"workload": names[workload], "kernels": "spatial {0,3,6} px x spectral {0,3,7,15} ch",
            "spatial_kernel": "sampled Gaussian (integer taps within 4 sigma)" if sampled else "3-box cascade",
            "n_pairs": len(kernels), "threshold": SC_THRESHOLD, "noise": mode, "replacement": SC_REPLACEMENT,
            "precision": precision, "l2": "inputs (cube 5.9 GB) larger than L2"
            if big else ("inputs (10.9 GB of sub-cubes) larger than L2" if workload == "batch64" else "no flush")}


def gauss_hist_roofline(st, peak, peak_kind):
    """Roofline of the Gaussian-fit histogram pass: 4 algorithmic bytes per
    value read (the float32 array; the 2 KiB of counts are negligible), over
    its live CUDA-event time."""
    if not st["ms_gauss_hist"] > 0:
        return None
    gbs = st["gauss_hist_values"] * 4.0 / (st["ms_gauss_hist"] * 1e-3) / 1e9
    return {"kernel": "k_gauss_hist", "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak, "peak_kind": peak_kind, "bytes_per_value": 4, "traffic": None}


def pair_kernels(sc, kernels, codes, sampled=False, cube_bytes=4.0):
    """(kernel name, algorithmic bytes per voxel) of every pair: a full
    smoothing pass reads C and the mask bits and writes S; the first pair of a
    run that the next pairs share also writes its int64 spatial sums; a shared
    pass reads those and writes S. cube_bytes: bytes per cube value read (2
    for a 16-bit cube the kernels read as such)."""
    d = 4.0 - cube_bytes
    out = []
    for k, pair in enumerate(kernels):
        code = codes[k]
        name = smoothing_kernel_name(sc, pair, code, sampled)
        if code == sc.SC_KERNEL_SHARED:
            out.append((name, SHARED_BYTES_PER_VOXEL))
        elif (k + 1 < len(kernels) and codes[k + 1] == sc.SC_KERNEL_SHARED and kernels[k + 1][0] == pair[0]
              and code in (sc.SC_KERNEL_WS32, sc.SC_KERNEL_WS16, getattr(sc, "SC_KERNEL_FIR", -1))):
            out.append((name + "+P", STORE_BYTES_PER_VOXEL - d))
        else:
            out.append((name, SMOOTH_BYTES_PER_VOXEL - d))
    return out


def dominant_kernel(sc, kernels, st, voxels_per_launch, steps, peak, peak_kind, sampled=False, cube_bytes=4.0):
    """Roofline object of the smoothing kernel with the largest share of the
    profiled smoothing time (per-pair CUDA events recorded by the library):
    algorithmic bytes of its launches over their event time."""
    groups = {}
    for k, (name, bpv) in enumerate(pair_kernels(sc, kernels, st["smooth_kernel_pair"], sampled, cube_bytes)):
        n_l = st["smooth_launches_pair"][k]
        if n_l == 0:
            continue
        g = groups.setdefault(name, [0.0, 0, 0.0])
        g[0] += st["ms_smooth_pair"][k]
        g[1] += n_l
        g[2] += bpv * voxels_per_launch * n_l
    dom = max(groups, key=lambda name: groups[name][0])
    dom_ms, dom_launches, dom_bytes = groups[dom]
    avg_ms = dom_ms / dom_launches
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    tr = smooth_traffic_record()
    dram = tr["kernels"].get(dom) if tr else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": dram * voxels_per_launch if dram is not None else None,
            "kernel": dom, "launch_ms": avg_ms, "share_of_smoothing": dom_ms / max(1e-9, st["ms_smooth"]),
            "peak_kind": peak_kind, "algorithmic_bytes_per_voxel": dom_bytes / (voxels_per_launch * dom_launches),
            "smoothing_ms_by_kernel": {name: round(v[0] / steps, 3) for name, v in groups.items()}}


def host_e2e(ctx, host_cube, kernels, t, mode, n_repl, nvox, e2e_steps, pg, dev, world, storage=0,
             host_scale=None, flags=0):
    """End to end through the C ABI's host-buffer entry sc_run_host_many: the
    step's cube (pinned host memory) goes host -> device and its mask device ->
    host inside the call, the next cube's copy and the previous mask's copy
    overlapped with the current run by the library; e2e_steps cubes per call
    (the same host cube, two host masks in turn), timed on the host around the
    call, which synchronises. The copy bandwidths are measured afterwards with
    the same pinned buffers."""
    import torch

    shape = tuple(host_cube.shape)
    masks = [torch.empty(shape, dtype=torch.uint8, pin_memory=True) for _ in range(2)]

    def run(k):
        return ctx.run_host_many([host_cube] * k, kernels, t, mode, n_repl, masks_host=[masks[i % 2] for i in range(k)],
                                 storage=storage, chan_scales_host=[host_scale] * k if host_scale is not None else None,
                                 flags=flags)

    run(2)
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    _, sigs, s0s = run(e2e_steps)
    dt = max_over_ranks(time.perf_counter() - t0, pg, dev)
    ok = all(s > 0 for s in s0s) and all(x > 0 for row in sigs for x in row)
    # the copies alone: the pipeline's fill (the first cube) and drain (the
    # last mask) overlap no compute
    d_in = torch.empty(shape, dtype=host_cube.dtype, device=dev)
    d_m = torch.empty(shape, dtype=torch.uint8, device=dev)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    d_in.copy_(host_cube, non_blocking=True)
    e1.record()
    masks[0].copy_(d_m, non_blocking=True)
    e2.record()
    torch.cuda.synchronize(dev)
    h2d_b = host_cube.numel() * host_cube.element_size() + (host_scale.numel() * 4 if host_scale is not None else 0)
    h2d_ms, d2h_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    return {"value": job_value(nvox, len(kernels), e2e_steps, world, dt), "unit": UNIT,
            "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": nvox + 8 * (len(kernels) + 1), "steps": e2e_steps,
            "sigmas_ok": ok, "h2d_gbs": host_cube.numel() * host_cube.element_size() / (h2d_ms * 1e-3) / 1e9,
            "d2h_gbs": nvox / (d2h_ms * 1e-3) / 1e9, "fill_and_drain_ms": h2d_ms + d2h_ms,
            "api": "sc_run_host_many (C ABI, pinned host buffers): every cube host -> device and its mask "
                   "device -> host inside the call, the next cube's copy and the previous mask's overlapped with "
                   "the current run by the library; sigmas returned by the call"}


def measure_batch(dev, local, steps, warmup, pg, world, rank, tune=True, with_e2e=False, e2e_steps=3):
    """The batched form: 64 uneven sub-cubes per rank in one graph-captured
    sc_run_batch call per step (optionally after autotuning every sub-cube
    shape). Timed without profiling events; the roofline comes from one more,
    profiled, batch (events per pair, no graph)."""
    import torch

    from paper_2106_15789_gb300 import Context, sc
    from synth.cubes import KERNELS_12, SC_REPLACEMENT, SC_THRESHOLD, batch_specs, make_cube

    kernels, t, n_repl = KERNELS_12, SC_THRESHOLD, SC_REPLACEMENT
    with torch.no_grad():
        cubes = [make_cube(spec, device=str(dev)) for spec in batch_specs(64, first_seed=64 * rank)]
    masks = [torch.empty(c.shape, dtype=torch.uint8, device=dev) for c in cubes]
    nvox = sum(c.numel() for c in cubes)
    ctx = Context(local, max(c.numel() for c in cubes))
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    if tune:
        for shape in sorted({tuple(c.shape) for c in cubes}):
            ctx.autotune(shape, kernels)
    tune_s = time.perf_counter() - t0

    def step():
        return ctx.run_batch(cubes, kernels, t, "mad", n_repl, masks=masks, flags=sc.SC_FLAG_GRAPH)

    for _ in range(max(2, warmup)):
        step()
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    launches = int(ctx.stats(reset=True)["launches"])
    value = job_value(nvox, len(kernels), steps, world, ms * 1e-3)

    ctx.set_profiling(True)
    ctx.run_batch(cubes, kernels, t, "mad", n_repl, masks=masks)
    torch.cuda.synchronize()
    ctx.set_profiling(False)
    st = ctx.stats(reset=True)
    peak, peak_kind = measured_hbm_peak()
    roofline = dominant_kernel(sc, kernels, st, nvox / len(cubes), 1, peak, peak_kind)
    roofline["measured_in"] = "one profiled batch after the timed region (events per pair, no graph)"

    # the plain path on the same sub-cubes: one sc_run per cube, in sequence
    def plain_all():
        for c, m in zip(cubes, masks):
            ctx.run(c, kernels, t, "mad", n_repl, mask=m)

    plain_all()
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(steps):
        plain_all()
    p1.record(stream)
    torch.cuda.synchronize()
    ms_plain = max_over_ranks(p0.elapsed_time(p1), pg, dev)
    plain_seq = {"value": job_value(nvox, len(kernels), steps, world, ms_plain * 1e-3),
                 "ms_per_step": ms_plain / steps,
                 "what": "the same 64 sub-cubes through sc_run one after the other (plain float32 path, sigmas "
                         "read back per cube)"}

    e2e = None
    if with_e2e:
        # pinned host sub-cubes; two device buffer sets so that the next
        # batch's H2D copies and the previous batch's mask D2H copies run on a
        # copy stream while the current batch computes
        hosts = [torch.empty(c.shape, dtype=torch.float32, pin_memory=True) for c in cubes]
        for h, c in zip(hosts, cubes):
            h.copy_(c)
        mask_h = [[torch.empty(c.shape, dtype=torch.uint8, pin_memory=True) for c in cubes] for _ in range(2)]
        work = [[torch.empty_like(c) for c in cubes] for _ in range(2)]
        wmask = [masks, [torch.empty_like(m) for m in masks]]
        copy = torch.cuda.Stream(dev)
        loaded = [torch.cuda.Event() for _ in range(2)]
        computed = [torch.cuda.Event() for _ in range(2)]
        sent = [torch.cuda.Event() for _ in range(2)]

        def e2e_run(n):
            with torch.cuda.stream(copy):
                for w, h in zip(work[0], hosts):
                    w.copy_(h, non_blocking=True)
                loaded[0].record(copy)
            for i in range(n):
                b, nb = i % 2, (i + 1) % 2
                if i + 1 < n:
                    with torch.cuda.stream(copy):
                        if i >= 1:
                            copy.wait_event(computed[nb])
                        for w, h in zip(work[nb], hosts):
                            w.copy_(h, non_blocking=True)
                        loaded[nb].record(copy)
                stream.wait_event(loaded[b])
                if i >= 2:
                    stream.wait_event(sent[b])
                ctx.run_batch(work[b], kernels, t, "mad", n_repl, masks=wmask[b])  # sigmas: synchronous
                computed[b].record(stream)
                with torch.cuda.stream(copy):
                    copy.wait_event(computed[b])
                    for mh, md in zip(mask_h[b], wmask[b]):
                        mh.copy_(md, non_blocking=True)
                    sent[b].record(copy)
            torch.cuda.synchronize(dev)

        e2e_run(2)
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        e2e_run(e2e_steps)
        dt = max_over_ranks(time.perf_counter() - t0, pg, dev)
        e2e = {"value": job_value(nvox, len(kernels), e2e_steps, world, dt), "unit": UNIT,
               "h2d_bytes_per_step": 4 * nvox, "d2h_bytes_per_step": nvox + 8 * len(cubes) * (len(kernels) + 1),
               "steps": e2e_steps,
               "api": "sc_run_batch on device copies of pinned host sub-cubes (torch copies); next batch's H2D and "
                      "previous masks' D2H overlap the current batch on a copy stream (two buffer sets); sigmas read "
                      "back synchronously"}
    ctx.close()
    del cubes, masks
    torch.cuda.empty_cache()
    peak, _ = measured_hbm_peak()
    return {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "warmup": max(2, warmup),
            "config": {**config_dict("batch64", kernels), "n_cubes": 64, "voxels": nvox, "graph": True,
                       "autotune_s": round(tune_s, 2) if tune else None},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": sampler.summary(),
            "plain_sequential": plain_seq, "frac_of_19B_model": value / world * 19.0 / (peak * 1e9)}


def run_batch_bench(args, rank, world, local):
    """The batched form as a bench line of its own."""
    import torch

    from paper_2106_15789_gb300 import sc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    sc.lib()
    r = measure_batch(dev, local, args.steps, args.warmup, pg, world, rank, tune=True, with_e2e=not args.no_e2e,
                      e2e_steps=args.e2e_steps)
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": r["config"],
                "roofline": r["roofline"], "cpu_baseline": None, "e2e": r["e2e"], "gpu_launches": r["gpu_launches"],
                "clocks": r["clocks"], "frac_of_19B_model": r["frac_of_19B_model"]}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def half_precision(cube, bits, scale, bf16, m_h, sig_h, s0_h, m_f, sig_f, s0_f, with_oracle):
    """Differences of a 16-bit run against float32 on the GPU and, for cubes
    small enough, against the FP64 oracle on the original float32 cube and on
    the decoded 16-bit cube."""
    from synth.cubes import KERNELS_12, SC_REPLACEMENT, SC_THRESHOLD, decode_half

    nvox = cube.numel()
    nd = int((m_h != m_f).sum().item())
    prec = {"format": "bf16" if bf16 else "fp16",
            "sigma_rel_err_vs_float32": max(abs(a - b) / b for a, b in zip(sig_h + [s0_h], sig_f + [s0_f])),
            "mask_disagreement_vs_float32": nd, "mask_disagreement_frac_vs_float32": nd / nvox}
    if with_oracle:
        from oracle.sc_oracle import sc_filter

        kernels, t, n_repl = KERNELS_12, SC_THRESHOLD, SC_REPLACEMENT
        m_o, s_o, s0_o = sc_filter(cube.cpu().numpy(), kernels, t, "mad", n_repl)
        dec = decode_half(bits.cpu().numpy(), scale.cpu().numpy(), bf16)
        m_d, s_d, s0_d = sc_filter(dec, kernels, t, "mad", n_repl)
        mh = m_h.cpu().numpy()
        no = int((mh != m_o).sum())
        prec.update({"sigma_rel_err_vs_oracle_fp64": max(abs(a - b) / b for a, b in zip(sig_h + [s0_h], s_o + [s0_o])),
                     "mask_disagreement_vs_oracle_fp64": no, "mask_disagreement_frac_vs_oracle_fp64": no / nvox,
                     "sigma_rel_err_vs_oracle_on_decoded": max(abs(a - b) / b for a, b in zip(sig_h + [s0_h],
                                                                                               s_d + [s0_d])),
                     "mask_disagreement_vs_oracle_on_decoded": int((mh != m_d).sum())})
    return prec


def measure_half(ctx, cube, bf16, steps, warmup, local, pg, world, dev, ref=None, with_oracle=False, e2e_steps=0):
    """The precision form on one cube: stored in 16 bits with per-channel
    float32 scales, run through sc_run_half; timed without profiling events,
    then one profiled step for the roofline; differences against float32
    (ref = its mask and sigmas, computed here when not given)."""
    import torch

    from paper_2106_15789_gb300 import sc
    from synth.cubes import KERNELS_12, SC_REPLACEMENT, SC_THRESHOLD, encode_half

    kernels, t, n_repl = KERNELS_12, SC_THRESHOLD, SC_REPLACEMENT
    bits, scale = encode_half(cube, bf16)
    nvox = cube.numel()
    mask = torch.empty(cube.shape, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        return ctx.run_half(bits, bf16, scale, kernels, t, "mad", n_repl, mask=mask)

    for _ in range(max(2, warmup)):
        step()
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    if pg:
        pg.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        m_h, sig_h, s0_h = step()
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    launches = int(ctx.stats(reset=True)["launches"])
    value = job_value(nvox, len(kernels), steps, world, ms * 1e-3)
    ctx.set_profiling(True)
    step()
    torch.cuda.synchronize()
    ctx.set_profiling(False)
    st = ctx.stats(reset=True)
    peak, peak_kind = measured_hbm_peak()
    in_kernel = int(st["half_path"]) == 1
    roofline = dominant_kernel(sc, kernels, st, nvox, 1, peak, peak_kind, cube_bytes=2.0 if in_kernel else 4.0)
    roofline["measured_in"] = "one profiled step after the timed region"
    m_h = m_h.clone()
    e2e = None
    if e2e_steps:
        e2e = host_e2e(ctx, bits.cpu().pin_memory(), kernels, t, "mad", n_repl, nvox, e2e_steps, pg, dev, world,
                       storage=sc.SC_STORE_BF16 if bf16 else sc.SC_STORE_FP16, host_scale=scale.cpu().pin_memory())
    if ref is None:
        m_f, sig_f, s0_f = ctx.run(cube, kernels, t, "mad", n_repl)
        ref = (m_f.clone(), sig_f, s0_f)
    prec = half_precision(cube, bits, scale, bf16, m_h, sig_h, s0_h, *ref, with_oracle)
    prec["half_path"] = int(st["half_path"])
    prec["cube_read"] = {1: "16-bit values by every kernel (SC_FLAG_HALF_DIRECT)",
                         2: "decoded into a float32 copy by a pass of its own",
                         3: "16-bit values by the raw-cube histogram pass, which writes the float32 working copy "
                            "every later pass reads"}.get(int(st["half_path"]), "float32")
    if not bf16 and not with_oracle:
        # mitigation study: FP16 plus a float32 sideband of the values above
        # 2.5 sigma_0 (the float32 path on the decoded cube with those values
        # restored), against float32
        from synth.cubes import decode_half

        dec = torch.from_numpy(decode_half(bits.cpu().numpy(), scale.cpu().numpy(), False)).to(dev)
        side = cube.abs() > 2.5 * ref[2]
        patched = torch.where(side, cube, dec)
        del dec
        m_s, _, _ = ctx.run(patched, kernels, t, "mad", n_repl)
        prec["sideband_2p5_sigma0"] = {"sideband_frac": float(side.float().mean().item()),
                                       "mask_disagreement_frac_vs_float32": int((m_s != ref[0]).sum().item()) / nvox}
        del patched, side
    del bits, scale, mask
    return {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "warmup": max(2, warmup),
            "dtype": "bf16" if bf16 else "fp16", "roofline": roofline, "gpu_launches": launches, "e2e": e2e,
            "clocks": sampler.summary(), "precision": prec,
            "breakdown_ms_per_step": {"smooth": st["ms_smooth"] + st["ms_share_prep"], "select": st["ms_select"],
                                      "decode_and_mask": st["ms_clip"]},
            "frac_of_17B_model": value / world * 17.0 / (peak * 1e9)}


def run_half_bench(args, rank, world, local):
    """The precision form as a bench line of its own (small or WALLABY cube)."""
    import torch

    from paper_2106_15789_gb300 import Context, sc
    from synth.cubes import KERNELS_12

    base, fmt = args.workload.split("-")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    sc.lib()
    spec, cube = make_workload(base, rank, str(dev))
    ctx = Context(local, cube.numel())
    if not args.no_autotune:
        ctx.autotune(cube.shape, KERNELS_12)  # as the plain form does, once per cube shape before timing
    r = measure_half(ctx, cube, fmt == "bf16", args.steps, args.warmup, local, pg, world, dev,
                     with_oracle=(base == "small"))
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": fmt, "data": "synthetic",
                "config": {**config_dict(args.workload, KERNELS_12), "storage_bytes_per_voxel": 2},
                "roofline": r["roofline"], "cpu_baseline": None, "e2e": None, "gpu_launches": r["gpu_launches"],
                "clocks": r["clocks"], "precision": r["precision"], "breakdown_ms_per_step": r["breakdown_ms_per_step"]}
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


def run_stream_bench(args, rank, world, local):
    """A stream of 512 sub-cubes (batch size distribution) arriving as a
    Poisson process at 50 cubes/s, admitted by sc_submit under a 120 GB budget
    with the masks kept on the device; once with BF16 storage and once with
    plain float32. Reports the throughput over the makespan and the p50 / p99
    latency (submission to completion) of both."""
    import numpy as np
    import torch

    from paper_2106_15789_gb300 import Context, sc
    from synth.cubes import KERNELS_20, SC_REPLACEMENT, batch_specs, encode_half, make_cube

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc.lib()
    kernels, t, n_repl, n_cubes, rate, budget = KERNELS_20, 4.0, SC_REPLACEMENT, 512, 50.0, 120e9
    specs = batch_specs(n_cubes, first_seed=n_cubes * rank)
    with torch.no_grad():
        cubes = [make_cube(sp, device=str(dev)) for sp in specs]
        halves = [encode_half(c, True) for c in cubes]
    masks = [torch.empty(c.shape, dtype=torch.uint8, device=dev) for c in cubes]
    nvox = sum(c.numel() for c in cubes)
    ctx = Context(local, max(c.numel() for c in cubes))
    ctx.set_budget(int(budget))
    arrivals = np.cumsum(np.random.default_rng(5 + rank).exponential(1.0 / rate, n_cubes))

    def submit(i, storage):
        if storage == sc.SC_STORE_F32:
            return ctx.submit(cubes[i], kernels, t, "mad", n_repl, mask=masks[i])[0]
        bits, scale = halves[i]
        return ctx.submit(bits, kernels, t, "mad", n_repl, mask=masks[i], storage=storage, chan_scale=scale)[0]

    def run(storage):
        lat, waits, i, pending, refused = {}, 0, 0, 0, 0
        t0 = time.perf_counter()
        while i < n_cubes or pending:
            now = time.perf_counter() - t0
            if i < n_cubes and now >= arrivals[i]:
                try:
                    submit(i, storage)
                    i += 1
                    pending += 1
                except sc.ScError as e:
                    if e.code != sc.SC_ERR_BUDGET:
                        raise
                    refused += 1
                    r = ctx.poll(len(kernels), wait=True)
                    lat[r[0]] = r[2]
                    pending -= 1
                continue
            r = ctx.poll(len(kernels), wait=(i >= n_cubes))
            if r is not None:
                assert r[1] == sc.SC_OK, r
                lat[r[0]] = r[2]
                pending -= 1
            elif i < n_cubes:
                time.sleep(min(max(arrivals[i] - now, 0.0), 5e-4))
        makespan = time.perf_counter() - t0
        ls = np.sort(np.array(list(lat.values())))
        return {"value": nvox * len(kernels) / makespan, "makespan_s": makespan,
                "latency_p50_ms": 1e3 * float(np.percentile(ls, 50)), "latency_p99_ms": 1e3 * float(np.percentile(ls, 99)),
                "latency_max_ms": 1e3 * float(ls[-1]), "refused_by_budget": refused}

    # warm-up: a few jobs of each storage (lanes, kernels, first-use allocations)
    for storage in (sc.SC_STORE_BF16, sc.SC_STORE_F32):
        for i in range(4):
            submit(i, storage)
        while ctx.poll(len(kernels), wait=True) is not None:
            pass
    sampler = ClockSampler(local)
    sampler.start()
    res_bf16 = run(sc.SC_STORE_BF16)
    res_f32 = run(sc.SC_STORE_F32)
    sampler.stop()
    if rank == 0:
        line = {"metric": METRIC, "value": res_bf16["value"], "unit": UNIT, "n_gpus": world, "steps": 1,
                "warmup": 1, "ms_per_step": 1e3 * res_bf16["makespan_s"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": "stream-512-subcubes-poisson-50-per-s", "n_cubes": n_cubes, "voxels": nvox,
                           "kernels": "spatial {0,3,6,10} px x spectral {0,3,7,15,31} ch", "n_pairs": len(kernels),
                           "threshold": t, "noise": "mad", "replacement": n_repl, "arrival_rate_per_s": rate,
                           "budget_bytes": budget, "masks": "kept on the device"},
                "stream_bf16": res_bf16, "stream_float32": res_f32, "roofline": None, "cpu_baseline": None,
                "e2e": None, "clocks": sampler.summary(),
                "note": "throughput over the makespan of a Poisson stream: bounded by the offered load when the "
                        "GPU keeps up"}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_noise_scale_bench(args, rank, world, local):
    """Local noise normalisation of the WALLABY-shaped cube: 31 x 31 x 31
    windows (the paper's speed test) on 16 x 16 x 16 cells, MAD noise; one step
    is one sc_noise_scale call (per-cell window noise, then the division)."""
    import numpy as np
    import torch

    from paper_2106_15789_gb300 import Context, sc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    sc.lib()
    window, grid = (31, 31, 31), (16, 16, 16)
    mode = "gauss" if args.workload.endswith("-gauss") else "mad"
    if args.workload == "medium-noisescale":  # a 256^3 cube for profiling
        from synth.cubes import CubeSpec, make_cube

        spec = CubeSpec(nx=256, ny=256, nz=256, seed=12, n_gal=40, ripple=0.3, nan_border=4, name="noise-256")
        with torch.no_grad():
            cube = make_cube(spec, device=str(dev))
    else:
        spec, cube = make_workload("wallaby", rank, str(dev))
    nvox = cube.numel()
    out = torch.empty_like(cube)
    ctx = Context(local, 1)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        ctx.noise_scale(cube, window, grid, mode, out=out)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ctx.stats(reset=True)
    ctx.set_profiling(True)
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.noise_scale(cube, window, grid, mode, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler.stop()
    ctx.set_profiling(False)
    ms = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    st = ctx.stats(reset=True)
    value = nvox * args.steps * world / (ms * 1e-3)
    win_ms, app_ms = st["ms_noise_window"] / args.steps, st["ms_noise_apply"] / args.steps
    # roofline of the division pass (read the cube, write the result: 8 B per
    # voxel); the window pass is bound by its shared-memory selections
    peak, peak_kind = measured_hbm_peak()
    achieved = 8.0 * nvox / (app_ms * 1e-3) / 1e9
    ncells = -(-spec.nx // grid[0]) * -(-spec.ny // grid[1]) * -(-spec.nz // grid[2])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "k_noise_apply", "launch_ms": app_ms, "peak_kind": peak_kind,
                "algorithmic_bytes_per_voxel": 8.0,
                "k_noise_window": {"launch_ms": win_ms, "cells": ncells,
                                   "window_voxels_per_s": ncells * float(np.prod(window)) / (win_ms * 1e-3)}}
    # end to end: pinned host cube in, normalised cube out, every step
    cube_h = torch.empty(cube.shape, dtype=torch.float32, pin_memory=True)
    cube_h.copy_(cube)
    out_h = torch.empty(cube.shape, dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_e2e = max(1, min(args.steps, 3))
    for _ in range(n_e2e):
        cube.copy_(cube_h, non_blocking=True)
        ctx.noise_scale(cube, window, grid, mode, out=out)
        out_h.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": nvox * n_e2e * world / e2e_s, "unit": "voxels/s", "h2d_bytes_per_step": 4 * nvox,
           "d2h_bytes_per_step": 4 * nvox, "steps": n_e2e, "api": "sc_noise_scale on a device copy of a pinned host "
           "cube, result copied back to pinned host memory"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle.noise_scale as NS

        sub = cube[:128, :1024, :1024].cpu().numpy()  # (the whole cube when it is smaller)
        t0 = time.perf_counter()
        NS.noise_scale(sub, window, grid, mode)
        dt = time.perf_counter() - t0
        cpu = {"value": sub.size / dt, "unit": "voxels/s", "cores": 1, "kind": "oracle",
               "sample": f"1024x1024x128 corner of the same cube, same windows and cells, numpy float64, one thread, "
                         f"{dt:.1f} s"}
    if rank == 0:
        line = {"metric": NOISE_SCALE_METRIC, "value": value, "unit": "voxels/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"noise-scale-{spec.nx}x{spec.ny}x{spec.nz}", "window": list(window),
                           "cells": list(grid), "noise": mode,
                           "l2": "inputs larger than L2" if nvox * 4 > 129e6 else "no flush"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(st["launches"]),
                "clocks": sampler.summary(),
                "breakdown_ms_per_step": {"noise_window": win_ms, "noise_apply": app_ms}}
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


def run_autoflag_bench(args, rank, world, local):
    """The auto-flagger on the WALLABY-shaped cube: channel and pixel noises
    (MAD), their median and MAD-based RMS, flags beyond 4 RMS, blanking; one
    step is one sc_autoflag call."""
    import torch

    from paper_2106_15789_gb300 import Context, sc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    sc.lib()
    spec, cube = make_workload("wallaby", rank, str(dev))
    mode = "gauss" if args.workload.endswith("-gauss") else "mad"
    nvox = cube.numel()
    out = torch.empty_like(cube)
    ctx = Context(local, 1)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        _, fc, fp, _, _ = ctx.autoflag(cube, 4.0, noise_mode=mode, out=out)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    ctx.stats(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, fc, fp, _, _ = ctx.autoflag(cube, 4.0, noise_mode=mode, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler.stop()
    st = ctx.stats(reset=True)
    ms = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    value = nvox * args.steps * world / (ms * 1e-3)
    peak, peak_kind = measured_hbm_peak()
    # algorithmic bytes: the cube read once for the channel noises, once for
    # the pixel noises and once for the blanking, the result written: 16 B
    achieved = 16.0 * nvox / (ms / args.steps * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "sc_autoflag (all kernels of a call)", "launch_ms": ms / args.steps,
                "peak_kind": peak_kind, "algorithmic_bytes_per_voxel": 16.0}
    cube_h = torch.empty(cube.shape, dtype=torch.float32, pin_memory=True)
    cube_h.copy_(cube)
    out_h = torch.empty(cube.shape, dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    n_e2e = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        cube.copy_(cube_h, non_blocking=True)
        ctx.autoflag(cube, 4.0, noise_mode=mode, out=out)
        out_h.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": nvox * n_e2e * world / e2e_s, "unit": "voxels/s", "h2d_bytes_per_step": 4 * nvox,
           "d2h_bytes_per_step": 4 * nvox, "steps": n_e2e,
           "api": "sc_autoflag on a device copy of a pinned host cube, blanked cube copied back"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle.flagger as FL

        side = 256 if mode == "mad" else 96  # about 10-30 s of oracle work either way
        sub = cube[:, :side, :side].cpu().numpy()
        t0 = time.perf_counter()
        FL.autoflag(sub, 4.0, mode=mode)
        dt = time.perf_counter() - t0
        cpu = {"value": sub.size / dt, "unit": "voxels/s", "cores": 1, "kind": "oracle",
               "sample": f"{side}x{side}x{sub.shape[0]} corner of the same cube, k = 4, numpy float64, one thread, "
                         f"{dt:.1f} s"}
    if rank == 0:
        line = {"metric": FLAG_METRIC, "value": value, "unit": "voxels/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "autoflag-wallaby-1200x1200x1024", "k": 4.0, "noise": mode,
                           "flagged_channels": int(fc.sum()), "flagged_pixels": int(fp.sum()),
                           "l2": "inputs (cube 5.9 GB) larger than L2"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(st["launches"]),
                "clocks": sampler.summary()}
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


def run_link_bench(args, rank, world, local):
    """The linker on the S+C mask of the WALLABY-shaped cube with the paper's
    settings (merging radius 2 pixels / channels, minimum size 8 pixels and 5
    channels); one step is one sc_link call."""
    import torch

    from paper_2106_15789_gb300 import Context, sc
    from synth.cubes import KERNELS_12, SC_REPLACEMENT, SC_THRESHOLD

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    sc.lib()
    spec, cube = make_workload("wallaby", rank, str(dev))
    nvox = cube.numel()
    ctx = Context(local, nvox)
    mask, _, _ = ctx.run(cube, KERNELS_12, SC_THRESHOLD, "mad", SC_REPLACEMENT)
    del cube
    labels = torch.empty(mask.shape, dtype=torch.int32, device=dev)
    params = dict(r_xy=2, r_z=2, min_xy=8, min_z=5)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        _, n_det, _ = ctx.link(mask, labels=labels, extents_cap=0, **params)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.stats(reset=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, n_det, _ = ctx.link(mask, labels=labels, extents_cap=0, **params)
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler.stop()
    st = ctx.stats(reset=True)
    ms = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    value = nvox * args.steps * world / (ms * 1e-3)
    peak, peak_kind = measured_hbm_peak()
    # algorithmic bytes: read the mask (1 B) and write the labels (4 B) per voxel
    achieved = 5.0 * nvox / (ms / args.steps * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "sc_link (all 13 kernels of a call)", "launch_ms": ms / args.steps,
                "peak_kind": peak_kind, "algorithmic_bytes_per_voxel": 5.0}
    # end to end: the mask from pinned host memory, the labels back to it
    mask_h = torch.empty(mask.shape, dtype=torch.uint8, pin_memory=True)
    mask_h.copy_(mask)
    lab_h = torch.empty(mask.shape, dtype=torch.int32, pin_memory=True)
    torch.cuda.synchronize()
    n_e2e = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        mask.copy_(mask_h, non_blocking=True)
        ctx.link(mask, labels=labels, extents_cap=0, **params)
        lab_h.copy_(labels, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": nvox * n_e2e * world / e2e_s, "unit": "voxels/s", "h2d_bytes_per_step": nvox,
           "d2h_bytes_per_step": 4 * nvox, "steps": n_e2e,
           "api": "sc_link on a device copy of a pinned host mask, labels copied back to pinned host memory"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle.linker as LK

        sub = mask[:256, :512, :512].cpu().numpy()
        t0 = time.perf_counter()
        LK.link(sub, **params)
        dt = time.perf_counter() - t0
        cpu = {"value": sub.size / dt, "unit": "voxels/s", "cores": 1, "kind": "oracle",
               "sample": f"512x512x256 corner of the same mask, same settings, numpy / scipy connected components, "
                         f"one thread, {dt:.1f} s"}
    if rank == 0:
        line = {"metric": LINK_METRIC, "value": value, "unit": "voxels/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": "link-wallaby-1200x1200x1024-sc-mask", **params,
                           "mask_fraction": float(mask.float().mean().item()), "detections": n_det,
                           "l2": "inputs (mask 1.5 GB, labels 5.9 GB) larger than L2"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(st["launches"]),
                "clocks": sampler.summary()}
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=WORKLOADS, default="wallaby")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-cube", choices=("wallaby", "small"), default="wallaby",
                    help="cube whose interior sub-cubes the reference arm times (small: a quick check)")
    ap.add_argument("--no-forms", action="store_true", help="default workload: skip the batched and 16-bit forms")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (predictable launch order for profiling captures)")
    ap.add_argument("--record-traffic", metavar="KEY=NCU_CSV", nargs="+",
                    help="write profiles/smooth_traffic.json from one-kernel ncu --csv DRAM captures of the medium "
                         "workload and exit (no GPU)")
    ap.add_argument("--traffic-command", default="", help="the command that made NCU_CSV (stored in the record)")
    args = ap.parse_args()
    if args.record_traffic:
        return record_traffic(args.record_traffic, args.traffic_command)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch64":
        return run_batch_bench(args, rank, world, local)
    if args.workload.endswith(("-bf16", "-fp16")):
        return run_half_bench(args, rank, world, local)
    if args.workload == "stream512":
        return run_stream_bench(args, rank, world, local)
    if args.workload.endswith(("-noisescale", "-noisescale-gauss")):
        return run_noise_scale_bench(args, rank, world, local)
    if args.workload == "wallaby-link":
        return run_link_bench(args, rank, world, local)
    if args.workload in ("wallaby-autoflag", "wallaby-autoflag-gauss"):
        return run_autoflag_bench(args, rank, world, local)

    import torch

    from paper_2106_15789_gb300 import Context, sc
    from synth.cubes import KERNELS_12, SC_REPLACEMENT, SC_THRESHOLD

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    sc.lib()  # fails loudly when the CUDA library is missing
    kernels = KERNELS_12
    t, n_repl = SC_THRESHOLD, SC_REPLACEMENT
    mode = "gauss" if args.workload.endswith("-gauss") else "mad"
    sampled = args.workload.endswith("-sampled")
    run_flags = sc.SC_FLAG_SAMPLED_GAUSS if sampled else 0
    spatial = "sampled" if sampled else "cascade"
    spec, cube = make_workload(args.workload.removesuffix("-gauss").removesuffix("-sampled"), rank, str(dev))
    nvox = cube.numel()
    mask = torch.empty(cube.shape, dtype=torch.uint8, device=dev)
    ctx = Context(local, nvox)
    stream = torch.cuda.current_stream(dev)
    t_tune = time.perf_counter()
    if not args.no_autotune:
        ctx.autotune(cube.shape, kernels)  # once per cube shape, before timing (as a user would)
    tune_s = time.perf_counter() - t_tune

    def step():
        return ctx.run(cube, kernels, t, mode, n_repl, mask=mask, flags=run_flags)

    for _ in range(max(args.warmup, 3 if args.warmup >= 3 else args.warmup)):
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()

    def timed(profiled):
        """K steps between CUDA events on the launching stream (barrier and
        synchronisation on both sides); returns ms and the library's stats."""
        ctx.stats(reset=True)
        ctx.set_profiling(profiled)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            out = step()
        e1.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        ctx.set_profiling(False)
        return max_over_ranks(e0.elapsed_time(e1), pg, dev), ctx.stats(reset=True), out

    sampler = ClockSampler(local)
    sampler.start()
    ms, st_plain, (_, sig, sig0) = timed(False)  # the headline: no profiling events
    sampler.stop()
    # the same steps again with the library's per-phase CUDA events, for the
    # per-kernel times of the roofline and the breakdown
    ms_prof, st, _ = timed(True)
    value = job_value(nvox, len(kernels), args.steps, world, ms * 1e-3)

    # roofline of the dominant kernel: the smoothing kernel with the largest
    # share of device time (live events, grouped by the kernel each pair runs)
    peak, peak_kind = measured_hbm_peak()
    roofline = dominant_kernel(sc, kernels, st, nvox, args.steps, peak, peak_kind, sampled)
    roofline["measured_in"] = "the profiled repeat of the timed steps (per-pair CUDA events on the launching stream)"
    mask_f32 = mask.clone() if not args.no_forms and world == 1 and mode == "mad" and not sampled else None

    e2e = None
    if not args.no_e2e:
        e2e = host_e2e(ctx, cube.cpu().pin_memory(), kernels, t, mode, n_repl, nvox, args.e2e_steps, pg, dev, world,
                       flags=run_flags)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cube, kernels, t, n_repl, mode, spatial)

    forms = None
    if mask_f32 is not None:
        # the metric's second half: the 16-bit forms of the same cube on the same
        # context, the 16-bit forms of the small cube against the FP64 oracle,
        # and the batched form, each timed like the headline (fewer steps)
        from synth.cubes import SMALL, make_cube

        fs = max(2, min(args.steps, 3))
        forms = {}
        for fmt in ("fp16", "bf16"):
            forms["wallaby-" + fmt] = measure_half(ctx, cube, fmt == "bf16", fs, 2, local, pg, world, dev,
                                                   ref=(mask_f32, sig, sig0), e2e_steps=0 if args.no_e2e else args.e2e_steps)
        with torch.no_grad():
            small = make_cube(SMALL, device=str(dev))
        sctx = Context(local, small.numel())
        for fmt in ("fp16", "bf16"):
            r = measure_half(sctx, small, fmt == "bf16", 3, 2, local, pg, world, dev, with_oracle=True)
            forms["small-" + fmt] = {"precision": r["precision"], "value": r["value"], "unit": UNIT}
        sctx.close()
        ctx.close()
        ctx = None
        del cube, mask_f32
        torch.cuda.empty_cache()
        forms["batch64"] = measure_batch(dev, local, fs, 2, pg, world, rank, tune=False)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {**config_dict(args.workload, kernels, mode), "autotune_s": round(tune_s, 2)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(st_plain["launches"]), "clocks": sampler.summary(),
                "profiled_ms_per_step": ms_prof / args.steps,
                "breakdown_ms_per_step": {"smooth": st["ms_smooth"] / args.steps,
                                          "share_prep": st["ms_share_prep"] / args.steps,
                                          "select": st["ms_select"] / args.steps,
                                          "clip": st["ms_clip"] / args.steps,
                                          **({"gauss_hist": st["ms_gauss_hist"] / args.steps,
                                              "gauss_fit": st["ms_gauss_fit"] / args.steps} if mode == "gauss"
                                             else {})},
                **({"roofline_gauss_hist": gauss_hist_roofline(st, peak, peak_kind)} if mode == "gauss" else {}),
                "sigma0": sig0, "sigmas": sig, "mask_fraction": float(mask.float().mean().item()),
                "frac_of_19B_model": value / world * 19.0 / (peak * 1e9),
                **({"forms": forms} if forms else {})}
        print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
