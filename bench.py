#!/usr/bin/env python
"""Benchmark of radiomic spatial mapping on GB300.

A step maps one whole synthetic volume: discretisation, VOI packing and the
mapping kernel (all 93 maps of every VOI voxel).  Default workload: the
largest single-GPU configuration, the CT-like 256 x 256 x 128 volume with a
VOI of three ellipsoids (2,014,083 voxels), fixed bin count 64, kernel radius
3 (7^3 windows), GLCM distance 1; the 128 x 128 x 64 CT-like volume (200,336
voxels, FBW 25 HU, r = 2) is timed as an extra leg.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl flashmap|reference]

Prints one JSON line (rank 0).  `value` is voxel-features/s over the K timed
steps measured with CUDA events on the launching stream (inputs resident in
HBM; L2 flushed between steps); `e2e` is the same metric through
fr_map_run_host (pinned host image in, host maps out, copies inside the timed
region).  Under torchrun every rank maps its own replica (weak scaling, no
collective on the data path); the timed region is bracketed by barriers and
the slowest rank's time is reported.  `--impl reference` times the FP64 CPU
oracle on the host cores on bounded samples of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-features/s for 3D texture maps, batched vs plain; serving p50/p99 latency"
UNIT = "voxel-features/s"
ALU_LANES_PER_SM = 128  # fp32/int32 lanes per Blackwell SM

# Counters of fr_map_kernel from ncu captures, keyed by workload and the
# SHA-256 of the CUDA sources they were taken with (a source change makes
# them stale and the bench reports null): DRAM bytes (read + write) per
# launch, issue-slot utilisation and shared-memory pipe utilisation (% of
# peak), as summarised under profiles/.
NCU_COUNTERS = {
    # profiles/: 477 B of DRAM traffic per VOI voxel on the 492,804-voxel band
    # of the same volume (24.8 MB read + 210.4 MB written), scaled by voxels
    # to the 2,014,083-voxel launch; issue slots and shared-memory pipe from
    # the band's full capture
    ("ct_large", "47d36ccb30ad34b976d0ebd50daadb834c44c01cd803c4f86cdde167701ab4d3"):
        {"traffic": 961114699, "traffic_basis": "band of 492,804 voxels, scaled by voxels",
         "issue_active_pct": 50.6, "shared_pipe_pct": 16.6},
    ("ct_large_slab16", "47d36ccb30ad34b976d0ebd50daadb834c44c01cd803c4f86cdde167701ab4d3"):
        {"traffic": 235164672, "issue_active_pct": 50.6, "shared_pipe_pct": 16.6},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="flashmap", choices=["flashmap", "reference"])
    ap.add_argument("--workload", default="ct_large",
                    choices=["ct_plain", "tiny", "ct_large", "ct_large_slab16", "paper_tiled"])
    ap.add_argument("--extra-workloads", default="ct_plain",
                    help="comma-separated workloads timed as extra legs (kernel only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-single-seconds", type=float, default=10.0)
    ap.add_argument("--tune", default="", help="brick_x,brick_y,brick_z,vpi,warps,stages")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-scalar", action="store_true")
    ap.add_argument("--no-drain", action="store_true")
    ap.add_argument("--batch-vois", type=int, default=64)
    ap.add_argument("--small-vois", type=int, default=256)
    ap.add_argument("--served-requests", type=int, default=2000)
    ap.add_argument("--served-rates", default="5,10,20,50,100,200,400,1000")
    ap.add_argument("--served-seconds", type=float, default=12.0,
                    help="time limit per served rate")
    return ap.parse_args()


def workload(name):
    from paper_2609_19190_gb300 import synth
    if name == "ct_plain":
        img, mask = synth.ct_plain(seed=2)
        kw = dict(disc_mode=1, bin_width=25.0, kernel_radius=2, glcm_distance=1)
        desc = ("CT-like 128x128x64 int16 (tissue means -900/-50/40/300 HU, noise sd 15), "
                "ellipsoidal VOI, FBW 25 HU, r=2 (5^3), delta=1, 93 maps")
    elif name == "tiny":
        img, mask = synth.tiny(seed=1)
        kw = dict(disc_mode=0, bin_count=16, kernel_radius=1, glcm_distance=1)
        desc = "32^3 uniform 0..255, ball VOI r=10, FBN 16, r=1, 93 maps"
    elif name == "ct_large":
        img, mask = synth.ct_large(seed=3)
        kw = dict(disc_mode=0, bin_count=64, kernel_radius=3, glcm_distance=1)
        desc = ("CT-like 256x256x128 int16, union of 3 ellipsoids, FBN 64, r=3 (7^3), "
                "delta=1, 93 maps")
    elif name == "ct_large_slab16":
        # the same volume, the VOI voxels of slices 56..71 only (492,804
        # voxels): a capture-sized case of the same kernel paths for ncu
        img, mask = synth.ct_large(seed=3)
        mask = mask.copy()
        mask[:56] = 0
        mask[72:] = 0
        kw = dict(disc_mode=0, bin_count=64, kernel_radius=3, glcm_distance=1)
        desc = ("CT-like 256x256x128 int16, the union-of-3-ellipsoids VOI cut to slices "
                "56..71, FBN 64, r=3 (7^3), delta=1, 93 maps")
    else:
        img, mask = synth.paper_tiled(reps=(2, 2, 2))
        kw = dict(disc_mode=1, bin_width=25.0, kernel_radius=1, glcm_distance=1)
        desc = "61x55x39 MR-like crop tiled 2x2x2 (404,904 VOI voxels), FBW 25, r=1, 93 maps"
    return img, mask, kw, desc


# ------------------------------------------------------------------ roofline work
def _box_sum(csum, lo, hi):
    """Sum over boxes [z+lo0, z+hi0] x ... of the array whose inclusive
    cumulative sum (padded by one leading zero plane per axis) is csum;
    returns an array over the original grid (clipped at the borders)."""
    Z, Y, X = (d - 1 for d in csum.shape)
    zz = np.arange(Z)[:, None, None]
    yy = np.arange(Y)[None, :, None]
    xx = np.arange(X)[None, None, :]
    z0 = np.clip(zz + lo[0], 0, Z); z1 = np.clip(zz + hi[0] + 1, 0, Z)
    y0 = np.clip(yy + lo[1], 0, Y); y1 = np.clip(yy + hi[1] + 1, 0, Y)
    x0 = np.clip(xx + lo[2], 0, X); x1 = np.clip(xx + hi[2] + 1, 0, X)
    S = csum
    return (S[z1, y1, x1] - S[z0, y1, x1] - S[z1, y0, x1] - S[z1, y1, x0]
            + S[z0, y0, x1] + S[z0, y1, x0] + S[z1, y0, x0] - S[z0, y0, x0])


def _csum(a):
    c = np.zeros(tuple(d + 1 for d in a.shape), dtype=np.int64)
    c[1:, 1:, 1:] = a.astype(np.int64).cumsum(0).cumsum(1).cumsum(2)
    return c


def algorithmic_ops(mask, r, delta):
    """Algorithmic work of one launch, in elementary window operations summed
    over all VOI voxels v (N_v = |V(v)|):
      GLCM symmetric increments 2 sum_d |{u : u, u + delta d in V(v)}|,
      GLRLM run-scan steps 13 N_v, GLSZM forward-union attempts 13 N_v,
      GLDM and NGTDM neighbour visits 26 N_v each, first-order sort
      N_v log2 N_v."""
    m = (mask > 0)
    cm = _csum(m)
    nv = _box_sum(cm, (-r, -r, -r), (r, r, r))[m].astype(np.float64)
    pairs = np.zeros_like(nv)
    Z, Y, X = m.shape
    dirs = [d for d in [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
            if d > (0, 0, 0)]
    for d in dirs:
        o = tuple(delta * k for k in d)
        # M_o(u) = mask(u) mask(u + o), for u with u + o inside the volume
        mo = np.zeros_like(m)
        src, dst = [], []
        for k, n in zip(o, m.shape):
            src.append(slice(0, max(0, n - k)) if k >= 0 else slice(-k, n))
            dst.append(slice(k, n) if k >= 0 else slice(0, max(0, n + k)))
        mo[tuple(src)] = m[tuple(src)] & m[tuple(dst)]
        lo = tuple(-r + max(0, -k) for k in o)
        hi = tuple(r - max(0, k) for k in o)
        pairs += _box_sum(_csum(mo), lo, hi)[m]
    sort = nv * np.log2(np.maximum(nv, 1.0))
    return float(np.sum(2.0 * pairs + 78.0 * nv + sort))


def source_digest():
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2609_19190_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of the SM clock and throttle reasons
    while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ distributed
def dist_setup(n):
    rank, world, local = 0, 1, 0
    if "WORLD_SIZE" in os.environ and int(os.environ["WORLD_SIZE"]) > 1:
        import torch
        import torch.distributed as dist
        rank = int(os.environ["RANK"])
        world = int(os.environ["WORLD_SIZE"])
        local = int(os.environ.get("LOCAL_RANK", rank))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    from paper_2609_19190_gb300 import dist as D
    import torch
    return D.max_over_ranks(v, device=torch.device("cuda", torch.cuda.current_device()))


# ------------------------------------------------------------------ batched / served
def _plain_ms(params, masks, images, outs, dev, steps):
    """Device time (CUDA events) of mapping the VOIs one plan at a time."""
    import torch
    import paper_2609_19190_gb300 as fm
    stream = torch.cuda.current_stream(dev)
    plans = [fm.fr_map_plan(p, m) for p, m in zip(params, masks)]
    for pl, im, o in zip(plans, images, outs):
        fm.fr_map_run(pl, im, o)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        e0.record(stream)
        for pl, im, o in zip(plans, images, outs):
            fm.fr_map_run(pl, im, o)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    for pl in plans:
        fm.fr_map_sync_status(pl)
        fm.fr_map_destroy(pl)
    return statistics.median(ms)


def measure_batched(kind, n_vois, dev, steps=3):
    """Many VOIs, plain against batched.  kind "mixed": 64 CT-like
    128x128x64 VOIs (log-uniform 4k-400k voxels); kind "small": 256 VOIs of
    4k-20k voxels in 64^3 CT-like volumes; r in {1,2,3}, FBN 16/32/64, 93
    maps.  Plain maps them one plan at a time (5 kernels each: reset,
    intensity range, discretise/pack, voxel order, map); batched maps all of
    them in one persistent launch (the same 5 kernels once, captured in a
    CUDA graph)
    with the autotuner's launch shape.  Device time with CUDA events."""
    import torch
    import paper_2609_19190_gb300 as fm
    from paper_2609_19190_gb300 import autotune, synth
    item = synth.batch_item if kind == "mixed" else synth.batch_small_item
    params, masks, images = [], [], []
    for i in range(n_vois):
        img, mask, r, bins = item(i)
        nz, ny, nx = img.shape
        params.append(fm.fr_map_params_init(nx, ny, nz, disc_mode=0, bin_count=bins,
                                            kernel_radius=r, device=dev.index or 0))
        masks.append(torch.from_numpy(mask))
        images.append(torch.from_numpy(img).to(dev))
    voxels = int(sum(int(m.sum()) for m in masks))
    tune, timings = autotune.pick(params, masks, images)
    stream = torch.cuda.current_stream(dev)
    outs = [torch.empty((93, int(m.sum())), dtype=torch.float32, device=dev) for m in masks]
    tp = _plain_ms(params, masks, images, outs, dev, steps)
    b = fm.fr_batch_plan(params, masks, tune=tune)
    fm.fr_batch_run(b, images, outs)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batch_ms = []
    for _ in range(steps):
        e0.record(stream)
        fm.fr_batch_run(b, images, outs)
        e1.record(stream)
        e1.synchronize()
        batch_ms.append(e0.elapsed_time(e1))
    fm.fr_batch_sync_status(b)
    fm.fr_batch_destroy(b)
    tb = statistics.median(batch_ms)
    desc = ("%d CT-like 128x128x64 VOIs, log-uniform 4k-400k voxels" % n_vois if kind == "mixed"
            else "%d VOIs of log-uniform 4k-20k voxels in 64^3 CT-like volumes" % n_vois)
    return {"value": voxels * 93 / (tb / 1e3), "unit": UNIT, "plain_value": voxels * 93 / (tp / 1e3),
            "vs_plain": tp / tb, "ms_batched": tb, "ms_plain": tp, "n_vois": n_vois,
            "voxels": voxels, "tune": tune, "tune_timings_ms": timings,
            "kernels": {"batched": 5, "plain": 5 * n_vois},
            "workload": desc + ", r in {1,2,3}, FBN 16/32/64, 93 maps; batched = one persistent "
                               "launch in a CUDA graph"}


def measure_served(n_requests, rates, dev, time_limit):
    """Poisson request stream (log-normal sizes, median 50k voxels, drawn
    in turn from 256 request templates), CT-like volumes resident on the
    device, admission by free HBM, continuous batching through fr_server_*;
    throughput and latency percentiles per rate, each rate until n_requests
    have finished or time_limit seconds have passed.  plain_value: the same
    templates mapped one plan at a time (device time)."""
    import torch
    import paper_2609_19190_gb300 as fm
    from paper_2609_19190_gb300 import serve, synth
    reqs = synth.served_requests(n_requests, seed=200, templates=256)
    images = {sh: torch.from_numpy(synth.ct_like(sh, 500 + k)).to(dev)
              for k, sh in enumerate(synth.SERVED_SHAPES)}
    base = reqs[:256]
    params = []
    for rq in base:
        nz, ny, nx = rq["shape"]
        params.append(fm.fr_map_params_init(nx, ny, nz, kernel_radius=rq["radius"],
                                            device=dev.index or 0, **rq["disc"]))
    outs = [torch.empty((93, rq["n_voi"]), dtype=torch.float32, device=dev) for rq in base]
    tp = _plain_ms(params, [torch.from_numpy(rq["mask"]) for rq in base],
                   [images[rq["shape"]] for rq in base], outs, dev, 1)
    del outs
    plain = sum(rq["n_voi"] for rq in base) * 93 / (tp / 1e3)
    serve.serve(reqs[:16], images, rate=0.0, seed=0, device=dev.index or 0)  # warm-up
    out = []
    for rate in rates:
        st = serve.serve(reqs, images, rate=rate, seed=3, voxel_budget=131072,
                         device=dev.index or 0, time_limit=time_limit)
        out.append({"rate": rate, "throughput": st["throughput"],
                    "vs_plain": st["throughput"] / plain, "p50_s": st["p50_s"],
                    "p99_s": st["p99_s"], "requests": st["requests"],
                    "makespan_s": st["makespan_s"], "steps": st["steps"]})
    return {"unit": UNIT, "plain_value": plain, "requests_per_rate": n_requests,
            "time_limit_s": time_limit, "rates": out,
            "workload": "Poisson arrivals; CT-like VOIs of log-normal size (median 50k voxels, "
                        "sigma_ln 1, <= 2M; 256 templates drawn in turn), r in {1,2,3}, FBN 64 "
                        "or FBW 25, 93 maps; continuous batching, 131072-voxel steps, "
                        "admission by free HBM"}


# ------------------------------------------------------------------ CPU oracle
def oracle_rate(img, mask, kw, seconds, seed=11, threads=None):
    """Time the oracle (as it stands) on `threads` host cores (all by
    default) on a seeded sample of the workload's VOI voxels sized to take
    about `seconds`."""
    from oracle import oracle as O
    from paper_2609_19190_gb300 import synth
    op = O.make_params(img.shape, disc_mode=kw["disc_mode"], bin_count=kw.get("bin_count", 16),
                       bin_width=kw.get("bin_width", 25.0), radius=kw["kernel_radius"],
                       distance=kw["glcm_distance"])
    levels, ng, _, _ = O.discretise(op, img, mask)
    cores = threads or os.cpu_count() or 1
    probe = synth.sample_voxels(mask, min(64 * cores, int(mask.sum())), seed)
    t0 = time.perf_counter()
    O.map_voxels(op, img, levels, ng, probe, nthreads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    n = int(min(mask.sum(), max(probe.size, probe.size * seconds / dt)))
    sample = synth.sample_voxels(mask, n, seed + 1)
    t0 = time.perf_counter()
    O.map_voxels(op, img, levels, ng, sample, nthreads=cores)
    dt = time.perf_counter() - t0
    return n * 93 / dt, cores, n, dt, (op, levels, ng)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2609_19190_gb300 import synth
    img, mask, kw, desc = workload(args.workload)
    op = O.make_params(img.shape, disc_mode=kw["disc_mode"], bin_count=kw.get("bin_count", 16),
                       bin_width=kw.get("bin_width", 25.0), radius=kw["kernel_radius"],
                       distance=kw["glcm_distance"])
    levels, ng, _, _ = O.discretise(op, img, mask)
    cores = os.cpu_count() or 1
    budget = 150.0 / max(1, args.steps + args.warmup)  # seconds per step
    probe = synth.sample_voxels(mask, 128 * cores, 5)
    t0 = time.perf_counter()
    O.map_voxels(op, img, levels, ng, probe, nthreads=cores)
    per_vox = (time.perf_counter() - t0) / probe.size
    n = int(max(cores, min(mask.sum(), budget / max(per_vox, 1e-9))))
    times = []
    for k in range(args.warmup + args.steps):
        sample = synth.sample_voxels(mask, n, 1000 + k)
        t0 = time.perf_counter()
        O.map_voxels(op, img, levels, ng, sample, nthreads=cores)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times)
    value = args.steps * n * 93 / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "n_voi": int(mask.sum()),
                   "sample_voxels_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d seeded VOI voxels per step (of %d), all 93 maps"
                                   % (n, int(mask.sum()))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def measure_scalar(img, mask, kw, dev, steps):
    """Scalar extraction (the features of the whole VOI) of the same volume:
    device time per extraction, CUDA events, L2 flushed between runs."""
    import torch

    import paper_2609_19190_gb300 as fm
    nz, ny, nx = img.shape
    p = fm.fr_map_params_init(nx, ny, nz, **{k: v for k, v in kw.items()
                                             if k not in ("kernel_radius",)})
    sp = fm.fr_scalar_plan(p, torch.from_numpy(mask))
    img_dev = torch.from_numpy(img).to(dev)
    out = torch.empty((sp.n_features,), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        fm.fr_scalar_run(sp, img_dev, out)
    fm.fr_scalar_sync_status(sp)
    ms = []
    for _ in range(max(steps, 5)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fm.fr_scalar_run(sp, img_dev, out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    fm.fr_scalar_sync_status(sp)
    med = statistics.median(ms)
    return {"ms_per_extraction": med, "voi_voxels_per_s": sp.n_voi / (med / 1e3),
            "features": sp.n_features, "n_voi": sp.n_voi,
            "launches_per_extraction": 13,
            "note": "whole-VOI scalar features of the same volume (window = VOI), FP64 "
                    "features from exact counts"}


def measure_plain(name, dev, steps, warmup):
    """An extra plain workload: device time per step (discretisation, packing
    and mapping kernel; CUDA events, L2 flushed between steps), the mapping
    kernel's own time and its window-op rate."""
    import torch

    import paper_2609_19190_gb300 as fm
    img, mask, kw, desc = workload(name)
    nz, ny, nx = img.shape
    params = fm.fr_map_params_init(nx, ny, nz, device=dev.index or 0, **kw)
    plan = fm.fr_map_plan(params, torch.from_numpy(mask))
    img_dev = torch.from_numpy(img).to(dev)
    out = torch.empty((plan.n_rows, plan.n_voi), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(warmup, 1)):
        fm.fr_map_run(plan, img_dev, out)
    fm.fr_map_sync_status(plan)
    step_ms, kern_ms = [], []
    for _ in range(max(steps, 3)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fm.fr_map_run(plan, img_dev, out)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(fm.fr_plan_last_kernel_ms(plan))
    fm.fr_map_sync_status(plan)
    ops = algorithmic_ops(mask, kw["kernel_radius"], kw["glcm_distance"])
    t = sum(step_ms) / len(step_ms) / 1e3
    kmean = statistics.mean(kern_ms) / 1e3
    res = {"workload": desc, "n_voi": plan.n_voi, "maps": plan.n_rows,
           "value": plan.n_voi * plan.n_rows / t, "unit": UNIT, "ms_per_step": 1e3 * t,
           "kernel_ms": 1e3 * kmean, "ops_per_launch": ops, "achieved_gops": ops / kmean / 1e9}
    fm.fr_map_destroy(plan)
    return res


def measure_drain(plan, params, out, img, mask):
    """Host-side HDF5 drain of the finished maps (fr_h5_write_maps): dense
    [nz][ny][nx] float32 maps with NaN outside the VOI, image, mask, geometry
    and settings, chunks encoded on all host threads; wall time per file."""
    import shutil
    import tempfile

    import paper_2609_19190_gb300 as fm
    maps = out.cpu().numpy()
    vox = fm.fr_plan_voxel_index(plan).cpu().numpy()
    tmp = tempfile.mkdtemp(prefix="fr_drain_")
    res = {"threads": os.cpu_count(), "raw_dense_mb": maps.shape[0] * img.size * 4 / 1e6}
    try:
        for codec in ("gzip", "lzf"):
            path = os.path.join(tmp, "maps_%s.h5" % codec)
            ts = []
            for _ in range(2):
                t0 = time.perf_counter()
                fm.fr_h5_write_maps(path, params, img, mask, maps, vox, codec=codec, level=1,
                                    source_id="bench volume")
                ts.append(time.perf_counter() - t0)
            res[codec] = {"seconds": min(ts), "file_mb": os.path.getsize(path) / 1e6,
                          "dense_mb_per_s": res["raw_dense_mb"] / min(ts)}
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    res["note"] = ("one HDF5 file per extraction: %d dense maps + image + mask, byte shuffle "
                   "then gzip level 1 or LZF; host wall time, best of 2" % maps.shape[0])
    return res


def run_flashmap(args):
    import torch
    import paper_2609_19190_gb300 as fm
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    img, mask, kw, desc = workload(args.workload)
    nz, ny, nx = img.shape
    tune = None
    if args.tune:
        v = [int(t) for t in args.tune.split(",")]
        keys = ["brick_x", "brick_y", "brick_z", "voxels_per_item", "consumer_warps", "stages",
                "ctas_per_sm"]
        tune = dict(zip(keys, v))
    params = fm.fr_map_params_init(nx, ny, nz, device=local, **kw)
    plan = fm.fr_map_plan(params, torch.from_numpy(mask), tune=tune)
    n_voi, nf = plan.n_voi, plan.n_rows
    img_dev = torch.from_numpy(img).to(dev)
    out = torch.empty((nf, n_voi), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        fm.fr_map_run(plan, img_dev, out)
    fm.fr_map_sync_status(plan)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    step_ms, kern_ms = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fm.fr_map_run(plan, img_dev, out)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(fm.fr_plan_last_kernel_ms(plan))
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    fm.fr_map_sync_status(plan)
    t_dev = max_over_ranks(sum(step_ms) / 1e3, world)
    value = world * args.steps * n_voi * nf / t_dev

    e2e = None
    if not args.no_e2e:
        img_pin = torch.from_numpy(img).pin_memory()
        out_pin = torch.empty((nf, n_voi), dtype=torch.float32).pin_memory()
        fm.fr_map_run_host(plan, img_pin, out_pin)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fm.fr_map_run_host(plan, img_pin, out_pin)
        t_e2e = max_over_ranks(time.perf_counter() - t0, world)
        barrier(world)
        e2e = {"value": world * args.steps * n_voi * nf / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(img.nbytes), "d2h_bytes_per_step": int(nf * n_voi * 4),
               "ms_per_step": 1e3 * t_e2e / args.steps}

    if rank != 0:
        return
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ops = algorithmic_ops(mask, kw["kernel_radius"], kw["glcm_distance"])
    kmean = statistics.mean(kern_ms) / 1e3
    achieved = ops / kmean / 1e9
    nominal = sms * ALU_LANES_PER_SM * sm_max * 1e6 / 1e9
    try:
        add_ops, mad_ops, fma_ops = fm.fr_measure_alu_peak(local)
        peak = max(add_ops, mad_ops, fma_ops) / 1e9
        basis = ("measured lane-op issue, %d SMs, full occupancy, best of 3: int32 add %.1f, "
                 "int32 multiply-add %.1f, fp32 FMA %.1f Gop/s; peak = the fastest pipe "
                 "(nominal %d x %d lanes x %.0f MHz = %.1f Gop/s)"
                 % (sms, add_ops / 1e9, mad_ops / 1e9, fma_ops / 1e9, sms, ALU_LANES_PER_SM,
                    sm_max, nominal))
    except Exception as e:  # the helper failed: the nominal figure, said so
        peak, basis = nominal, "nominal (measurement failed: %s)" % e
    counters = NCU_COUNTERS.get((args.workload, source_digest()), {})
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
            "frac": achieved / peak, "traffic": counters.get("traffic"),
            "traffic_basis": counters.get("traffic_basis"),
            "kernel": "fr_map_kernel", "kernel_ms": 1e3 * kmean,
            "ops_per_launch": ops, "peak_basis": basis,
            "issue_active_pct": counters.get("issue_active_pct"),
            "shared_pipe_pct": counters.get("shared_pipe_pct"),
            "hbm_gbs_achieved": (img.nbytes + 4 * nf * n_voi + 4 * n_voi) / kmean / 1e9,
            "hbm_peak_gbs": peaks.get("hbm_gbs")}
    extra = {}
    for name in [w for w in args.extra_workloads.split(",") if w and w != args.workload]:
        extra[name] = measure_plain(name, dev, args.steps, args.warmup)
    batched = None
    if not args.no_batched:
        batched = measure_batched("mixed", args.batch_vois, dev)
        batched["small_vois"] = measure_batched("small", args.small_vois, dev)
    served = None
    if not args.no_served:
        served = measure_served(args.served_requests,
                                [float(r) for r in args.served_rates.split(",")], dev,
                                args.served_seconds)
    scalar = None
    if not args.no_scalar:
        scalar = measure_scalar(img, mask, kw, dev, args.steps)
    drain = None
    if not args.no_drain and world == 1:
        drain = measure_drain(plan, params, out, img, mask)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, cores, n, dt, _ = oracle_rate(img, mask, kw, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d seeded VOI voxels of the workload, all 93 maps, %.1f s" % (n, dt)}
        rate1, _, n1, dt1, _ = oracle_rate(img, mask, kw, args.cpu_single_seconds, seed=12,
                                           threads=1)
        cpu["single_thread"] = {"value": rate1, "unit": UNIT, "cores": 1,
                                "sample": "%d seeded VOI voxels, all 93 maps, %.1f s"
                                          % (n1, dt1)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "n_voi": n_voi, "maps": nf,
                   "l2": "flushed between steps (256 MiB write, outside the events)",
                   "replicas": "each rank maps its own copy (no data-path collective)",
                   "launch": {"grid_note": "persistent, one CTA of 16 warps per SM; thread 0 "
                                            "feeds the TMA halo copies",
                              "tune": tune}},
        "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
        "extra_workloads": extra,
        "batched": batched, "served": served, "scalar": scalar, "drain": drain,
        "gpu_launches": 5 * args.steps,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_flashmap(args)
    if "WORLD_SIZE" in os.environ and int(os.environ["WORLD_SIZE"]) > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
