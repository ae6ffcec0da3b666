"""Benchmark: Gsegments/s of the octree ray-casting pass on one GB300.

A step is one pass of the whole hot path over one batch: 64 cameras of uneven
map sizes (128^2 .. 2048^2), fields of view (1 .. 1/64 of the box) and level
cuts, mixed modes (column / weighted mean / max), rendered by one persistent
launch fed by the ray-tile work queue, on a 16.0M-leaf synthetic galaxy octree
(leaves at levels 7-12, cap 16, density + 3 velocity fields, float32), FP32
compensated accumulation.  A segment is one leaf crossed by one ray (the sum of
the per-pixel visited counts).  The same batch is also timed with the FP64
kernel, and the FP32 maps are compared with the FP64 ones.

The default run then measures the other workloads, each in its own record
under "configs" (with its own clock samples): the plain-method tiny tree
(256^2, FP64 and FP32 against the oracle), the 1024^2 galaxy precision case
(every mode and precision, errors against the FP64 kernel and the oracle), the
8-frame 4096^2 zoom on the 193M-leaf level-22 tree (per-frame error against
the FP64 kernel, slice map and adaptive blur beside it) and a Poisson request
stream at 50 req/s on the batch tree (p50/p99 latency, queue wait and render
time).  Comparisons with the oracle belong to each record's CPU-baseline leg,
which also times the oracle on the same sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config batch|precision|zoom|serve|tiny] [--headline-only]

--impl reference times the CPU oracle (plain FP64 C, all host cores) on a
bounded sample of each step's rays.  Under torchrun (N > 1) every rank renders
its own batch (seeded by rank, weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "Gsegments/s (FP32-Kahan batch; FP64 kernel and rel err vs FP64 reported beside)"
UNIT = "Gsegments/s"
# Algorithmic bytes a segment must read: the child word that says the cell is a
# leaf at this cut (4 B) and the scalars: density (column, max), density and
# three velocity components (wmean); float32 fields, or float64 (8 B each).
BYTES_PER_SEG = {0: 8, 1: 20, 2: 8}
BYTES_PER_SEG_F64 = {0: 12, 1: 36, 2: 12}
# Essential lane operations per segment of the exact incremental step (FP32
# compensated kernel), by mode: exit face 6, chord 5, accumulate 5, error-term
# update 4, neighbour 4, leaf test 3, field fetch 2, count 1 = 30 (column);
# max replaces chord + accumulate by one fmax (21); wmean adds three loads, the
# dot product, a multiply and the Neumaier sum (43).
OPS_PER_SEG = {0: 30, 1: 43, 2: 21}
# 152 SMs x 128 lanes x 2.07 GHz: one lane operation per lane per clock.
ALU_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12
FP64_OPS_PER_SEG = 5       # int64->f64, the chord's multiply by the per-camera factor, float->double, multiply, add
FP64_PEAK_TFLOPS = 1.25    # nominal GB300 FP64 rate


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--config", choices=("batch", "precision", "zoom", "serve", "tiny"), default="batch")
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--graph", action="store_true", help="replay batches through CUDA graphs")
    ap.add_argument("--cams", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--headline-only", action="store_true", help="skip the other workloads' records")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(config, rank, n_cams, precision):
    from paper_1210_8014_gb300 import inputs
    if config == "batch":
        tree = inputs.cached("galaxy_batch", inputs.batch_tree)
        cams = inputs.batch_cameras(tree, n_cams=n_cams, precision=precision, seed=3 + 1000 * rank)
        name = (f"{n_cams}-camera batch, sizes 128^2..2048^2, fov 1..1/64, pixel-rule level cut, mixed modes; "
                f"galaxy octree {tree.n_leaves} leaves (levels {min(map(int, tree.info['leaf_hist']))}-{tree.depth}, "
                f"mass threshold 2^-22 of total)")
    elif config == "tiny":
        tree = inputs.plain_tree()
        cams = [inputs.axis_camera(256, max_level=7, precision=precision)]
        name = f"plain-method tiny tree ({tree.n_leaves} leaves, float64), +z view 256^2 at level 7, column"
    elif config == "precision":
        tree = inputs.cached("galaxy_precision", inputs.galaxy_precision_tree)
        cams = [c for c in inputs.galaxy_precision_cameras(tree, precisions=(precision,))]
        name = f"1024^2 random-direction view, 3 modes; galaxy octree {tree.n_leaves} leaves, threshold 2^-20"
    else:
        tree = inputs.cached("galaxy_zoom", inputs.zoom_tree)
        cams = inputs.zoom_cameras(tree, precision=precision)
        name = f"8-frame 4096^2 zoom toward the centre; galaxy octree {tree.n_leaves} leaves to level {tree.depth}"
    return tree, cams, name


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for name, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the batch kernel's own sources (the kernel and the structs it reads)."""
    h = hashlib.sha256()
    for name in ("amr_trace.cuh", "amr_kernels.cu", "amr_internal.h"):
        h.update((ROOT / "paper_1210_8014_gb300" / "csrc" / "amr" / name).read_bytes())
    return h.hexdigest()[:16]


def recorded_profile(config):
    """Figures of the committed ncu summary for this workload (DRAM bytes per
    launch, cache hit rates), if it was taken on the current kernel source."""
    f = ROOT / "profiles" / f"batch_kernel_{config}_traffic.txt"
    if not f.exists():
        return {}
    kv = {}
    for line in f.read_text().splitlines():
        if ":" in line and not line.lstrip().startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha") != kernel_source_hash():
        return {}
    out = {}
    for key in ("dram_bytes_per_launch_full_workload", "l1_sector_hit_pct", "l2_sector_hit_pct", "issue_active_pct",
                "alu_pipe_pct", "fma_pipe_pct", "thread_inst_per_segment"):
        try:
            out[key] = float(kv[key])
        except (KeyError, ValueError):
            pass
    return out


def recorded_traffic(config):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source."""
    return recorded_profile(config).get("dram_bytes_per_launch_full_workload")


def recorded_compulsory(config):
    """Compulsory bytes per launch (unique oct records and values the
    workload's cameras touch under their cuts), counted by the oracle's
    instrumented pass and committed as profiles/compulsory_bytes_<config>.txt;
    None without that file."""
    f = ROOT / "profiles" / f"compulsory_bytes_{config}.txt"
    if not f.exists():
        return None
    out = {}
    for line in f.read_text().splitlines():
        if ":" in line and not line.lstrip().startswith("#"):
            k, v = line.split(":", 1)
            try:
                out[k.strip()] = float(v.strip())
            except ValueError:
                pass
    return out or None


def dram_view(prof, ms, peak):
    """Measured DRAM traffic (ncu, per launch) as GB/s over the live kernel
    time, its fraction of the measured copy bandwidth, and the cache hit
    rates of the same summary; None without a summary for this kernel source."""
    if "dram_bytes_per_launch_full_workload" not in prof:
        return None
    gbs = prof["dram_bytes_per_launch_full_workload"] / (ms * 1e-3) / 1e9
    return {"gbs": gbs, "frac": gbs / peak, "l1_sector_hit_pct": prof.get("l1_sector_hit_pct"),
            "l2_sector_hit_pct": prof.get("l2_sector_hit_pct")}


def pipe_view(prof):
    """Issue and pipe utilisation of the committed full capture of this kernel
    source (what actually bounds it: the integer ALU pipe runs at half the
    lane rate the essential-ops peak assumes); None without one."""
    keys = ("issue_active_pct", "alu_pipe_pct", "fma_pipe_pct", "thread_inst_per_segment")
    if not all(k in prof for k in keys):
        return None
    out = {k: prof[k] for k in keys}
    out["source"] = "ncu --set full, first 8 cameras of the batch"
    return out


def hbm_roofline(algo_bytes, ms, config, extra=None):
    """The kernel against HBM bandwidth: the algorithmic bytes of the launch
    (bytes per segment x segments) over its measured time, as a fraction of
    the measured copy bandwidth, with the ncu DRAM traffic of the same kernel
    source (null when the source changed since the capture)."""
    peak, kind = measured_peaks()
    achieved = algo_bytes / (ms * 1e-3) / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": recorded_traffic(config), "peak_kind": kind + " (MEASURED_PEAKS.json hbm_gbs)",
           "algorithmic_bytes_per_launch": algo_bytes}
    if extra:
        out.update(extra)
    return out


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest value of x over all ranks (the step time every rank waits for)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: int, device="cpu") -> int:
    """Sum of x over all ranks (every rank renders its own seeded batch)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def replica_throughput(total_segments: int, ms_max: float) -> float:
    """Whole-job Gsegments/s: the segments every rank rendered in one step
    (weak scaling: a fixed batch per rank), over the slowest rank's step time."""
    return total_segments / (ms_max * 1e-3) / 1e9


def map_errors(mode, a, b):
    """(max, p99) error of map a against reference b: columns per pixel relative
    (where b > 0), weighted means and mean levels normwise, max absolute."""
    import torch
    a = a.double()
    b = b.double()
    if mode == 0:
        pos = b > 0
        if not bool(pos.any()):
            return 0.0, 0.0
        rel = (a[pos] - b[pos]).abs() / b[pos]
        return float(rel.max()), float(torch.quantile(rel[:1 << 24].float(), 0.99))
    if mode in (1, 3):
        s = float(b.abs().max())
        e = (a - b).abs() / s if s > 0 else (a - b).abs()
        return float(e.max()), float(torch.quantile(e.flatten()[:1 << 24].float(), 0.99))
    e = float((a - b).abs().max())
    return e, e


# ---------------------------------------------------------------- timing helpers
class Timer:
    """CUDA-event timing of one launch sequence per step on `stream`, with a
    256 MiB buffer (larger than the 129 MB L2) written on the same stream
    before each step."""

    def __init__(self, device, stream):
        import torch
        self.torch = torch
        self.stream = stream
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{device}")

    def run(self, fn, steps, warmup=0):
        torch = self.torch
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            with torch.cuda.stream(self.stream):
                self.flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            fn()
            e1.record(self.stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return times


def _oracle_sample(oracle, lib, tree, cams, budget_s, threads, seed):
    """Segments/s of the oracle on random rays of the cameras, growing the
    sample until it has taken about budget_s of oracle time."""
    rng = np.random.default_rng(seed)
    per_cam = 8
    total_segs, total_t, total_rays = 0, 0.0, 0
    while True:
        for cam in cams:
            pi = rng.integers(0, cam.nx, per_cam)
            pj = rng.integers(0, cam.ny, per_cam)
            t0 = time.perf_counter()
            _, cnt = oracle.render(tree, cam, pixels=(pi, pj), threads=threads, lib=lib)
            total_t += time.perf_counter() - t0
            total_segs += int(cnt.sum())
            total_rays += per_cam
        if total_t >= budget_s or per_cam >= 65536:
            break
        per_cam = int(min(65536, per_cam * max(2.0, budget_s / max(total_t, 1e-3) * 0.6)))
    return total_segs / total_t / 1e9, (f"{total_rays} random rays spread over the {len(cams)} cameras "
                                        f"({total_segs} segments, {total_t:.1f} s of oracle time)")


def cpu_baseline(tree, cams, budget_s=12.0, seed=0):
    """The oracle as it stands, on a bounded random sample of the batch's rays:
    on all host cores (the reported value) and on one thread beside it."""
    import oracle
    threads = os.cpu_count() or 1
    lib = oracle.load()
    tree = oracle.prepare(tree)
    value, sample = _oracle_sample(oracle, lib, tree, cams, budget_s, threads, seed)
    v1, s1 = _oracle_sample(oracle, lib, tree, cams, min(3.0, budget_s), 1, seed + 1)
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": s1}}


def cpu_baseline_vs_gpu(tree, cams, gpu, per_cam, seed, what):
    """CPU-baseline leg of a workload record: the oracle on per_cam sampled
    pixels of each camera (per_cam None: every pixel), on all host cores, timed
    as the baseline; and the GPU maps and counts at the same pixels compared
    with it.  gpu[k] = (map, counts) host arrays of camera k."""
    import oracle
    threads = os.cpu_count() or 1
    lib = oracle.load()
    prepared = oracle.prepare(tree)
    rng = np.random.default_rng(seed)
    segs, t_total, rays = 0, 0.0, 0
    worst = {}
    counts_equal = True
    for cam, (gm, gc) in zip(cams, gpu):
        if per_cam is None:
            t0 = time.perf_counter()
            ref, rc = oracle.render(prepared, cam, threads=threads, lib=lib)
            t_total += time.perf_counter() - t0
            a, c = gm, gc
        else:
            pi = rng.integers(0, cam.nx, per_cam)
            pj = rng.integers(0, cam.ny, per_cam)
            t0 = time.perf_counter()
            ref, rc = oracle.render(prepared, cam, pixels=(pi, pj), threads=threads, lib=lib)
            t_total += time.perf_counter() - t0
            a, c = gm[pj, pi], gc[pj, pi]
        segs += int(rc.sum())
        rays += rc.size
        counts_equal &= bool((np.asarray(c) == rc).all())
        a = np.asarray(a, np.float64)
        if cam.mode == 0:
            pos = ref > 0
            e = float((np.abs(a[pos] - ref[pos]) / ref[pos]).max(initial=0.0))
        elif cam.mode in (1, 3):
            s = float(np.abs(ref).max(initial=0.0))
            e = float(np.abs(a - ref).max(initial=0.0)) / (s if s > 0 else 1.0)
        else:
            e = float(np.abs(a - ref).max(initial=0.0))
        key = f"{['column', 'wmean', 'max', 'level'][cam.mode]}_{['fp64', 'fp32_kahan', 'fp32_plain'][cam.precision]}"
        worst[key] = max(worst.get(key, 0.0), e)
    return {"value": segs / max(t_total, 1e-9) / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{what}: {rays} rays, {segs} segments, {t_total:.2f} s of oracle time",
            "gpu_vs_oracle": {"counts_bit_exact": counts_equal, "max_error": worst}}


def aux_kernels(r, cams, timer, reps=5):
    """Time the slice map, the adaptive blur and the sort-last merge on one
    frame of the workload (the 4th zoom frame): slice = one descent per pixel;
    blur = the mean-level render it needs plus the two gather passes; merge =
    eight partial renders of the frame combined on the device."""
    import torch
    from paper_1210_8014_gb300 import amr
    cam = cams[min(3, len(cams) - 1)]
    dev = torch.device(f"cuda:{r.device}")
    stream = timer.stream
    m = torch.empty((cam.ny, cam.nx), dtype=torch.float32, device=dev)
    lv = torch.empty_like(m)
    lvl_i = torch.empty((cam.ny, cam.nx), dtype=torch.int32, device=dev)
    out = torch.empty_like(m)

    def timed(fn):
        return float(np.median(timer.run(fn, reps, warmup=1)))

    slice_ms = timed(lambda: amr.amr_slice(r.ctx, cam, m, lvl_i, 1, stream.cuda_stream))
    level_cam = cam.with_(mode=amr.AMR_MODE_LEVEL)
    level_ms = timed(lambda: amr.amr_render(r.ctx, level_cam, lv, None, 1, stream.cuda_stream))
    amr.amr_render(r.ctx, cam, m, None, 1, stream.cuda_stream)
    pixel = cam.fov[0] / cam.nx
    blur_ms = timed(lambda: amr.amr_blur(r.ctx, cam.nx, cam.ny, m, lv, pixel, out, stream.cuda_stream))
    torch.cuda.synchronize()
    px = cam.nx * cam.ny
    depth = float(lvl_i.float().mean())
    peak, peak_kind = measured_peaks()
    # slice: without reuse a pixel reads one 8-byte record per level of its
    # descent and its 4-byte value, and writes the value and the level
    slice_bytes = px * (8.0 * depth + 12.0)
    slice_gbs = slice_bytes / (slice_ms * 1e-3) / 1e9
    # blur: 2R + 1 four-byte taps per pixel and pass (R = 0 where it is left
    # sharp), each an L1-served load
    sig = 0.5 * np.exp2(-lv.double().cpu().numpy()) / pixel
    radius = np.where(sig >= 0.5, np.minimum(64, np.floor(3.0 * sig + 0.5)), 0.0)
    taps = 2.0 * float((2.0 * radius + 1.0).sum())
    l1_peak = 152 * 32 * 2.07e9 / 1e12
    blur_ttaps = taps / (blur_ms * 1e-3) / 1e12
    # sort-last merge: eight partials of this frame (FP32 compensated column
    # pairs, 8 B per pixel each, distinct buffers) merged on the device; it
    # reads every partial once and writes the map
    n_parts = 8
    part, _ = r.render_partial([cam])[0]
    parts = [part.clone() for _ in range(n_parts)]
    merged = torch.empty((cam.ny, cam.nx), dtype=torch.float32, device=dev)
    merge_ms = timed(lambda: amr.amr_merge_partials(cam.mode, cam.precision, px, parts, merged, stream.cuda_stream))
    merge_bytes = float(px) * (n_parts * 8 + 4)
    merge_gbs = merge_bytes / (merge_ms * 1e-3) / 1e9
    del parts, part
    return {"frame": f"{cam.nx}^2, fov {cam.fov[0]:g}, level {amr.amr_camera_check(r.ctx, cam)}",
            "merge_ms": merge_ms,
            "merge_roofline": {"bound": "hbm", "achieved": merge_gbs, "peak": peak, "unit": "GB/s",
                               "frac": merge_gbs / peak, "peak_kind": peak_kind,
                               "bytes": merge_bytes, "partials": n_parts},
            "slice_ms": slice_ms, "slice_gpixels_per_s": px / (slice_ms * 1e-3) / 1e9,
            "slice_mean_leaf_level": depth, "level_render_ms": level_ms, "blur_ms": blur_ms,
            "blur_gpixels_per_s": px / (blur_ms * 1e-3) / 1e9,
            "slice_roofline": {"bound": "hbm", "achieved": slice_gbs, "peak": peak, "unit": "GB/s",
                               "frac": slice_gbs / peak, "peak_kind": peak_kind,
                               "bytes_per_pixel": 8.0 * depth + 12.0},
            "blur_roofline": {"bound": "l1", "achieved": blur_ttaps, "peak": l1_peak, "unit": "Ttaps/s",
                              "frac": blur_ttaps / l1_peak,
                              "peak_kind": "derived: 152 SMs x 32 four-byte L1 loads per clock x 2.07 GHz",
                              "taps_per_frame": taps}}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    from paper_1210_8014_gb300 import inputs
    import oracle
    tree, cams, name = workload(args.config, 0, args.cams, inputs.PREC_FP32_KAHAN)
    lib = oracle.load()
    tree = oracle.prepare(tree)
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(123)
    per_cam = 512

    def step():
        segs = 0
        t0 = time.perf_counter()
        for cam in cams:
            pi = rng.integers(0, cam.nx, per_cam)
            pj = rng.integers(0, cam.ny, per_cam)
            _, cnt = oracle.render(tree, cam, pixels=(pi, pj), threads=threads, lib=lib)
            segs += int(cnt.sum())
        return segs, time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    tot_s, tot_t = 0, 0.0
    for _ in range(args.steps):
        s, t = step()
        tot_s += s
        tot_t += t
    value = tot_s / tot_t / 1e9
    sample = f"{per_cam} random rays per camera per step ({per_cam * len(cams)} rays/step)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+int128",
        "data": "synthetic", "config": {"workload": name, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- other workloads
def bench_tiny(device, steps, warmup, with_cpu):
    """Plain-method tiny tree: 256^2 +z view at level 7, column, FP64 and FP32
    compensated kernels; the oracle renders the whole map in the CPU leg."""
    import torch
    from paper_1210_8014_gb300 import amr, inputs
    tree, cams = inputs.tiny_workload()
    cam64 = cams[0]
    cam32 = cam64.with_(precision=amr.AMR_PREC_FP32_KAHAN)
    r = amr.Renderer(tree, device=device)
    stream = torch.cuda.Stream(device=device)
    timer = Timer(device, stream)
    out = {"workload": f"plain-method tiny tree ({tree.n_leaves} leaves, float64), +z view 256^2, level 7, column",
           "rays": cam64.nx * cam64.ny}
    maps = {}
    with Clocks(device) as clk:
        for name, cam in (("fp64", cam64), ("fp32_kahan", cam32)):
            m, c = r.alloc(cam)
            ts = timer.run(lambda: amr.amr_render(r.ctx, cam, m, c, 1, stream.cuda_stream), steps, warmup)
            ms = float(np.median(ts))
            segs = int(c.sum())
            out[name] = {"ms_per_frame": ms, "gsegments_per_s": segs / (ms * 1e-3) / 1e9, "segments": segs,
                         "gpu_launches": steps}
            maps[name] = (m.cpu().numpy(), c.cpu().numpy())
    out["clocks"] = clk.summary()
    out["fp32_vs_fp64_err"] = map_errors(0, torch.from_numpy(maps["fp32_kahan"][0]),
                                         torch.from_numpy(maps["fp64"][0]))[0]
    out["note"] = "latency-bound: the tree fits in L2 (no roofline claim)"
    r.close()
    if with_cpu:
        out["cpu_baseline"] = cpu_baseline_vs_gpu(tree, [cam64, cam32], [maps["fp64"], maps["fp32_kahan"]], None, 0,
                                                  "whole 256^2 map, FP64 and FP32 kernels")
    return out


def bench_precision(device, steps, warmup, with_cpu, tune=True):
    """Galaxy precision case: 1024^2 random-direction whole-box view on the
    5.6M-leaf tree, column / wmean / max, each in FP64, FP32 compensated and
    FP32 plain; errors against the FP64 kernel (whole maps) and the oracle
    (sampled pixels, CPU leg).  With tune, each (mode, precision) frame is
    timed with the launch configuration the autotuner picks for it (the best
    register cap differs between modes)."""
    import torch
    from paper_1210_8014_gb300 import amr, inputs
    tree = inputs.cached("galaxy_precision", inputs.galaxy_precision_tree)
    cams = inputs.galaxy_precision_cameras(tree)
    r = amr.Renderer(tree, device=device)
    stream = torch.cuda.Stream(device=device)
    timer = Timer(device, stream)
    modes = {0: "column", 1: "wmean", 2: "max"}
    precs = {0: "fp64", 1: "fp32_kahan", 2: "fp32_plain"}
    res, host = {}, {}
    with Clocks(device) as clk:
        for cam in cams:
            m, c = r.alloc(cam)
            opts = amr.amr_autotune(r.ctx, [cam], reps=3)[0] if tune else amr.amr_get_options(r.ctx).as_dict()
            ts = timer.run(lambda: amr.amr_render(r.ctx, cam, m, c, 1, stream.cuda_stream), steps, warmup)
            ms = float(np.median(ts))
            segs = int(c.sum())
            key = (cam.mode, cam.precision)
            host[key] = (m, c)
            res[f"{modes[cam.mode]}_{precs[cam.precision]}"] = {
                "ms_per_frame": ms, "gsegments_per_s": segs / (ms * 1e-3) / 1e9, "segments": segs,
                "options": opts}
    errs = {}
    for mode in modes:
        ref = host[(mode, 0)][0]
        for p in (1, 2):
            e, p99 = map_errors(mode, host[(mode, p)][0], ref)
            errs[f"{modes[mode]}_{precs[p]}"] = {"max": e, "p99": p99}
            assert torch.equal(host[(mode, p)][1], host[(mode, 0)][1]), "precisions visited different leaves"
    out = {"workload": f"1024^2 random-direction view, galaxy octree {tree.n_leaves} leaves (threshold 2^-20), "
                       f"column / wmean / max x FP64 / FP32 compensated / FP32 plain",
           "per_mode": res, "err_vs_fp64_kernel": errs, "clocks": clk.summary(),
           "fp32_kahan_over_fp64": {modes[m]: res[f"{modes[m]}_fp32_kahan"]["gsegments_per_s"] /
                                    res[f"{modes[m]}_fp64"]["gsegments_per_s"] for m in modes}}
    gpu = [(host[(c.mode, c.precision)][0].cpu().numpy(), host[(c.mode, c.precision)][1].cpu().numpy())
           for c in cams]
    r.close()
    if with_cpu:
        out["cpu_baseline"] = cpu_baseline_vs_gpu(tree, cams, gpu, 1500, 2,
                                                  "1500 random pixels per mode and precision")
    return out


def bench_zoom(device, steps, warmup, with_cpu):
    """Milky-Way scale: 8 frames of 4096^2, fov 1 -> 1/128 toward the centre
    of the 193M-leaf level-22 tree, one persistent launch per step, FP32
    compensated; FP64 kernel beside it; per-frame errors; slice map and
    adaptive blur on the 4th frame."""
    import torch
    from paper_1210_8014_gb300 import amr, inputs
    t0 = time.perf_counter()
    tree = inputs.cached("galaxy_zoom", inputs.zoom_tree)
    gen_s = time.perf_counter() - t0
    cams32 = inputs.zoom_cameras(tree)
    cams64 = [c.with_(precision=amr.AMR_PREC_FP64) for c in cams32]
    t0 = time.perf_counter()
    r = amr.Renderer(tree, device=device)
    torch.cuda.synchronize()
    load_s = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=device)
    timer = Timer(device, stream)
    o32 = [r.alloc(c) for c in cams32]
    o64 = [r.alloc(c) for c in cams64]

    def launch(cams, outs):
        amr.amr_render_batch(r.ctx, cams, [o[0] for o in outs], [o[1] for o in outs], 1, stream.cuda_stream)

    with Clocks(device) as clk:
        t32 = timer.run(lambda: launch(cams32, o32), steps, warmup)
    t64 = timer.run(lambda: launch(cams64, o64), max(2, steps // 2), 1)
    ms32, ms64 = float(np.median(t32)), float(np.median(t64))
    seg_frame = [int(o[1].sum()) for o in o32]
    assert seg_frame == [int(o[1].sum()) for o in o64], "FP32 and FP64 kernels visited different leaves"
    segs = sum(seg_frame)
    frames = []
    for c, a, b, s in zip(cams32, o32, o64, seg_frame):
        e, p99 = map_errors(0, a[0], b[0])
        frames.append({"fov": c.fov[0], "level": amr.amr_camera_check(r.ctx, c), "segments": s,
                       "max_rel_err_vs_fp64": e, "p99_rel_err_vs_fp64": p99})
    algo = segs * BYTES_PER_SEG[0]
    aux = aux_kernels(r, cams32, timer)
    out = {"workload": f"8-frame 4096^2 zoom (fov 1 -> 1/128) toward the centre, column, FP32 compensated; "
                       f"galaxy octree {tree.n_leaves} leaves, {tree.n_oct} octs, levels 7-{tree.depth}",
           "gsegments_per_s": segs / (ms32 * 1e-3) / 1e9, "ms_per_step": ms32, "ms_per_frame": ms32 / len(cams32),
           "segments_per_step": segs, "gpu_launches": steps,
           "fp64_kernel": {"gsegments_per_s": segs / (ms64 * 1e-3) / 1e9, "ms_per_step": ms64},
           "frames": frames, "roofline": hbm_roofline(algo, ms32, "zoom", {"compulsory": recorded_compulsory("zoom")}),
           "clocks": clk.summary(),
           "setup_s": {"generate": gen_s, "load": load_s}, "aux_kernels": aux}
    gpu = [(o[0].cpu().numpy(), o[1].cpu().numpy()) for o in o32]
    del o32, o64
    r.close()
    torch.cuda.empty_cache()
    if with_cpu:
        out["cpu_baseline"] = cpu_baseline_vs_gpu(tree, cams32, gpu, 96, 4, "96 random pixels per frame")
    return out


def serve_stream(r, tree, seconds, device, slots=3, budget=1 << 30, max_batch=16, graph=False):
    """Poisson 50 req/s on the batch tree through amr_submit / amr_wait: each
    request a random-direction camera of 256^2..2048^2, fov 2^-12..1 around a
    disk point and a random mode, delivered into page-locked host buffers (the
    kernel writes them in place).  Latency is arrival to result."""
    import queue as _q
    import torch
    from paper_1210_8014_gb300 import amr, inputs
    reqs = inputs.request_stream(tree, duration_s=seconds)
    amr.amr_server_config(r.ctx, slots=slots, map_budget_bytes=budget, max_batch=max_batch)
    if graph:
        amr.amr_set_options(r.ctx, use_graph=1)
    # warm-up: one render of each size and mode outside the measured stream
    for n in inputs.SIZES_SERVE:
        for mode in (0, 1, 2):
            c = reqs[0][1].with_(nx=n, ny=n, mode=mode)
            amr.amr_render(r.ctx, c, np.empty((n, n), np.float32), np.empty((n, n), np.int32), 0)
    bufs = {n: [(torch.empty((n, n), dtype=torch.float32, pin_memory=True).numpy(),
                 torch.empty((n, n), dtype=torch.int32, pin_memory=True).numpy()) for _ in range(48)]
            for n in inputs.SIZES_SERVE}
    done_segments = [0]
    waitq = _q.Queue()

    def waiter():
        while True:
            item = waitq.get()
            if item is None:
                return
            t, counts = item
            amr.amr_wait(r.ctx, t, -1)
            done_segments[0] += int(counts.sum())

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    use = {n: 0 for n in bufs}
    before = r.stats()["server"]
    with Clocks(device) as clk:
        t0 = time.perf_counter()
        for t_arr, cam in reqs:
            now = time.perf_counter() - t0
            if t_arr > now:
                time.sleep(t_arr - now)
            m, c = bufs[cam.nx][use[cam.nx] % 48]
            use[cam.nx] += 1
            waitq.put((amr.amr_submit(r.ctx, cam, m, c), c))
        waitq.put(None)
        th.join()
        wall = time.perf_counter() - t0
    st = r.stats()["server"]
    # The floor of each request's latency: the same request rendered alone on
    # the idle device (device outputs, CUDA events), after the stream.
    stream = torch.cuda.Stream(device=device)
    solo = []
    for _, cam in reqs:
        m = torch.empty((cam.ny, cam.nx), dtype=torch.float32, device=f"cuda:{device}")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        amr.amr_render(r.ctx, cam, m, None, 1, stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        solo.append(e0.elapsed_time(e1))
    solo = np.array(solo)
    return {"requests": len(reqs), "wall_s": wall, "frames_per_s": (st["done"] - before["done"]) / wall,
            "solo_render_ms": {"p50": float(np.percentile(solo, 50)), "p90": float(np.percentile(solo, 90)),
                               "p99": float(np.percentile(solo, 99)), "max": float(solo.max()),
                               "note": "each request rendered alone on the idle device: the latency floor"},
            "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"]},
            "queue_wait_ms": {"p50": st.get("wait_p50_ms"), "p99": st.get("wait_p99_ms")},
            "render_ms": {"p50": st.get("service_p50_ms"), "p99": st.get("service_p99_ms")},
            "segments_per_s": done_segments[0] / wall / 1e9, "server": st, "clocks": clk.summary(),
            "slots": slots, "map_budget_bytes": budget, "max_batch": max_batch}


def bench_serving(device, seconds):
    from paper_1210_8014_gb300 import amr, inputs
    tree = inputs.cached("galaxy_batch", inputs.batch_tree)
    r = amr.Renderer(tree, device=device)
    try:
        out = serve_stream(r, tree, seconds, device)
    finally:
        r.close()
    out["workload"] = (f"Poisson 50 req/s for {seconds:.0f} s on the {tree.n_leaves}-leaf galaxy octree; "
                       f"256^2..2048^2, fov 2^-12..1, mixed modes, FP32 compensated")
    return out


# ---------------------------------------------------------------- headline
def run_ours(args):
    import torch
    from paper_1210_8014_gb300 import amr, inputs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = local if world > 1 else 0
    torch.cuda.set_device(device)
    dev = f"cuda:{device}"

    t0 = time.perf_counter()
    tree, cams32, name = workload(args.config, rank, args.cams, inputs.PREC_FP32_KAHAN)
    cams64 = [c.with_(precision=inputs.PREC_FP64) for c in cams32]
    gen_s = time.perf_counter() - t0
    t1 = time.perf_counter()
    r = amr.Renderer(tree, device=device)       # validation, linearisation, links, upload
    torch.cuda.synchronize()
    load_s = time.perf_counter() - t1
    stream = torch.cuda.Stream(device=device)
    timer = Timer(device, stream)
    if args.graph:
        amr.amr_set_options(r.ctx, use_graph=1)
    tuned = None
    if not args.no_autotune:
        # Tile shape, block size and queue grab picked on this batch (outside the timed region).
        tuned, _ = amr.amr_autotune(r.ctx, cams32, reps=3)

    def outputs(cams):
        maps = [torch.empty((c.ny, c.nx), dtype=torch.float64 if c.precision == 0 else torch.float32, device=dev)
                for c in cams]
        cnts = [torch.empty((c.ny, c.nx), dtype=torch.int32, device=dev) for c in cams]
        return maps, cnts

    m32, c32 = outputs(cams32)
    m64, c64 = outputs(cams64)

    def launch(cams, maps, cnts):
        amr.amr_render_batch(r.ctx, cams, maps, cnts, 1, stream.cuda_stream)

    # warm-up, parity of FP32 vs FP64 on this batch, per-camera segments
    for _ in range(max(1, args.warmup)):
        launch(cams32, m32, c32)
        launch(cams64, m64, c64)
    torch.cuda.synchronize()
    seg_cam = [int(c.sum()) for c in c32]
    assert seg_cam == [int(c.sum()) for c in c64], "FP32 and FP64 kernels visited different leaves"
    segs = sum(seg_cam)
    f64_fields = tree.fields[0].dtype == np.float64
    bps = BYTES_PER_SEG_F64 if f64_fields else BYTES_PER_SEG
    algo_bytes = sum(s * bps[min(c.mode, 2)] for s, c in zip(seg_cam, cams32))
    err = {"column": 0.0, "wmean": 0.0, "max": 0.0}
    per_camera = []
    for c, a, b in zip(cams32, m32, m64):
        e, p99 = map_errors(c.mode, a, b)
        key = {0: "column", 1: "wmean", 2: "max"}[min(c.mode, 2)]
        err[key] = max(err[key], e)
        per_camera.append({"mode": c.mode, "n": c.nx, "max": e, "p99": p99})

    def timed(cams, maps, cnts, steps):
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        times = timer.run(lambda: launch(cams, maps, cnts), steps)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return times, time.perf_counter() - wall0

    with Clocks(device) as clk:
        t32, wall32 = timed(cams32, m32, c32, args.steps)
    t64, _ = timed(cams64, m64, c64, max(3, args.steps // 2))
    ms32 = float(np.mean(t32))
    ms64 = float(np.mean(t64))
    total_segs = segs
    if world > 1:
        ms32 = max_over_ranks(ms32, dev)
        total_segs = sum_over_ranks(segs, dev)
    value = replica_throughput(total_segs, ms32)
    value64 = segs / (ms64 * 1e-3) / 1e9

    # end to end through the C ABI with host buffers: camera upload and map/count readback inside.
    # Page-locked host buffers (what a serving client would keep): the kernel
    # writes the maps and counts straight into them over the host link.
    hmaps = [torch.empty((c.ny, c.nx), dtype=torch.float32, pin_memory=True).numpy() for c in cams32]
    hcnts = [torch.empty((c.ny, c.nx), dtype=torch.int32, pin_memory=True).numpy() for c in cams32]
    amr.amr_render_batch(r.ctx, cams32, hmaps, hcnts, 0)
    e2e_t = []
    h2d_before = r.stats()["h2d_bytes"]
    for _ in range(max(3, args.steps // 2)):
        with torch.cuda.stream(stream):
            timer.flush.fill_(1)
        torch.cuda.synchronize()
        a = time.perf_counter()
        amr.amr_render_batch(r.ctx, cams32, hmaps, hcnts, 0)
        e2e_t.append(time.perf_counter() - a)
    e2e_ms = float(np.mean(e2e_t)) * 1e3
    d2h = sum(m.nbytes + c.nbytes for m, c in zip(hmaps, hcnts))
    # what the library uploaded per step (camera records, tile prefix sums,
    # pixel-offset tables), counted by the library itself
    h2d = (r.stats()["h2d_bytes"] - h2d_before) // len(e2e_t)

    aux = aux_kernels(r, cams32, timer) if args.config == "zoom" else None
    algo_ops = sum(s_ * OPS_PER_SEG[min(c.mode, 2)] for s_, c in zip(seg_cam, cams32))
    alu_achieved = algo_ops / (ms32 * 1e-3) / 1e12
    fp64_achieved = segs * FP64_OPS_PER_SEG / (ms64 * 1e-3) / 1e12
    stats = r.stats()
    prof = recorded_profile(args.config)
    roof = hbm_roofline(algo_bytes, ms32, args.config, {
        "bytes_per_segment": bps, "compulsory": recorded_compulsory(args.config),
        "dram": dram_view(prof, ms32, measured_peaks()[0]),
        "alu": {"bound": "alu", "achieved": alu_achieved, "peak": ALU_PEAK_TOPS, "unit": "Tops/s",
                "frac": alu_achieved / ALU_PEAK_TOPS, "peak_kind": "derived: 152 SMs x 128 lanes x 2.07 GHz",
                "ops_per_segment": OPS_PER_SEG, "algorithmic_ops_per_launch": algo_ops,
                "pipes": pipe_view(prof)}})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+int64", "data": "synthetic",
        "config": {"workload": name, "cameras": len(cams32), "rays_per_step": int(sum(c.nx * c.ny for c in cams32)),
                   "segments_per_step": total_segs, "segments_per_step_rank0": segs,
                   "l2": "256 MiB buffer written on the timed stream before each timed step",
                   "options": tuned or amr.amr_get_options(r.ctx).as_dict(), "parallelism": f"replicas{world}"},
        "ms_per_frame": ms32 / len(cams32),
        "fp64_kernel": {"value": value64, "ms_per_step": ms64, "unit": UNIT,
                        "roofline": {"bound": "fp64", "achieved": fp64_achieved, "peak": FP64_PEAK_TFLOPS,
                                     "unit": "TFLOP/s", "frac": fp64_achieved / FP64_PEAK_TFLOPS,
                                     "peak_kind": "nominal", "ops_per_segment": FP64_OPS_PER_SEG}},
        "fp32_over_fp64": value / world / value64,
        "fp32_vs_fp64_err": err,
        "fp32_vs_fp64_err_per_frame": per_camera if len(cams32) <= 8 else None,
        "roofline": roof,
        "e2e": {"value": segs / (e2e_ms * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "timed_wall_s": wall32,
        "setup_s": {"generate": gen_s, "load": load_s},
        "regs": stats.get("regs"),
        "aux_kernels": aux,
    }
    with_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    if with_cpu:
        line["cpu_baseline"] = cpu_baseline(tree, cams32)
    del m32, c32, m64, c64
    r.close()
    torch.cuda.empty_cache()
    if args.config == "batch" and world == 1 and not args.headline_only:
        sub_steps = max(3, min(args.steps, 10))
        sub_warm = max(3, min(args.warmup, 5))
        line["configs"] = {
            "tiny_plain_256": bench_tiny(device, sub_steps, sub_warm, with_cpu),
            "galaxy_precision_1024": bench_precision(device, sub_steps, sub_warm, with_cpu,
                                                     tune=not args.no_autotune),
            "zoom_level22_8x4096": bench_zoom(device, min(sub_steps, 5), 2, with_cpu),
            "serving_poisson_50rps": bench_serving(device, 20.0),
        }
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def run_serve(args):
    """Interactive-zoom serving on its own: the request stream of
    bench_serving for --serve-seconds, as one JSON line."""
    from paper_1210_8014_gb300 import amr, inputs
    tree = inputs.cached("galaxy_batch", inputs.batch_tree)
    r = amr.Renderer(tree)
    try:
        st = serve_stream(r, tree, args.serve_seconds, 0, graph=args.graph)
    finally:
        r.close()
    line = {
        "metric": "served frames/s at 50 req/s offered (p50/p99 latency beside)", "value": st["frames_per_s"],
        "unit": "frames/s", "n_gpus": 1, "steps": st["requests"], "warmup": 12,
        "ms_per_step": 1e3 * st["wall_s"] / max(1, st["requests"]), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+int64", "data": "synthetic",
        "config": {"workload": f"Poisson 50 req/s for {args.serve_seconds:.0f} s on the {tree.n_leaves}-leaf galaxy "
                               f"octree; 256^2..2048^2, fov 2^-12..1, mixed modes, FP32 compensated",
                   "requests": st["requests"], "slots": st["slots"], "map_budget_bytes": st["map_budget_bytes"],
                   "graph": bool(args.graph)},
    }
    line.update({k: st[k] for k in ("latency_ms", "queue_wait_ms", "render_ms", "solo_render_ms", "server",
                                     "segments_per_s", "clocks")})
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
