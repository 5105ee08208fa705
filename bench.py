#!/usr/bin/env python3
"""Benchmark: depth points fused per second (allocate + integrate) on one
640x480 synthetic room frame into a hash-blocked TSDF volume (voxel 5 mm,
truncation 2 cm, 2^20 table slots, 2^18 pool blocks).

One step = one pass of the whole hot path (allocate + integrate, paper
Section 2.2) over one frame through tsdf_fuse_frame_async -- by default the
fused tile kernel -- into a freshly reset volume (so allocation never
degenerates into a lookup-only pass, Section 4.2). Between steps, outside the
timed events, the volume is reset and L2 is scrubbed (512 MB write, then
512 MB read). Each step is timed with CUDA events on the launching stream. The
same frames are also run as the two separate stages (stage A, then stage B),
each with its own events, for the per-stage rooflines.

Prints ONE JSON line. With --impl reference the CPU oracle (single thread,
host cores) is timed on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("depth pts fused/s (alloc+integrate, 640x480) + % HBM roofline; "
          "serving p50/p99")
UNIT = "pts/s"
WORKLOAD = "room_640x480_single_frame"

# The paper's own full integrate path (allocate plus update), median of three
# passes, on the two sm_120 GPUs it names (Section 5, the table of full
# integrate times; synthetic rows only: the real-depth rows need a dataset
# that is not here). Other hardware and other scenes: context, not a target.
PAPER_CONTEXT = {
    "source": "Section 5, full integrate path (allocate + update), median of three passes",
    "rows": [
        {"workload": "plane, 320,356 points", "gpu": "RTX 5070 Ti",
         "ms": {"cuda_cpp": 0.363, "rust": 0.379, "triton": 0.875}},
        {"workload": "plane, 320,356 points", "gpu": "RTX 5060",
         "ms": {"cuda_cpp": 0.673, "rust": 0.686, "triton": 1.665}},
        {"workload": "sphere, 320k points", "gpu": "RTX 5070 Ti",
         "ms": {"cuda_cpp": 0.278, "rust": 0.308, "triton": 0.828}},
        {"workload": "sphere, 320k points", "gpu": "RTX 5060",
         "ms": {"cuda_cpp": 0.511, "rust": 0.538, "triton": 1.526}},
        {"workload": "sphere, 1.28M points", "gpu": "RTX 5070 Ti",
         "ms": {"cuda_cpp": 0.975, "rust": 1.023, "triton": 2.982}},
        {"workload": "sphere, 1.28M points", "gpu": "RTX 5060",
         "ms": {"cuda_cpp": 1.709, "rust": 1.737, "triton": 5.707}},
    ],
    "best_pts_per_s": {"value": 1.31e9, "row": "sphere, 1.28M points, CUDA C++, RTX 5070 Ti"},
}
N_FRAMES = 4           # distinct orbit frames, cycled over the steps
FLUSH_BYTES = 512 << 20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def config_dict(spec, frames, l2_fetch_bytes=0):
    return {"workload": WORKLOAD, "width": 640, "height": 480,
            "voxel_m": spec.voxel_size, "truncation_m": spec.truncation,
            "table_slots": spec.table_slots, "pool_blocks": spec.pool_blocks,
            "points_per_frame": int(np.mean([f.valid_points for f in frames])),
            "distinct_frames": len(frames), "colour": True,
            "l2": "flushed between steps (512 MB write + 512 MB read, outside the timed events)",
            "l2_fetch_bytes": l2_fetch_bytes or "context default",
            "volume": "reset between steps: every step fuses into an empty volume"}


def l2_scrub(flush, scrub, i):
    """Leave L2 cold and clean: write 512 MB (evicts everything), then read
    another 512 MB (writes those dirty lines back and refills L2 with clean
    lines), so the timed kernels neither hit in L2 nor pay for write-backs of
    the scrub."""
    flush.fill_(i & 0xFF)
    scrub.sum()


def frame_indices(rank=0):
    """Orbit frames that rank `rank` fuses: every rank a distinct set (replicas
    of the path on different inputs, no data exchanged)."""
    return [37 * (rank * N_FRAMES + i) for i in range(N_FRAMES)]


def make_frames(rank=0):
    from paper_2608_08287_gb300 import synth
    return [synth.room_frame(k) for k in frame_indices(rank)]


def reduce_job(points, elapsed, world, device):
    """Whole-job totals over the ranks: points summed, elapsed time the maximum
    (the job ends with its slowest rank). The only collective on the bench
    path; it runs outside the timed region. `device` is "cuda" under NCCL,
    "cpu" under gloo."""
    if world <= 1:
        return int(points), float(elapsed)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([int(points)], device=device, dtype=torch.int64)
    dist.all_reduce(p)
    return int(p.item()), float(t.item())


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, interval_ms=100):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.rows = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ----------------------------------------------------------------------------
# traffic from a committed ncu summary, valid only for the current kernel source
# ----------------------------------------------------------------------------
def kernel_source_hash():
    """Hash of the device code (comments and blank space removed, so that
    documentation edits do not invalidate a capture of the same kernels)."""
    import re
    h = hashlib.sha256()
    for f in ("tsdf_device.cuh", "tsdf_tile.cuh", "tsdf_kernels.cu", "tsdf_kernels_split.cu"):
        with open(os.path.join(ROOT, "paper_2608_08287_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def committed_traffic(kernel):
    """dram bytes per launch recorded under profiles/ for this kernel source, else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel \
                and parts[1] == src:
            return float(parts[2])
    return None


# ----------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------
def vol_fuse_mode(vol):
    return getattr(vol, "_fuse_mode", 2)


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2608_08287_gb300 import synth, tsdf
    from paper_2608_08287_gb300.build import build_library

    torch.cuda.set_device(local_rank)
    if rank == 0:
        build_library()
    if world > 1:
        torch.distributed.barrier()
    # the L2 fetch granularity (0: the CUDA context's default, unchanged)
    if args.l2_fetch_bytes:
        st, _ = tsdf.tsdf_set_l2_fetch_bytes(args.l2_fetch_bytes)
        assert st == "OK", st
    spec = synth.ROOM_640
    frames = make_frames(rank)
    vol = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    for k, x in (("probe_load", args.probe_load), ("integrate_mode", args.integrate_mode),
                 ("allocate_mode", args.allocate_mode), ("fuse_mode", args.fuse_mode)):
        if x is not None:
            assert vol.set_option(k, x) == "OK"
    vol._fuse_mode = 2 if args.fuse_mode is None else args.fuse_mode
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    dev = [(torch.from_numpy(f.depth).cuda(), torch.from_numpy(f.rgb).cuda()) for f in frames]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    scrub = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    W, H = 640, 480

    # per-frame work counts (units of the algorithmic bytes) from the oracle,
    # before any timing; the GPU's own export of each frame is compared with
    # them as a cross-check
    work = oracle_work_counts(frames, spec)
    gpu_counts_match = True
    for f, (d, c), w in zip(frames, dev, work):
        assert vol.reset(sp) == "OK"
        assert tsdf.tsdf_fuse_frame(vol.handle, d, W, H, f.intr, f.pose, c, sp) == "OK"
        coords, vox = vol.export(sp)
        gpu_counts_match &= (len(coords) == w["blocks"] and
                             int((vox[:, 1] > 0).sum()) == w["voxels"])

    def prepare(i):
        vol.reset(sp)
        with torch.cuda.stream(stream):
            l2_scrub(flush, scrub, i)

    # the C structs of each frame's intrinsics and pose, built once
    structs = [(tsdf.intrinsics(f.intr), tsdf.pose_struct(f.pose)) for f in frames]

    def one_step(i, evs=None):
        """The whole hot path for one frame: tsdf_fuse_frame_async (default mode)."""
        f = frames[i % len(frames)]
        d, c = dev[i % len(frames)]
        intr, pose = structs[i % len(frames)]
        prepare(i)
        if evs:
            evs[0].record(stream)
        assert tsdf.tsdf_fuse_frame_async(vol.handle, d, W, H, intr, pose, c, sp) == "OK"
        if evs:
            evs[1].record(stream)
        return f.valid_points

    def split_step(i, evs):
        """The same frame as two kernels, stage A then stage B, each timed."""
        f = frames[i % len(frames)]
        d, c = dev[i % len(frames)]
        prepare(i)
        evs[0].record(stream)
        assert tsdf.tsdf_allocate_async(vol.handle, d, W, H, f.intr, f.pose, sp) == "OK"
        evs[1].record(stream)
        assert tsdf.tsdf_integrate_async(vol.handle, d, W, H, f.intr, f.pose, c, sp) == "OK"
        evs[2].record(stream)

    for i in range(args.warmup):
        one_step(i)
    assert vol.status(sp) == "OK"
    torch.cuda.synchronize()

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = tsdf.tsdf_launch_count()
    points = 0
    with ClockSampler(local_rank, args.clock_ms) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            points += one_step(args.warmup + i, events[i])
        stream.synchronize()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    launches = tsdf.tsdf_launch_count() - launches0
    st = vol.status(sp)
    assert st == "OK", st
    step_ms = [events[i][0].elapsed_time(events[i][1]) for i in range(args.steps)]
    points_all, total_ms = reduce_job(points, float(sum(step_ms)), world, "cuda")
    value = points_all / (total_ms / 1e3)

    # the two-stage split of the same frames, for the per-stage rooflines
    n_split = min(args.steps, 100)
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n_split)]
    for i in range(3):
        split_step(i, sev[0])
    for i in range(n_split):
        split_step(args.warmup + i, sev[i])
    torch.cuda.synchronize()
    assert vol.status(sp) == "OK"
    ta = [e[0].elapsed_time(e[1]) for e in sev]
    tb_ = [e[1].elapsed_time(e[2]) for e in sev]

    # the paper's amortised protocol on the same frames (secondary)
    amortized = None
    if rank == 0:
        try:
            amortized = run_amortized(torch, tsdf, spec, frames, dev, structs, stream, flush,
                                      scrub)
        except Exception as e:  # noqa: BLE001
            amortized = {"error": repr(e)}

    # rooflines: the algorithmic bytes of each stage from the oracle's work
    # counts of the timed frames (every block is new: each step fuses into an
    # empty volume, so N_new = U_b)
    hbm, peak_kind = peaks()
    mean = lambda k: float(np.mean([w[k] for w in work]))
    a_bytes, b_bytes, f_bytes = (float(np.mean(x)) for x in zip(*[stage_bytes(w) for w in work]))
    a_ms, b_ms = float(np.mean(ta)), float(np.mean(tb_))
    step_mean = total_ms / args.steps
    a_gbs, b_gbs = a_bytes / (a_ms * 1e6), b_bytes / (b_ms * 1e6)
    f_gbs = f_bytes / (step_mean * 1e6)
    fused = vol_fuse_mode(vol) != 0
    if fused:
        dom = ("fused", f_bytes, step_mean, f_gbs, "fuse_kernel")
    elif b_ms >= a_ms:
        dom = ("integrate", b_bytes, b_ms, b_gbs, "integrate_kernel")
    else:
        dom = ("allocate", a_bytes, a_ms, a_gbs, "allocate_kernel")
    roof = {"bound": "hbm", "kernel": dom[0], "achieved": round(dom[3], 1), "peak": hbm,
            "peak_kind": f"{peak_kind} hbm_gbs", "unit": "GB/s",
            "frac": round(dom[3] / hbm, 4), "algorithmic_bytes": int(dom[1]),
            "work_counts": "oracle (U_b, N_new, U_v of each timed frame); the GPU export "
                           + ("agrees" if gpu_counts_match else "DISAGREES"),
            "traffic": committed_traffic(dom[4])}

    # what the single-frame autotuner picks for this workload (a report: the
    # headline above times the default configuration)
    tuning = None
    if rank == 0 and not args.headline_only:
        assert vol.reset(sp) == "OK"
        d, c = dev[0]
        st, tuning = tsdf.tsdf_autotune_frame(vol.handle, d, W, H, frames[0].intr,
                                              frames[0].pose, c, 10, sp)
        tuning = tuning if st == "OK" else {"status": st}
        # back to the configuration the headline timed
        for k, x, default in (("allocate_mode", args.allocate_mode, 1),
                              ("integrate_mode", args.integrate_mode, 0),
                              ("fuse_mode", args.fuse_mode, 2),
                              ("probe_load", args.probe_load, 0)):
            assert vol.set_option(k, default if x is None else x) == "OK"

    # surface extraction of the four frames fused together (compute timed
    # apart from the device-to-host copy, as the paper splits it)
    extraction = None
    if rank == 0 and not args.headline_only:
        extraction = run_extraction(args, vol, frames, dev, tsdf, sp, hbm)

    # end to end through the public C ABI with host buffers
    e2e = run_e2e(args, vol, frames, torch, tsdf, sp, stream, flush, scrub, world)
    vol.close()
    del flush, scrub
    torch.cuda.empty_cache()

    extra = {}
    if rank == 0 and not args.headline_only:
        from paper_2608_08287_gb300 import serving
        try:
            import multiprocessing as mp
            with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
                bank = serving.FrameBank(torch, n_frames=args.bank_frames, step=12, pool=pool)
                sweep_frames = (pool.starmap(serving._render,
                                             [(640, 480, k) for k in range(args.sweep_frames)])
                                if args.sweep_frames else None)
        except Exception as e:  # noqa: BLE001
            bank = sweep_frames = None
            extra["batched"] = extra["serving"] = {"error": repr(e)}
        if bank is not None:
            for key, fn in (("batched", lambda: run_batched(args, torch, tsdf, serving, bank)),
                            ("serving", lambda: run_serving(args, torch, serving, bank))):
                try:
                    extra[key] = fn()
                except Exception as e:  # noqa: BLE001
                    extra[key] = {"error": repr(e)}
        if sweep_frames:
            try:
                extra["load_sweep"] = run_load_sweep(args, torch, tsdf, sweep_frames)
            except Exception as e:  # noqa: BLE001
                extra["load_sweep"] = {"error": repr(e)}
        try:
            extra["small_frames"] = run_small_frames(args, torch, tsdf)
        except Exception as e:  # noqa: BLE001
            extra["small_frames"] = {"error": repr(e)}

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(spec, frames, args.l2_fetch_bytes),
            "stages": {"path": "fused kernel" if fused else "stage A + stage B",
                       "fused_hbm_frac": round(f_gbs / hbm, 4),
                       "split_allocate_ms": round(a_ms, 5), "split_integrate_ms": round(b_ms, 5),
                       "split_allocate_hbm_frac": round(a_gbs / hbm, 4),
                       "split_integrate_hbm_frac": round(b_gbs / hbm, 4),
                       "split_pts_per_s": round(mean("points") / ((a_ms + b_ms) / 1e3), 1),
                       "step_ms_p50": round(float(np.percentile(step_ms, 50)), 5),
                       "step_ms_p95": round(float(np.percentile(step_ms, 95)), 5),
                       "step_ms_p99": round(float(np.percentile(step_ms, 99)), 5),
                       "step_ms_max": round(float(np.max(step_ms)), 5),
                       "steps_over_2x_median": int(np.sum(np.array(step_ms) >
                                                          2 * np.median(step_ms))),
                       "blocks_per_frame": mean("blocks"), "voxels_per_frame": mean("voxels")},
            "roofline": roof,
            "paper_protocol_timing": amortized,
            "e2e": e2e,
            "autotune_frame": tuning,
            "extraction": extraction,
            **extra,
            "gpu_launches": int(launches),
            "gpu_launches_detail": "per step: the fusion kernel(s) inside the step events, plus "
                                   "1 reset kernel between steps, outside them",
            "clocks": clk.summary(),
            "wall_s_timed_region": round(wall, 4),
            "kernel_source": kernel_source_hash(),
            "paper_context": PAPER_CONTEXT,
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
            if not args.headline_only:
                try:
                    out["cpu_baseline"]["multicore"] = cpu_baseline_multicore(
                        args.cpu_seconds)
                except Exception as e:  # noqa: BLE001
                    out["cpu_baseline"]["multicore"] = {"error": repr(e)}
    return out


def run_amortized(torch, tsdf, spec, frames, dev, structs, stream, flush, scrub):
    """The paper's own timing protocol on the same frames (its Section 4): K =
    20 launches per event window, each frame into its own freshly reset
    volume (distinct volumes, so no launch finds the blocks of the one
    before), L2 scrubbed before each window but not between the launches in
    it; three passes of 10 windows, with each pass's median, p95 and p99 per
    launch. A secondary number: the headline times every launch alone, from
    a cold L2."""
    K, WINDOWS, PASSES = 20, 10, 3
    sp = stream.cuda_stream
    vols = []
    try:
        for _ in range(K):
            vols.append(tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots,
                                    spec.pool_blocks))
        passes = []
        window_points = 0
        for p in range(PASSES):
            per_launch = []
            for w in range(WINDOWS):
                for v in vols:
                    assert v.reset(sp) == "OK"
                with torch.cuda.stream(stream):
                    l2_scrub(flush, scrub, w)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                window_points = 0
                e0.record(stream)
                for j, v in enumerate(vols):
                    i = j % len(frames)
                    d, c = dev[i]
                    intr, pose = structs[i]
                    assert tsdf.tsdf_fuse_frame_async(v.handle, d, 640, 480, intr, pose, c,
                                                      sp) == "OK"
                    window_points += frames[i].valid_points
                e1.record(stream)
                stream.synchronize()
                per_launch.append(e0.elapsed_time(e1) / K)
            for v in vols:
                assert v.status(sp) == "OK"
            passes.append({"median_ms": round(float(np.median(per_launch)), 5),
                           "p95_ms": round(float(np.percentile(per_launch, 95)), 5),
                           "p99_ms": round(float(np.percentile(per_launch, 99)), 5)})
        med = float(np.median([x["median_ms"] for x in passes]))
        return {"protocol": f"{K} launches per event window into {K} distinct reset volumes, "
                            f"L2 scrubbed before each window, {WINDOWS} windows x {PASSES} passes",
                "passes": passes, "pts_per_s": round(window_points / K / (med / 1e3), 1)}
    finally:
        for v in vols:
            v.close()


def run_extraction(args, vol, frames, dev, tsdf, sp, hbm):
    """Marching tetrahedra over the bench frames fused into one volume:
    kernel time and device-to-host copy time of the triangle soup, medians
    of 10 calls through tsdf_extract_mesh."""
    W, H = 640, 480
    assert vol.reset(sp) == "OK"
    for f, (d, c) in zip(frames, dev):
        assert tsdf.tsdf_fuse_frame(vol.handle, d, W, H, f.intr, f.pose, c, sp) == "OK"
    blocks = vol.block_count(sp)
    runs = [vol.extract_mesh(sp, cells=False) for _ in range(11)][1:]
    n = len(runs[0][0])
    comp = float(np.median([r[2]["compute_ms"] for r in runs]))
    d2h = float(np.median([r[2]["d2h_ms"] for r in runs]))
    nbytes = runs[0][2]["d2h_bytes"]
    # algorithmic bytes: the {tsdf, weight} sums of every allocated voxel read
    # once (16-byte records), the triangles written once
    alg = blocks * 512 * 16 + n * 36
    return {"frames_fused": len(frames), "blocks": blocks, "triangles": n,
            "compute_ms": round(comp, 4), "d2h_ms": round(d2h, 4),
            "d2h_bytes": nbytes, "d2h_gbs": round(nbytes / (d2h * 1e6), 1) if d2h else None,
            "kernel_algorithmic_bytes": alg,
            "kernel_hbm_frac": round(alg / (comp * 1e6) / hbm, 4),
            "call": "tsdf_extract_mesh (triangles only, pageable host buffer)"}


def run_extraction_only(args):
    import torch
    from paper_2608_08287_gb300 import synth, tsdf
    from paper_2608_08287_gb300.build import build_library
    build_library()
    spec = synth.ROOM_640
    frames = make_frames(0)
    vol = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    stream = torch.cuda.Stream()
    dev = [(torch.from_numpy(f.depth).cuda(), torch.from_numpy(f.rgb).cuda()) for f in frames]
    hbm, _ = peaks()
    out = run_extraction(args, vol, frames, dev, tsdf, stream.cuda_stream, hbm)
    vol.close()
    return {"extraction": out}


E2E_STREAM = 16  # frames per streaming call, each into its own volume


def run_e2e(args, vol, frames, torch, tsdf, sp, stream, flush, scrub, world=1):
    """Same metric end to end through the public C ABI with host buffers.

    Headline: tsdf_fuse_frames_host, the streaming call. Each call takes
    E2E_STREAM frames from pinned host memory (the bench frames in turn), each
    into its own freshly reset volume, as the device-timed steps do; inside
    the call every frame's depth and colour are copied in (overlapping the
    previous frame's kernel), fused, and its status word read back. Timed on
    the host around each call; volumes reset and L2 scrubbed before each call,
    outside the timing.
    Also reported: tsdf_fuse_frame_host, one frame per call (copy in, fuse,
    status read back, all in series)."""
    from paper_2608_08287_gb300 import synth
    spec = synth.ROOM_640
    host = [(torch.from_numpy(f.depth).pin_memory(), torch.from_numpy(f.rgb).pin_memory())
            for f in frames]
    W, H = 640, 480
    structs = [(tsdf.intrinsics(f.intr), tsdf.pose_struct(f.pose)) for f in frames]
    vols = [vol] + [tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots,
                                spec.pool_blocks) for _ in range(E2E_STREAM - 1)]
    calls = max(1, args.steps // E2E_STREAM)

    def items(c):
        out = []
        for j in range(E2E_STREAM):
            i = (c * E2E_STREAM + j) % len(frames)
            out.append((vols[j].handle, host[i][0], host[i][1], structs[i][0], structs[i][1]))
        return out

    arrays = [tsdf.make_host_frames(items(c)) for c in range(min(calls, len(frames)))]
    for c in range(max(1, args.warmup)):
        for v in vols:
            v.reset(sp)
        st, per = tsdf.tsdf_fuse_frames_host(arrays[c % len(arrays)], stream=sp)
        assert st == "OK", per
    total = 0.0
    points = 0
    for c in range(calls):
        for v in vols:
            v.reset(sp)
        with torch.cuda.stream(stream):
            l2_scrub(flush, scrub, c)
        stream.synchronize()
        t0 = time.perf_counter()
        st, per = tsdf.tsdf_fuse_frames_host(arrays[c % len(arrays)], stream=sp)
        total += time.perf_counter() - t0
        assert st == "OK", per
        points += sum(frames[(c * E2E_STREAM + j) % len(frames)].valid_points
                      for j in range(E2E_STREAM))
    for v in vols[1:]:
        v.close()

    # one frame per call, all in series
    one_total = 0.0
    one_points = 0
    for i in range(max(1, args.warmup)):
        vol.reset(sp)
        assert tsdf.tsdf_fuse_frame_host(vol.handle, host[i % len(frames)][0], W, H,
                                         structs[i % len(frames)][0],
                                         structs[i % len(frames)][1],
                                         host[i % len(frames)][1], sp) == "OK"
    for i in range(min(args.steps, 100)):
        f = frames[i % len(frames)]
        d, c = host[i % len(frames)]
        intr, pose = structs[i % len(frames)]
        vol.reset(sp)
        with torch.cuda.stream(stream):
            l2_scrub(flush, scrub, i)
        stream.synchronize()
        t0 = time.perf_counter()
        st = tsdf.tsdf_fuse_frame_host(vol.handle, d, W, H, intr, pose, c, sp)
        one_total += time.perf_counter() - t0
        assert st == "OK", st
        one_points += f.valid_points
    points, total = reduce_job(points, total, world, "cuda")
    one_points, one_total = reduce_job(one_points, one_total, world, "cuda")
    return {"value": round(points / total, 1), "unit": UNIT,
            "h2d_bytes_per_step": W * H * 4 + W * H * 3, "d2h_bytes_per_step": 4,
            "call": f"tsdf_fuse_frames_host, {E2E_STREAM} frames per call from pinned host "
                    "memory, each into its own reset volume; per frame: depth + colour in, "
                    "status word out",
            "l2": "scrubbed before each call; frames within a call run back to back",
            "single_frame_call": {
                "value": round(one_points / one_total, 1), "unit": UNIT,
                "h2d_bytes_per_step": W * H * 4 + W * H * 3, "d2h_bytes_per_step": 8,
                "call": "tsdf_fuse_frame_host (pinned host depth+rgb in, status words out)"}}


def run_batched(args, torch, tsdf, serving, bank):
    """Config-4 style: 64 sessions (mixed 160x120 / 320x240 / 640x480, tables
    2^16..2^20), one frame each per step into fresh volumes, as one batch call
    -- its default form, one launch per frame over the batch's 8 streams, and
    its persistent form, one launch for all frames replayed from a CUDA graph
    -- against a loop of per-frame launches on one stream. Device time per
    step, L2 scrubbed between steps."""
    n = BATCH_SESSIONS
    res = batch_resolutions(n)
    vols = []
    for r in res:
        sp = serving.SESSION_CLASSES[r]
        vols.append(tsdf.Volume(sp.voxel_size, sp.truncation, sp.table_slots, sp.pool_blocks))
    stream = torch.cuda.Stream()
    sp_ = stream.cuda_stream
    dev = []
    for i, r in enumerate(res):
        depth_h, rgb_h, intr, pose, pts = bank.get(r, i)
        dev.append((depth_h.cuda(), rgb_h.cuda(), intr, pose, pts))
    points = sum(x[4] for x in dev)
    batch = tsdf.Batch(n, use_graph=1)                          # per-frame launches, 8 streams
    batch_p = tsdf.Batch(n, use_graph=1, batch_streams=0)       # one persistent launch (graph)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    scrub = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    items = [(v, d, c, intr, pose) for v, (d, c, intr, pose, _) in zip(vols, dev)]

    def prep(i):
        for v in vols:
            v.reset(sp_)
        with torch.cuda.stream(stream):
            l2_scrub(flush, scrub, i)

    def timed(fn, steps):
        out = []
        for i in range(steps):
            prep(i)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            stream.synchronize()
            out.append(a.elapsed_time(b))
        return out

    def batched():
        assert batch.fuse_async(items, stream=sp_) == "OK"

    def persistent():
        assert batch_p.fuse_async(items, stream=sp_) == "OK"

    def per_frame():
        for v, d, c, intr, pose in items:
            assert tsdf.tsdf_fuse_frame_async(v.handle, d, d.shape[1], d.shape[0], intr, pose,
                                              c, sp_) == "OK"

    timed(batched, 3)
    tb = timed(batched, args.batch_steps)
    st, _ = batch.status(n, stream=sp_)
    assert st == "OK", st
    timed(persistent, 3)
    tpers = timed(persistent, args.batch_steps)
    st, _ = batch_p.status(n, stream=sp_)
    assert st == "OK", st
    batch_p.close()
    timed(per_frame, 3)
    tp = timed(per_frame, args.batch_steps)
    for v in vols:
        assert v.status(sp_) == "OK"

    # the two-stage batched path, each stage timed on its own: stage A (tile
    # allocator) for all 64 frames, then stage B (per-thread scatter), in the
    # persistent form (one launch each, replayed from its own graph) and in
    # the per-frame form (one launch per frame and stage over 8 streams)
    def stage_times(streams):
        batch_a = tsdf.Batch(n, use_graph=1, fuse_mode=0, allocate_mode=1, integrate_mode=0,
                             batch_stages=1, batch_streams=streams)
        batch_b = tsdf.Batch(n, use_graph=1, fuse_mode=0, allocate_mode=1, integrate_mode=0,
                             batch_stages=2, batch_streams=streams)
        ta, tb2 = [], []
        for i in range(3 + args.batch_steps):
            prep(i)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            assert batch_a.fuse_async(items, stream=sp_) == "OK"
            ev[1].record(stream)
            assert batch_b.fuse_async(items, stream=sp_) == "OK"
            ev[2].record(stream)
            stream.synchronize()
            if i >= 3:
                ta.append(ev[0].elapsed_time(ev[1]))
                tb2.append(ev[1].elapsed_time(ev[2]))
        st_, _ = batch_b.status(n, stream=sp_)
        assert st_ == "OK", st_
        batch_a.close()
        batch_b.close()
        return ta, tb2

    ta_, tb_ = stage_times(0)
    ta_l, tb_l = stage_times(8)
    # algorithmic bytes of the batch from the oracle's work counts of its frames
    wk = oracle_work_counts([(d.numpy(), c.numpy(), np.array([intr.fx, intr.fy, intr.cx, intr.cy],
                                                              np.float32),
                              np.array(pose.m, np.float32).reshape(4, 4),
                              serving.SESSION_CLASSES[r])
                             for (d, c, intr, pose, _), r in
                             ((bank.get(r, i), r) for i, r in enumerate(res))], None)
    sums = [sum(x) for x in zip(*[stage_bytes(w) for w in wk])]
    hbm, peak_kind = peaks()
    sa_ms, sb_ms = float(np.mean(ta_)), float(np.mean(tb_))
    stage_rooflines = {
        "peak_gbs": hbm, "peak_kind": f"{peak_kind} hbm_gbs",
        "work_counts": "oracle, each frame into an empty volume",
        "stage_a": {"kernel": "batch_tile_allocate_kernel", "ms": round(sa_ms, 4),
                    "algorithmic_bytes": int(sums[0]),
                    "frac": round(sums[0] / (sa_ms * 1e6) / hbm, 4)},
        "stage_b": {"kernel": "batch_point_kernel (scatter)", "ms": round(sb_ms, 4),
                    "algorithmic_bytes": int(sums[1]),
                    "frac": round(sums[1] / (sb_ms * 1e6) / hbm, 4)},
        "two_stage_pts_per_s": round(points / ((sa_ms + sb_ms) / 1e3), 1),
        "two_stage_per_frame_pts_per_s": round(
            points / ((float(np.mean(ta_l)) + float(np.mean(tb_l))) / 1e3), 1),
        "stage_a_per_frame": {"kernel": "tile_allocate_kernel, one launch per frame over 8 streams",
                              "ms": round(float(np.mean(ta_l)), 4),
                              "algorithmic_bytes": int(sums[0]),
                              "frac": round(sums[0] / (float(np.mean(ta_l)) * 1e6) / hbm, 4)},
        "stage_b_per_frame": {"kernel": "integrate_scatter_kernel, one launch per frame over 8 "
                                        "streams",
                              "ms": round(float(np.mean(tb_l)), 4),
                              "algorithmic_bytes": int(sums[1]),
                              "frac": round(sums[1] / (float(np.mean(tb_l)) * 1e6) / hbm, 4)},
        "fused": {"kernel": "tile_fused_kernel, one launch per frame over 8 streams (default)",
                  "ms": round(float(np.mean(tb)), 4), "algorithmic_bytes": int(sums[2]),
                  "frac": round(sums[2] / (float(np.mean(tb)) * 1e6) / hbm, 4)},
        "fused_persistent": {"kernel": "batch_tile_fused_kernel (one persistent launch)",
                             "ms": round(float(np.mean(tpers)), 4),
                             "algorithmic_bytes": int(sums[2]),
                             "frac": round(sums[2] / (float(np.mean(tpers)) * 1e6) / hbm, 4)}}
    # the batch autotuner on the same frames (volumes empty before and after)
    for v in vols:
        assert v.reset(sp_) == "OK"
    st, tuning = batch.autotune(items, reps=5, stream=sp_)
    assert st == "OK", st
    timed(batched, 3)
    tt = timed(batched, args.batch_steps)
    for v in vols:
        assert v.status(sp_) == "OK"
        v.close()
    batch.close()
    mb, mp_, mt = float(np.mean(tb)), float(np.mean(tp)), float(np.mean(tt))
    mpers = float(np.mean(tpers))
    return {"sessions": n, "points_per_step": int(points),
            "batched_pts_per_s": round(points / (mb / 1e3), 1), "batched_ms_per_step": round(mb, 4),
            "batched_form": "default: one launch per frame, largest first, over 8 streams",
            "persistent_pts_per_s": round(points / (mpers / 1e3), 1),
            "persistent_ms_per_step": round(mpers, 4),
            "per_frame_pts_per_s": round(points / (mp_ / 1e3), 1),
            "per_frame_ms_per_step": round(mp_, 4),
            "autotuned_pts_per_s": round(points / (mt / 1e3), 1),
            "autotuned_ms_per_step": round(mt, 4), "autotuned_config": tuning,
            "launches_per_step": {"batched": n, "persistent": 1, "per_frame": n},
            "stage_rooflines": stage_rooflines,
            "steps": args.batch_steps, "graph": "persistent form only"}


def run_serving(args, torch, serving, bank):
    """Config-5 style: 256 sessions, Poisson arrivals at 30 fps each, 10 s
    window, volumes admitted by memory; continuous batching against per-frame
    launches on the same schedule, at the nominal rate and with arrivals
    compressed by each factor in args.serve_stress. Latency = completion - arrival."""
    free, _ = torch.cuda.mem_get_info()
    budget = min(0.7 * free, 200e9)
    plans = serving.plan_sessions(args.serve_sessions, window=args.serve_window,
                                  budget_bytes=budget)
    admitted = [p for p in plans if len(p.arrivals)]
    waits = np.array([p.admit - p.request for p in admitted])
    out = {"sessions": len(plans), "window_s": args.serve_window,
           "budget_gb": round(budget / 1e9, 1),
           "admission_wait_ms_p50": round(float(np.percentile(waits, 50)) * 1e3, 2),
           "admission_wait_ms_p99": round(float(np.percentile(waits, 99)) * 1e3, 2),
           "frames_offered": int(sum(len(p.arrivals) for p in admitted))}
    out["server"] = "tsdf_server (native continuous batching) vs one launch per frame"
    out["repeats"] = args.serve_repeats
    out["max_inflight"] = args.serve_inflight
    speeds = [1.0] + [float(x) for x in str(args.serve_stress).split(",") if x]
    # warm-up, not recorded: the whole schedule once at the highest rate for
    # each server, so every kernel the servers launch is loaded (lazily, on
    # first use) before the measured runs
    for mode in (0, 1):
        serving.native_replay(torch, bank, plans, mode, speed=max(speeds),
                              max_inflight=args.serve_inflight)
        torch.cuda.synchronize()
    out["warmup"] = f"one unrecorded replay per server at {max(speeds):g}x"
    for speed in speeds:
        into = out if speed == 1.0 else out.setdefault(f"stress_{speed:g}x", {})
        runs = {"batched": [], "per_frame": []}
        for rep in range(args.serve_repeats):
            # the two servers alternate, so drifts of the box hit both alike
            for name, mode in (("batched", 0), ("per_frame", 1)):
                res, st, _ = serving.native_replay(torch, bank, plans, mode, speed=speed,
                                                   max_inflight=args.serve_inflight)
                torch.cuda.synchronize()
                summ = res.summary()
                summ["status"] = st
                runs[name].append(summ)
        for name, rs in runs.items():
            # the median run by p99 is reported whole; the spread over repeats beside it
            pick = sorted(rs, key=lambda r: r["p99_ms"])[len(rs) // 2]
            into[name] = dict(pick)
            into[name]["repeats"] = {k: [r[k] for r in rs]
                                     for k in ("p50_ms", "p99_ms", "frames_per_s")}
    return out


def run_small_frames(args, torch, tsdf):
    """Frames too small to fill the GPU with one thread per point: the
    160x120 plane-and-sphere frame (voxel 1 cm, truncation 4 cm, 2^16 slots,
    pool 2^14) and a 320x240 room frame (1 cm / 4 cm, 2^18 slots, pool 2^16),
    each fused into an empty volume by the fused tile kernel with the threads
    per point chosen per frame (the default) and set to 1, 2, 4 and 8, and
    what tsdf_autotune_frame picks. Device time per
    step (CUDA events), L2 scrubbed and volume reset between steps."""
    from paper_2608_08287_gb300 import synth
    cases = [("plane_sphere_160x120", synth.plane_sphere_frame(), synth.PLANE_SPHERE_160),
             ("room_320x240", synth.room_frame(12, width=320, height=240),
              synth.VolumeSpec(0.01, 0.04, 1 << 18, 1 << 16))]
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    scrub = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    steps = max(20, args.small_steps)
    out = {"timed": f"median of {steps} steps after 5 warm-up, L2 scrubbed, empty volume"}
    for name, f, spec in cases:
        d = torch.from_numpy(f.depth).cuda()
        c = torch.from_numpy(f.rgb).cuda()
        intr, pose = tsdf.intrinsics(f.intr), tsdf.pose_struct(f.pose)
        vol = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
        row = {"points": int(f.valid_points)}
        for tpp in (0, 1, 2, 4, 8):
            assert vol.set_option("threads_per_point", tpp) == "OK"
            ms = []
            for i in range(5 + steps):
                vol.reset(sp)
                with torch.cuda.stream(stream):
                    l2_scrub(flush, scrub, i)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                assert tsdf.tsdf_fuse_frame_async(vol.handle, d, f.depth.shape[1],
                                                  f.depth.shape[0], intr, pose, c, sp) == "OK"
                e1.record(stream)
                stream.synchronize()
                if i >= 5:
                    ms.append(e0.elapsed_time(e1))
            assert vol.status(sp) == "OK"
            med = float(np.median(ms))
            name_t = f"tpp{tpp}" if tpp else "tpp_auto"
            row[f"{name_t}_ms"] = round(med, 5)
            row[f"{name_t}_pts_per_s"] = round(f.valid_points / (med / 1e3), 1)
        assert vol.set_option("threads_per_point", 0) == "OK"
        assert vol.reset(sp) == "OK"
        st, tuning = vol.autotune(d, f.intr, f.pose, c, reps=10, stream=sp)
        assert st == "OK", st
        row["autotune"] = {k: tuning[k] for k in ("fuse_mode", "probe_load", "threads_per_point",
                                                  "best_ms", "default_ms", "candidates")}
        vol.close()
        out[name] = row
    del flush, scrub
    return out


SWEEP_LOADS = (0.1, 0.3, 0.5, 0.7, 0.9)
SWEEP_SLOTS = 1 << 17
SWEEP_BOUND = 8        # the trip count of the printed bounded probe (Section 7)


def run_load_sweep(args, torch, tsdf, rendered):
    """Load-factor sweep up to 0.9 with the table decoupled from the block
    count (Section 8's open question: where probe chains really lengthen).
    The room orbit (640x480, 5 mm voxels, 2 cm truncation) is fused frame by
    frame into a volume whose table and pool both hold 2^17 blocks. When the
    load first passes each target, the volume is snapshotted and the NEXT
    frame's fusion is timed from that snapshot (restored before every
    repetition, outside the events; L2 scrubbed) for each strategy, beside
    the table's probe lengths and what a probe bounded at 8 (fed the same
    frames from the start) has silently lost by then."""
    from paper_2608_08287_gb300 import synth
    spec = synth.VolumeSpec(0.005, 0.02, SWEEP_SLOTS, SWEEP_SLOTS)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    frames = [(torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda(), tsdf.intrinsics(i),
               tsdf.pose_struct(p), int(np.count_nonzero(d > 0))) for d, c, i, p in rendered]

    def vol(**opts):
        v = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
        for k, x in opts.items():
            assert v.set_option(k, x) == "OK"
        return v

    fill, snap, work = vol(), vol(), vol()
    kfill, ksnap, kwork = vol(slot_index=1), vol(slot_index=1), vol(slot_index=1)
    bfill = vol(probe_bound=SWEEP_BOUND, fuse_mode=0, allocate_mode=0, integrate_mode=0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    scrub = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    variants = (("fused_tile", work, snap, dict(fuse_mode=2)),
                ("tile+scatter", work, snap, dict(allocate_mode=1, integrate_mode=0, fuse_mode=0)),
                ("tile+tile", work, snap, dict(allocate_mode=1, integrate_mode=2, fuse_mode=0)),
                ("paper_protocol", work, snap, dict(allocate_mode=0, integrate_mode=0, fuse_mode=0)),
                ("fused_warp", work, snap, dict(fuse_mode=1)),
                ("slot_index", kwork, ksnap, dict(fuse_mode=2)))

    def fuse(v, fr):
        d, c, intr, pose, _ = fr
        assert tsdf.tsdf_fuse_frame_async(v.handle, d, 640, 480, intr, pose, c, sp) == "OK"

    def time_next(name, w, src, opts, fr):
        for k, x in opts.items():
            assert w.set_option(k, x) == "OK"
        d, c, intr, pose, _ = fr
        ta, tb = [], []
        for r in range(3 + args.sweep_reps):
            assert w.copy_from(src, sp) == "OK"
            with torch.cuda.stream(stream):
                l2_scrub(flush, scrub, r)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            if opts.get("fuse_mode", 0):
                assert tsdf.tsdf_fuse_frame_async(w.handle, d, 640, 480, intr, pose, c, sp) == "OK"
                ev[1].record(stream)
            else:
                assert tsdf.tsdf_allocate_async(w.handle, d, 640, 480, intr, pose, sp) == "OK"
                ev[1].record(stream)
                assert tsdf.tsdf_integrate_async(w.handle, d, 640, 480, intr, pose, c, sp) == "OK"
            ev[2].record(stream)
            stream.synchronize()
            if r >= 3:
                ta.append(ev[0].elapsed_time(ev[1]))
                tb.append(ev[1].elapsed_time(ev[2]))
        assert w.status(sp) == "OK", name
        total = float(np.median(np.add(ta, tb)))
        out = {"ms": round(total, 4), "pts_per_s": round(fr[4] / (total / 1e3), 1),
               "blocks_after": w.block_count(sp)}
        if not opts.get("fuse_mode", 0):
            out["allocate_ms"] = round(float(np.median(ta)), 4)
            out["integrate_ms"] = round(float(np.median(tb)), 4)
        return out

    points = []
    targets = list(SWEEP_LOADS)
    for k in range(len(frames) - 1):
        if not targets:
            break
        for v in (fill, kfill, bfill):
            fuse(v, frames[k])
        n = fill.block_count(sp)
        if n < targets[0] * SWEEP_SLOTS:
            continue
        while targets and n >= targets[0] * SWEEP_SLOTS:
            targets.pop(0)
        assert fill.status(sp) == kfill.status(sp) == bfill.status(sp) == "OK"
        st, bst = fill.table_stats(sp), bfill.table_stats(sp)
        assert kfill.block_count(sp) == n
        assert snap.copy_from(fill, sp) == "OK" and ksnap.copy_from(kfill, sp) == "OK"
        row = {"frame": k, "blocks": n, "load": round(n / SWEEP_SLOTS, 4),
               "probe_mean": round(st["probe_sum"] / max(1, st["occupied_slots"]), 2),
               "probe_max": st["probe_max"],
               f"bounded{SWEEP_BOUND}": {
                   "status": bfill.status(sp),
                   "blocks_lost": n - bst["blocks"],
                   "contributions_lost": st["weight_sum"] - bst["weight_sum"],
                   "contributions": st["weight_sum"]},
               "next_frame_points": frames[k + 1][4]}
        timings = {name: time_next(name, w, src, opts, frames[k + 1])
                   for name, w, src, opts in variants}
        after = {t["blocks_after"] for t in timings.values()}
        assert len(after) == 1, timings   # every strategy allocates the same blocks
        row["timings"] = timings
        points.append(row)
    for v in (fill, snap, work, kfill, ksnap, kwork, bfill):
        v.close()
    return {"workload": "room orbit 640x480, voxel 5 mm, truncation 2 cm, "
                        "table 2^17 slots, pool 2^17 blocks",
            "timed": "fusion of the frame after the checkpoint, from a restored snapshot, "
                     f"median of {args.sweep_reps}, L2 scrubbed",
            "points": points}


PROBE_CASE_LOADS = (0.1, 0.9)


BATCH_CASE_SESSIONS = 16
BATCH_CASE_POOL = 1 << 13


def run_batch_profile_case(args):
    """The batched fused kernel on a case small enough for an ncu capture of
    all its sections: 16 sessions, alternately 320x240 and 160x120 room frames
    of the session classes (the 640x480 class is left out), each into its own
    empty volume with its class's table and a pool of 2^13 blocks (more than a
    frame of these classes touches), so the device holds about 1.5 GB. The
    3,040 tiles are at least the 2,048 a batch needs to replay its CUDA graph
    of the persistent launch, the configuration the 64-session workload runs.
    Each rep resets the volumes and scrubs L2 outside the CUDA events around
    the batch; with --batch-case-reps 0 there is one warm-up batch and one
    more, with no scrub (for ncu -s 1 -c 1, which flushes caches itself)."""
    import torch
    from paper_2608_08287_gb300 import serving, synth, tsdf
    from paper_2608_08287_gb300.build import build_library
    build_library()
    torch.cuda.set_device(0)
    classes = [(320, 240), (160, 120)]
    sess = []
    for i in range(BATCH_CASE_SESSIONS):
        w, h = classes[i % 2]
        cs = serving.SESSION_CLASSES[(w, h)]
        spec = synth.VolumeSpec(cs.voxel_size, cs.truncation, cs.table_slots, BATCH_CASE_POOL)
        sess.append((spec, synth.room_frame(12 * (i % 24), width=w, height=h)))
    work = oracle_work_counts([(f.depth, f.rgb, np.asarray(f.intr, np.float32),
                                np.asarray(f.pose, np.float32), sp) for sp, f in sess], None)
    sums = [sum(x) for x in zip(*[stage_bytes(wk) for wk in work])]
    points = sum(wk["points"] for wk in work)
    stream = torch.cuda.Stream()
    sp_ = stream.cuda_stream
    vols = [tsdf.Volume(sp.voxel_size, sp.truncation, sp.table_slots, sp.pool_blocks)
            for sp, _ in sess]
    dev = [(torch.from_numpy(f.depth).cuda(), torch.from_numpy(f.rgb).cuda()) for _, f in sess]
    items = [(v, d, c, f.intr, f.pose) for v, (d, c), (_, f) in zip(vols, dev, sess)]
    # the persistent form by default; --batch-case-streams k > 0 takes the
    # per-frame form over k streams
    batch = tsdf.Batch(len(sess), use_graph=1, batch_streams=args.batch_case_streams)
    reps = args.batch_case_reps
    flush = scrub = None
    if reps > 0:
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        scrub = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    times = []
    for i in range(1 + max(reps, 1)):
        for v in vols:
            assert v.reset(sp_) == "OK"
        if flush is not None:
            with torch.cuda.stream(stream):
                l2_scrub(flush, scrub, i)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        assert batch.fuse_async(items, stream=sp_) == "OK"
        b.record(stream)
        stream.synchronize()
        if i >= 1:
            times.append(a.elapsed_time(b))
    st, _ = batch.status(len(sess), stream=sp_)
    assert st == "OK", st
    counts_match = all(v.block_count(sp_) == wk["blocks"] for v, wk in zip(vols, work))
    batch.close()
    for v in vols:
        v.close()
    ms = float(np.median(times))
    hbm, peak_kind = peaks()
    return {"case": ("batch_tile_fused_kernel" if args.batch_case_streams == 0 else
                     f"tile_fused_kernel per frame over {args.batch_case_streams} streams") +
                    ", 16 sessions (8 x 320x240, 8 x 160x120 room frames), each into an "
                    "empty volume",
            "tiles": sum(((w + 15) // 16) * ((h + 15) // 16) for w, h in
                         (classes[i % 2] for i in range(BATCH_CASE_SESSIONS))),
            "points": int(points), "reps": reps, "ms_median": round(ms, 4),
            "pts_per_s": round(points / (ms / 1e3), 1),
            "algorithmic_bytes": int(sums[2]), "peak_gbs": hbm, "peak_kind": peak_kind,
            "frac": round(sums[2] / (ms * 1e6) / hbm, 4),
            "gpu_block_counts_match_oracle": bool(counts_match)}


def run_probe_policy_case(args):
    """The probe-load policy case (Section 6.2: whether a probe read is kept in
    L1 decided speed there). The room orbit (640x480) is fused into a table
    and pool of 2^17 blocks, with stage A and stage B as separate kernels of
    the paper's own strategies (so no launch of the kernels below happens
    while it fills). When the load first passes 0.1 and 0.9 the volume is
    snapshotted. Then, at each load and for each probe-load policy (L1-cached,
    L2-only, relaxed atomic), the next frame is fused from the snapshot by the
    fused tile kernel, and allocated by the tile allocator of stage A: twelve
    launches, each timed with CUDA events (median of --probe-case-reps, L2
    scrubbed), in the order an ncu capture with -k and -c 12 sees them when
    --probe-case-reps is 0 (one launch each, no scrub: ncu flushes the caches
    itself). The snapshots are checkpoints in host memory, restored before
    every launch, so the device holds a single volume."""
    import multiprocessing as mp
    import torch
    from paper_2608_08287_gb300 import serving, synth, tsdf
    from paper_2608_08287_gb300.build import build_library
    build_library()
    torch.cuda.set_device(0)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        rendered = pool.starmap(serving._render, [(640, 480, k) for k in range(args.sweep_frames)])
    spec = synth.VolumeSpec(0.005, 0.02, SWEEP_SLOTS, SWEEP_SLOTS)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream

    def vol(**opts):
        v = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
        for k, x in opts.items():
            assert v.set_option(k, x) == "OK"
        return v

    # snapshots are kept in host memory (checkpoints), so that the device holds
    # one volume while the kernels below run (an ncu capture saves and
    # restores device memory around its passes)
    fill = vol(fuse_mode=0, allocate_mode=0, integrate_mode=0)
    snaps = {}
    targets = list(PROBE_CASE_LOADS)
    for k, (d, c, intr, pose) in enumerate(rendered[:-1]):
        dd, cc = torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda()
        assert tsdf.tsdf_fuse_frame(fill.handle, dd, 640, 480, intr, pose, cc, sp) == "OK"
        n = fill.block_count(sp)
        while targets and n >= targets[0] * SWEEP_SLOTS:
            st_, snap = fill.save(sp)
            assert st_ == "OK"
            st = fill.table_stats(sp)
            snaps[targets.pop(0)] = (snap, k + 1, {
                "blocks": n, "load": round(n / SWEEP_SLOTS, 4),
                "probe_mean": round(st["probe_sum"] / max(1, st["occupied_slots"]), 2),
                "probe_max": st["probe_max"]})
        if not targets:
            break
    fill.close()
    del fill
    torch.cuda.empty_cache()
    work = vol()
    flush = scrub = None
    if args.probe_case_reps > 0:
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        scrub = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {"workload": "room orbit 640x480, voxel 5 mm, truncation 2 cm, table 2^17 slots, "
                       "pool 2^17 blocks; the next frame after each snapshot",
           "policies": {"0": "ld.global.ca (L1-cached)", "1": "ld.global.cg (L2 only)",
                        "2": "ld.relaxed.gpu (scoped atomic load)"},
           "launch_order": "for each load: for each policy: fused tile kernel, then tile "
                           "allocator", "loads": []}
    for load in PROBE_CASE_LOADS:
        if load not in snaps:
            out["loads"].append({"target": load, "error": "not reached"})
            continue
        snap, nxt, info = snaps[load]
        d, c, intr, pose = rendered[nxt]
        dd, cc = torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda()
        row = dict(info, target=load, frame=nxt, policies={})
        for policy in (0, 1, 2):
            times = {}
            for name, opts in (("fused_tile", dict(fuse_mode=2, probe_load=policy)),
                               ("tile_allocate", dict(fuse_mode=0, allocate_mode=1,
                                                      probe_load=policy))):
                for k, x in opts.items():
                    assert work.set_option(k, x) == "OK"
                ts = []
                for r in range(max(1, args.probe_case_reps)):
                    assert work.load(snap, sp) == "OK"
                    stream.synchronize()   # the restore's copy ends before the events
                    if flush is not None:
                        with torch.cuda.stream(stream):
                            l2_scrub(flush, scrub, r)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    if name == "fused_tile":
                        assert tsdf.tsdf_fuse_frame_async(work.handle, dd, 640, 480, intr, pose,
                                                          cc, sp) == "OK"
                    else:
                        assert tsdf.tsdf_allocate_async(work.handle, dd, 640, 480, intr, pose,
                                                        sp) == "OK"
                    e1.record(stream)
                    stream.synchronize()
                    assert work.status(sp) == "OK"
                    ts.append(e0.elapsed_time(e1))
                times[name + "_ms"] = round(float(np.median(ts)), 4)
            row["policies"][str(policy)] = times
        out["loads"].append(row)
    return out


def oracle_work_counts(frames, spec):
    """The units of the algorithmic bytes for each frame, from the oracle:
    valid points, distinct blocks (U_b), new blocks (N_new) and distinct
    voxels (U_v), each frame fused into an empty volume (the CPU leg of the
    bench; computed before any timing). frames: synth frames, or tuples
    (depth, rgb, intr (4,), pose (4, 4), spec) each with its own volume spec."""
    import oracle
    out = []
    for f in frames:
        if isinstance(f, tuple):
            depth, rgb, intr, pose, sp = f
        else:
            depth, rgb, intr, pose, sp = f.depth, f.rgb, f.intr, f.pose, spec
        ov = oracle.OracleVolume(sp.voxel_size, sp.truncation, sp.table_slots, sp.pool_blocks)
        assert ov.fuse(depth, intr, pose, rgb) == "OK"
        st = ov.last_stats
        ov.close()
        out.append({"points": st["points"], "blocks": st["unique_blocks"],
                    "new_blocks": st["new_blocks"], "voxels": st["unique_voxels"],
                    "pixels": int(depth.shape[0] * depth.shape[1])})
    return out


def stage_bytes(w):
    """Section 8(d) algorithmic bytes of one frame's stage A, stage B and both
    stages fused, from its work counts (each frame into an empty volume)."""
    a = 4 * w["pixels"] + 16 * w["blocks"] + 28 * w["new_blocks"]
    b = 7 * w["pixels"] + 16 * w["blocks"] + 40 * w["voxels"]
    f = 7 * w["pixels"] + 16 * w["blocks"] + 28 * w["new_blocks"] + 40 * w["voxels"]
    return a, b, f


def cpu_baseline(seconds):
    """The oracle as it stands, single-threaded on a host core, on whole frames."""
    import oracle
    from paper_2608_08287_gb300 import synth
    spec = synth.ROOM_640
    frames = make_frames(0)       # the GPU arm's frames and config
    n = 0
    points = 0
    t0 = time.perf_counter()
    while True:
        f = frames[n % len(frames)]
        ov = oracle.OracleVolume(spec.voxel_size, spec.truncation, spec.table_slots,
                                 spec.pool_blocks)
        assert ov.fuse_frame(f) == "OK"
        ov.close()
        n += 1
        points += f.valid_points
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": round(points / el, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} whole 640x480 room frames into empty volumes, one thread"}


BATCH_SESSIONS = 64


def batch_resolutions(n=BATCH_SESSIONS):
    """The batched workload's per-session resolutions (seeded)."""
    from paper_2608_08287_gb300 import serving, synth
    u = synth.uniform(20261208, 1, n)
    return [list(serving.SESSION_CLASSES)[int(x * 3) % 3] for x in u]


def _oracle_sessions_worker(worker, cores, seconds):
    """One host core's share of the batched workload: sessions worker,
    worker + cores, ... each fuse their frame into a fresh oracle volume, in
    turn, until `seconds` have passed. Frames are rendered before the clock
    starts. Returns (points, frames, elapsed)."""
    import oracle
    from paper_2608_08287_gb300 import serving, synth
    res = batch_resolutions()
    mine = []
    for i in range(worker, len(res), cores):
        w, h = res[i]
        mine.append((serving.SESSION_CLASSES[res[i]], synth.room_frame(12 * (i % 24), width=w,
                                                                      height=h)))
    points = frames = 0
    t0 = time.perf_counter()
    while mine:
        spec, f = mine[frames % len(mine)]
        ov = oracle.OracleVolume(spec.voxel_size, spec.truncation, spec.table_slots,
                                 spec.pool_blocks)
        assert ov.fuse_frame(f) == "OK"
        ov.close()
        frames += 1
        points += f.valid_points
        if time.perf_counter() - t0 >= seconds:
            break
    return points, frames, time.perf_counter() - t0


def cpu_baseline_multicore(seconds):
    """One oracle instance per host core over the batched workload's sessions
    (independent volumes, so embarrassingly parallel): points of all cores over
    the slowest core's time. A process pool started with spawn."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_sessions_worker,
                           [(w, cores, seconds) for w in range(cores)])
    points = sum(r[0] for r in res)
    frames = sum(r[1] for r in res)
    el = max(r[2] for r in res)
    return {"value": round(points / el, 1), "unit": UNIT, "cores": cores,
            "kind": "oracle, one instance per core",
            "sample": f"{frames} frames of the {BATCH_SESSIONS}-session batched workload "
                      "(mixed 160x120 / 320x240 / 640x480 room frames), each into a fresh "
                      f"volume, about {seconds:g} s per core"}


def run_reference(args):
    """--impl reference: the CPU oracle timed on the same workload and metric."""
    import oracle
    from paper_2608_08287_gb300 import synth
    oracle.build()
    spec = synth.ROOM_640
    frames = make_frames(0)       # the GPU arm's frames and config

    def step(i):
        f = frames[i % len(frames)]
        ov = oracle.OracleVolume(spec.voxel_size, spec.truncation, spec.table_slots,
                                 spec.pool_blocks)
        assert ov.fuse_frame(f) == "OK"
        ov.close()
        return f.valid_points

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    points = sum(step(args.warmup + i) for i in range(args.steps))
    el = time.perf_counter() - t0
    value = points / el
    return {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": args.gpus,
            "device": "host CPU, one thread (the oracle; no GPU is used)",
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "impl": "reference", "config": config_dict(spec, frames),
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1,
                             "kind": "oracle",
                             "sample": f"{args.steps} whole 640x480 room frames, one thread"},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--probe-load", type=int, default=None)
    ap.add_argument("--integrate-mode", type=int, default=None)
    ap.add_argument("--allocate-mode", type=int, default=None)
    ap.add_argument("--fuse-mode", type=int, default=None)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the batched and serving measurements")
    ap.add_argument("--extraction-only", action="store_true",
                    help="only fuse the bench frames and time surface extraction "
                         "(a small command for profiling the extraction kernel)")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--clock-ms", type=int, default=100,
                    help="nvidia-smi sampling interval during the timed region")
    ap.add_argument("--serve-sessions", type=int, default=256)
    ap.add_argument("--serve-window", type=float, default=10.0)
    ap.add_argument("--serve-repeats", type=int, default=5,
                    help="runs of each server at each arrival rate (median reported, spread kept)")
    ap.add_argument("--serve-inflight", type=int, default=4,
                    help="launches in flight at most, for both servers")
    ap.add_argument("--serve-stress", default="3,10",
                    help="arrival-rate multiples of the further serving runs (comma-separated)")
    ap.add_argument("--bank-frames", type=int, default=24)
    ap.add_argument("--sweep-frames", type=int, default=142,
                    help="orbit frames rendered for the load-factor sweep (0 = no sweep)")
    ap.add_argument("--sweep-reps", type=int, default=10)
    ap.add_argument("--l2-fetch-bytes", type=int, default=0,
                    help="set the context's L2 fetch granularity (32, 64, 128) through "
                         "tsdf_set_l2_fetch_bytes before the run; 0 leaves the default")
    ap.add_argument("--probe-policy-case", action="store_true",
                    help="only the probe-load policy case: loads 0.1 and 0.9, three policies, "
                         "the fused tile kernel and the stage A tile allocator (a small command "
                         "for an ncu capture of the probe reads)")
    ap.add_argument("--probe-case-reps", type=int, default=5,
                    help="timed repetitions per launch of the probe-load policy case "
                         "(0: one launch each and no L2 scrub, for an ncu capture)")
    ap.add_argument("--batch-profile-case", action="store_true",
                    help="only the batched fused kernel on a 16-session case of about 1.5 GB "
                         "(a small command for an ncu capture of the batched kernel)")
    ap.add_argument("--batch-case-streams", type=int, default=0,
                    help="batch profile case: 0 = the persistent batched kernel, k > 0 = one "
                         "launch per frame over k streams")
    ap.add_argument("--batch-case-reps", type=int, default=20,
                    help="timed batches of the batch profile case (0: one batch after a "
                         "warm-up, no L2 scrub, for an ncu capture)")
    ap.add_argument("--small-steps", type=int, default=100,
                    help="timed steps per threads-per-point setting on the small frames")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if args.probe_policy_case:
        if rank == 0:
            print(json.dumps(run_probe_policy_case(args)), flush=True)
        return

    if args.batch_profile_case:
        if rank == 0:
            print(json.dumps(run_batch_profile_case(args)), flush=True)
        return

    if args.extraction_only:
        if rank == 0:
            print(json.dumps(run_extraction_only(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
