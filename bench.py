#!/usr/bin/env python
"""Benchmark: points clustered per second by FDbscan-DenseBox on 2^24 3D
cosmology-like points on one GB300 (plus the fraction of the HBM roofline).

One step is one complete dbscan_run (bounds, keys, radix sort, gather,
DenseBox cells, LBVH build and refit, union-find init, preprocessing, main
traversal with fused union-find, finalize and relabel) on device-resident
points; the output labels stay on the device.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
  python bench.py --mode batch   # one fused batch of 4096 instances vs one run each
  python bench.py --mode serve   # Poisson-arrival serving vs sequential runs
  python bench.py --mode sweep   # several minPts over one index vs one run each
  python bench.py --mode slabs   # slab-wise clustering of host points (out-of-core path)
With N > 1 it is launched by torch.distributed.run; each rank clusters its own
replica of the workload (replicas only: the method has no exchange step on
one node), and the value is the points of all ranks over the slowest rank's
time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "points clustered/sec (DenseBox, 16M 3D, 1 GB300)"
UNIT = "points/s"
FALLBACK_HBM_GBS = 6800.0


# ----------------------------------------------------------------- bytes model
def bytes_model(n: int, d: int, m: int, key_bytes: int, packed: bool = False) -> dict:
    """Compulsory device-memory traffic of each stage (each logical array read
    or written once per stage), in bytes per run. n points, d dims, m BVH
    leaves, key_bytes 8 (DenseBox cell keys) or 4 (FDbscan Morton codes);
    packed: DenseBox keys sorted as one 64-bit word with the point index,
    which the gather splits into permutation and keys."""
    kv = key_bytes + 4
    if packed:
        keys, sort, gather = 4 * d * n + 8 * n, 16 * n, 8 * n + 8 * d * n + 12 * n
    else:
        keys, sort, gather = 4 * d * n + kv * n, 2 * kv * n, 4 * n + 8 * d * n
    return {
        "bounds": 4 * d * n,                              # read coordinates
        "keys": keys,                                     # read coordinates, write key + index
        "sort": sort,                                     # read and write (key, index) once
        "gather": gather,                                 # read index and coordinates, write sorted coordinates
        "leaves": key_bytes * n + 5 * n + 8 * m,          # read keys, write flags, leaf records
        "lbvh": 4 * d * n + 8 * m + 64 * m + 64 * m,      # leaf boxes from points, keys, node records, refit
        "init": 5 * n,                                    # labels + core flags
        "preprocess": 4 * d * n + 64 * m + n,             # points once, tree once, core flags
        "main": 4 * d * n + 64 * m + n + 4 * n + 4 * n,   # points, tree, core flags, labels read and written
        "finalize": 8 * n + 8 * n,                        # labels + index read, output labels + core written
    }


TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traversal_traffic_densebox_halos.json")
STAGE_KERNELS = {"preprocess": ("k_pre", "k_list_claims"), "main": ("k_intra", "k_kinds_count", "k_kinds_write",
                                                                     "k_main")}


def measured_traffic(n: int, stage: str) -> float | None:
    """DRAM bytes (read + write) of one run of a traversal stage
    ("preprocess" or "main") on n points of the halo workload (DenseBox,
    minPts 10), from the committed ncu summary (bytes per point of the
    captured size, scaled by the points); None if the summary is missing or
    the sources have changed since it was taken."""
    try:
        with open(TRAFFIC_JSON) as f:
            t = json.load(f)
        if t["sources_sha256"] != sources_sha256(COUNT_SOURCES):
            return None
        return t["bytes_per_point"][stage] * n
    except Exception:
        return None


COUNTS_JSON = os.path.join(ROOT, "profiles", "traversal_counts_densebox_halos16m.json")
COUNT_SOURCES = [os.path.join(ROOT, "paper_2103_05162_gb300", "csrc", f)
                 for f in ("traverse.cu", "internal.cuh", "build.cuh", "build.cu", "capi.cu")]
PHASES = ("lists", "preprocess", "main")
KINDS = ("distance_tests", "box_tests", "node_visits_per_warp", "leaf_visits_per_warp")


def sources_sha256(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def fp32_ops(d: int, dist_tests: float, box_tests: float) -> float:
    """FP32 arithmetic of the tests (compares not counted): a distance test
    is d subtractions, d products and d-1 sums; a point- or box-to-box test
    is, per axis, two differences, two maxima and a product, then d-1 sums."""
    return dist_tests * (3 * d - 1) + box_tests * (5 * d + d - 1)


def traversal_counts(n: int) -> dict | None:
    """Counts per point of the traversal phases on the benchmark workload,
    from the committed counters run (None if missing, for another size, or
    taken on other sources)."""
    try:
        with open(COUNTS_JSON) as f:
            c = json.load(f)
        if c["n"] != n or c["sources_sha256"] != sources_sha256(COUNT_SOURCES):
            return None
        return c
    except Exception:
        return None


def measured_peak_hbm() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- workload
def workload(n: int, seed: int):
    """The 3D halo family; below 2^24 points the number of halos shrinks in
    proportion so that the halo size distribution is kept."""
    from workloads import halo_eps, halos
    n_halos = max(10, round(50000 * n / (1 << 24)))
    return halos(n, seed, n_halos=n_halos), halo_eps(n)


def workload_desc(n: int, eps: float, min_pts: int) -> str:
    return (f"halos3d: {n} 3D float32 points, 50k NFW halos (r_s=0.002, sizes ~s^-2 on [10,1e5]) "
            f"+ 30% uniform background in [0,1]^3, eps={eps:.6g} (0.2 x mean spacing), minPts={min_pts}, "
            f"DBSCAN mode, FDbscan-DenseBox")


def cpu_sample(X: np.ndarray, frac_side: float):
    """The points of the workload inside the cube [0, a)^3: the same density
    and structure on a bounded part of the volume."""
    sel = np.all(X < frac_side, axis=1)
    return np.ascontiguousarray(X[sel])


def time_oracle(W: np.ndarray, eps: float, min_pts: int) -> float:
    import oracle
    t = time.perf_counter()
    oracle.dbscan(W, eps, min_pts, 0)
    return time.perf_counter() - t


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x of all ranks (the slowest rank's time); x itself on one
    rank. device: where the reduction tensor lives (cuda for NCCL, cpu for
    gloo)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# -------------------------------------------------------------------- main arms
def run_reference(args, rank: int) -> None:
    """The oracle (plain single-threaded C) on the host cores, on a bounded
    sample of the same workload each step."""
    if rank != 0:
        return
    X, eps = workload(args.n, args.seed)
    W = cpu_sample(X, args.ref_side)
    for _ in range(args.warmup):
        time_oracle(W, eps, args.min_pts)
    ts = [time_oracle(W, eps, args.min_pts) for _ in range(args.steps)]
    tot = sum(ts)
    value = W.shape[0] * args.steps / tot
    sample = f"points of the workload inside [0,{args.ref_side})^3: {W.shape[0]} points, same eps/minPts"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc(args.n, eps, args.min_pts), "n": args.n, "min_pts": args.min_pts,
                   "eps": eps, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def timed_two_streams(gb, pts, eps, args, algo, labels, labels2, stream, s2, n, world, dev, barrier) -> dict:
    """The timed steps with two runs in flight (alternating streams)."""
    import torch
    u0 = torch.cuda.Event(enable_timing=True)
    u1 = torch.cuda.Event(enable_timing=True)
    u0.record(stream)
    s2.wait_event(u0)
    for i in range(args.steps):
        gb.dbscan_run(pts, eps, args.min_pts, mode=gb.MODE_DBSCAN, algo=algo,
                      labels_out=labels if i % 2 == 0 else labels2, stream=stream if i % 2 == 0 else s2)
    done2 = torch.cuda.Event()
    done2.record(s2)
    stream.wait_event(done2)
    u1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    gb.stream_status(stream)
    gb.stream_status(s2)
    ms2 = max_over_ranks(u0.elapsed_time(u1), world, dev)
    two_streams = {"value": n * world * args.steps / (ms2 / 1e3), "unit": UNIT,
                   "ms_per_step": ms2 / args.steps,
                   "how": f"{args.steps} steps alternating between 2 streams, device-resident inputs, CUDA events"}
    return two_streams


def run_gb300(args, rank: int, world: int) -> None:
    import torch
    import torch.distributed as dist

    import paper_2103_05162_gb300 as gb

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    gb.load()
    gb.set_tuning(args.block, args.cell_factor)
    if args.border_lists is not None:
        gb.set_border_lists(bool(args.border_lists))
    algo = gb.ALGO_DENSEBOX if args.algo == "densebox" else gb.ALGO_FDBSCAN
    X, eps = workload(args.n, args.seed + rank)
    n, d = X.shape
    pts = torch.from_numpy(X).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def step():
        gb.dbscan_run(pts, eps, args.min_pts, mode=gb.MODE_DBSCAN, algo=algo, labels_out=labels, stream=stream)

    for _ in range(args.warmup):
        step()  # (the first call of this kind runs the autotuner)
    torch.cuda.synchronize(dev)
    stats = gb.last_stats(stream)
    tuned = gb.tuning_lookup(d, n, args.min_pts, algo=algo)
    tuning = ({"block": tuned[0], "cell_factor": tuned[1], "source": "autotuner (first call of this kind)"}
              if tuned else {"block": None, "cell_factor": None, "source": "fixed (dbscan_set_tuning)"})

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid or str(dev.index))
    gb.profile_enable(True)
    gb.profile_collect(stream)  # drop warm-up records
    sampler.start()
    time.sleep(0.2)
    barrier()
    torch.cuda.synchronize(dev)
    launches0 = gb.kernel_launches()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    launches = gb.kernel_launches() - launches0
    clocks = sampler.stop()
    prof = gb.profile_collect(stream)
    gb.profile_enable(False)
    ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    value = n * world * args.steps / (ms / 1e3)

    # the same steps with two runs in flight: device-resident inputs, steps
    # alternating between two streams (each with its own workspace), so that
    # one run's idle phases (launch gaps, kernel tails, latency-bound stages)
    # fill with the other's work; CUDA events on the first stream, which
    # waits for the second before the end event
    s2 = torch.cuda.Stream(dev)
    labels2 = torch.empty_like(labels)
    two_streams = None
    for _ in range(0 if args.no_two_streams else 2):  # the second stream's workspace
        gb.dbscan_run(pts, eps, args.min_pts, mode=gb.MODE_DBSCAN, algo=algo, labels_out=labels2, stream=s2)
    torch.cuda.synchronize(dev)
    gb.stream_status(s2)
    barrier()
    if not args.no_two_streams:
        two_streams = timed_two_streams(gb, pts, eps, args, algo, labels, labels2, stream, s2, n, world, dev,
                                        barrier)

    # end to end through the host-buffer entry points: H2D of the points, the
    # clustering, D2H of the labels, every step. `e2e`: the asynchronous entry
    # point with steps alternating between two streams, so that one step's
    # copies overlap the other's kernels (pinned host buffers, one label
    # buffer per stream); `e2e_serial`: the synchronous entry point, one step
    # after the other
    e2e = e2e_serial = None
    if not args.no_e2e:
        host_pts = torch.from_numpy(X).pin_memory()
        hp = host_pts.numpy()
        streams = [stream, s2]
        host_labs = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in streams]
        hls = [t.numpy() for t in host_labs]
        e2e_steps = max(4, args.steps // 2)
        io = {"unit": UNIT, "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(4 * n)}
        for k in range(2):  # each stream's workspace and staging area
            gb.dbscan_run_host_async(hp, eps, args.min_pts, hls[k], algo=algo, stream=streams[k])
        for st in streams:
            st.synchronize()
            gb.stream_status(st)
        barrier()
        te = time.perf_counter()
        for i in range(e2e_steps):
            gb.dbscan_run_host_async(hp, eps, args.min_pts, hls[i % 2], algo=algo, stream=streams[i % 2])
        for st in streams:
            st.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - te, world, dev)
        for st in streams:
            gb.stream_status(st)  # the runs' device-side status
        e2e = {"value": n * world * e2e_steps / e2e_s, **io,
               "how": "dbscan_run_host_async, steps alternating between 2 streams (copies of one step overlap "
                      "the kernels of the other), pinned host buffers, wall clock from the first enqueue to "
                      "both streams done"}
        hl = hls[0]
        gb.dbscan_run_host(hp, eps, args.min_pts, algo=algo, labels_out=hl, stream=stream)
        barrier()
        te = time.perf_counter()
        for _ in range(e2e_steps):
            gb.dbscan_run_host(hp, eps, args.min_pts, algo=algo, labels_out=hl, stream=stream)
        e2e_s = max_over_ranks(time.perf_counter() - te, world, dev)
        e2e_serial = {"value": n * world * e2e_steps / e2e_s, **io,
                      "how": "dbscan_run_host, one step after the other (each waits for its labels)"}

    # roofline of the dominant stage (its kernels timed with CUDA events on the
    # launching stream over the timed region)
    m = stats["leaves"]
    # DenseBox keys of the halo grid (3 x 12 bits) share a word with the index
    model = bytes_model(n, d, m, 8 if algo == gb.ALGO_DENSEBOX else 4, packed=algo == gb.ALGO_DENSEBOX)
    stage_ms = {k: v[0] / max(1, args.steps) for k, v in prof.items() if v[1] > 0}
    top = max(stage_ms, key=stage_ms.get)
    peak, peak_kind = measured_peak_hbm()
    achieved = model[top] / (stage_ms[top] / 1e3) / 1e9
    path_bytes = sum(model[k] for k in stage_ms)
    traffic = None
    if top in ("preprocess", "main") and algo == gb.ALGO_DENSEBOX and args.min_pts == 10:
        traffic = measured_traffic(n, top)
        if traffic is not None:
            traffic /= 1.0  # bytes per launch of the stage (one launch per step)
    kernels = {"preprocess": "k_pre + k_list_claims", "main": "k_intra + k_kinds_* + k_main x3"}
    counts = traversal_counts(n) if (algo == gb.ALGO_DENSEBOX and args.min_pts == 10) else None
    stage_frac_hbm = {k: model[k] / (stage_ms[k] / 1e3) / 1e9 / peak for k in stage_ms}
    if top in ("preprocess", "main") and counts is not None:
        # the traversals are bound by instruction issue of fp32 / integer
        # work, not by DRAM: their roofline is the fp32 ALU rate, SMs x 128
        # lanes x the SM clock under load (one non-fused fp32 operation per
        # lane per cycle)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
        peak_alu = sms * 128 * mhz * 1e6 / 1e12
        per_pt = counts["per_point"][top]
        ops = fp32_ops(d, per_pt["distance_tests"], per_pt["box_tests"]) * n
        achieved_alu = ops / (stage_ms[top] / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved_alu, "peak": peak_alu, "unit": "TFLOP/s",
                    "frac": achieved_alu / peak_alu, "traffic": traffic, "kernel": kernels.get(top, top),
                    "stage": top, "peak_source": f"derived: {sms} SMs x 128 fp32 lanes x {mhz:.0f} MHz (sampled)",
                    "fp32_ops_per_launch": ops, "launch_ms": stage_ms[top],
                    "tests_per_point": per_pt, "counts_source": os.path.relpath(COUNTS_JSON, ROOT),
                    "hbm_frac": stage_frac_hbm[top]}
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "kernel": kernels.get(top, top), "stage": top,
                    "peak_source": peak_kind, "algorithmic_bytes_per_launch": model[top],
                    "launch_ms": stage_ms[top]}

    small = small_job_figures(args, dev) if (rank == 0 and not args.no_small_jobs) else {}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the reference arm's sample (the same window, so that both CPU
        # figures are one measurement), run until about 10 s of CPU work
        W = cpu_sample(X, args.ref_side)
        ts = [time_oracle(W, eps, args.min_pts)]
        while sum(ts) < 10.0 and len(ts) < 100:
            ts.append(time_oracle(W, eps, args.min_pts))
        tcpu = sum(ts)
        cpu = {"value": W.shape[0] * len(ts) / tcpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"points of the workload inside [0,{args.ref_side})^3: {W.shape[0]} points, "
                         f"same eps/minPts, {len(ts)} runs ({tcpu:.1f} s; the window of --impl reference)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(n, eps, args.min_pts), "n": n, "dim": d, "eps": eps,
                       "min_pts": args.min_pts, "algo": args.algo, "mode": "dbscan",
                       "border_claims": "neighbour lists" if gb.border_lists() else "main traversal (no lists)",
                       "tuning": tuning,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (201 MB of points; multi-GB working set per step)"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "e2e_serial": e2e_serial,
            "two_streams": two_streams,
            "clocks": clocks,
            "gpu_launches": int(launches),
            "stages_ms_per_step": {k: round(v, 4) for k, v in stage_ms.items()},
            "stages_hbm_frac": {k: round(v, 4) for k, v in stage_frac_hbm.items()},
            "hbm_frac_path": path_bytes / (ms / args.steps / 1e3) / 1e9 / peak,
            "features_per_s": value * d,
            "stats": stats,
            **small,
        }
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------ measurement modes
def run_counters_mode(args) -> None:
    """Counts the traversal's tests on the benchmark workload with the
    counters build of the library (libgbdbscan_counters.so, -DGBD_COUNTERS)
    and writes them per point to profiles/ (the default line reads them for
    its ALU roofline). Timing is meaningless in that build and is not taken."""
    import ctypes

    import torch

    from paper_2103_05162_gb300 import _build

    lib = ctypes.CDLL(_build.build(counters=True))
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
    lib.dbscan_run.argtypes = [vp, i64, i32, f32, i32, i32, i32, vp, vp, vp]
    lib.dbscan_traversal_counters.argtypes = [vp, i32]
    lib.dbscan_set_tuning.argtypes = [i32, f32]
    lib.dbscan_last_stats.argtypes = [vp, vp]
    lib.dbscan_stream_status.argtypes = [vp]
    for f in (lib.dbscan_run, lib.dbscan_traversal_counters, lib.dbscan_set_tuning, lib.dbscan_last_stats,
              lib.dbscan_stream_status):
        f.restype = i32
    assert lib.dbscan_set_tuning(128, 1.0) == 0  # the autotuner's choice for this workload; no tuning runs
    algo = 1 if args.algo == "densebox" else 0
    X, eps = workload(args.n, args.seed)
    n, d = X.shape
    pts = torch.from_numpy(X).cuda()
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = (ctypes.c_uint64 * 12)()

    def run():
        assert lib.dbscan_run(ctypes.c_void_p(pts.data_ptr()), n, d, eps, args.min_pts, 0, algo,
                              ctypes.c_void_p(labels.data_ptr()), None, stream) == 0
        assert lib.dbscan_stream_status(stream) == 0

    run()
    assert lib.dbscan_traversal_counters(out, 12) == 0  # discard the first run's
    run()
    assert lib.dbscan_traversal_counters(out, 12) == 0
    st = (ctypes.c_int64 * 2)()
    lib.dbscan_last_stats(stream, st)
    per_point = {ph: {k: out[4 * i + j] / n for j, k in enumerate(KINDS)} for i, ph in enumerate(PHASES)}
    rec = {
        "what": "traversal tests per point, one dbscan_run (counters build; the product build counts nothing)",
        "workload": workload_desc(n, eps, args.min_pts), "n": n, "dim": d, "min_pts": args.min_pts,
        "algo": args.algo, "leaves": int(st[0]), "dense_cells": int(st[1]),
        "per_point": per_point, "totals": {ph: {k: int(out[4 * i + j]) for j, k in enumerate(KINDS)}
                                             for i, ph in enumerate(PHASES)},
        "fp32_ops_per_test": {"distance": 3 * d - 1, "box": 6 * d - 1},
        "sources_sha256": sources_sha256(COUNT_SOURCES),
        "command": f"python bench.py --mode counters --n {args.n} --min-pts {args.min_pts} --algo {args.algo}",
    }
    if args.n == 1 << 24 and args.min_pts == 10 and args.algo == "densebox":
        with open(COUNTS_JSON, "w") as f:
            json.dump(rec, f, indent=1)
    print(json.dumps(rec), flush=True)


def run_traffic_mode(args) -> None:
    """Per-point DRAM bytes of the traversal stages from an ncu launch CSV
    (metrics dram__bytes_read.sum, dram__bytes_write.sum; one run of the
    halo workload at --n points after warm-up), written to profiles/ with the
    capture size, the sources' hash and the scaling rule."""
    import csv
    rows = list(csv.reader(open(args.ncu_csv)))
    hdr_i = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hdr_i]
    kcol, mcol, ucol, vcol = (hdr.index(c) for c in ("Kernel Name", "Metric Name", "Metric Unit", "Metric Value"))
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    per_kernel = {}
    for r in rows[hdr_i + 1:]:
        if len(r) <= vcol or not r[mcol].startswith("dram__bytes"):
            continue
        name = r[kcol].split("(")[0].split("<")[0].split("::")[-1].split()[-1]
        per_kernel[name] = per_kernel.get(name, 0.0) + float(r[vcol].replace(",", "")) * scale[r[ucol]]
    runs = args.traffic_runs
    by_stage = {st: sum(v for k, v in per_kernel.items() if k in ks) / runs for st, ks in STAGE_KERNELS.items()}
    rec = {
        "what": "DRAM bytes (read + write) per point of the traversal stages, ncu dram__bytes_read.sum + "
                "dram__bytes_write.sum over their kernels, per run",
        "capture_n": args.n, "runs_captured": runs,
        "bytes_per_point": {st: v / args.n for st, v in by_stage.items()},
        "kernels_bytes_per_run": {k: v / runs for k, v in per_kernel.items()},
        "scaling": "bytes of a run at n points = bytes_per_point x n (same workload family, halos shrunk in "
                   "proportion below 2^24 points)",
        "sources_sha256": sources_sha256(COUNT_SOURCES),
        "command": args.ncu_command,
    }
    with open(TRAFFIC_JSON, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec), flush=True)


def run_tune_mode(args) -> None:
    """The autotuner's choice on each workload of the measurement plan: the
    table is cleared, the first call of the kind measures the candidates,
    and the steady-state time per call (CUDA events, 5 runs after 2) is taken
    with the tuned knobs and with the fixed defaults (block 128, f = 1)."""
    import torch

    import paper_2103_05162_gb300 as gb
    from workloads import blobs, halo_eps, halos, roads

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    cases = [("blobs 16K 3D", blobs(16384, 3, 0), 0.03, 5, "densebox"),
             ("blobs 16K 3D", blobs(16384, 3, 0), 0.03, 5, "fdbscan"),
             ("roads 4M 2D", roads(1 << 22, 1), 2e-4, 10, "fdbscan"),
             ("roads 4M 2D", roads(1 << 22, 1), 2e-4, 10, "densebox")]
    H = halos(1 << 24, 2)
    for mp in (10, 2):
        for al in ("densebox", "fdbscan"):
            cases.append(("halos 16M 3D", H, halo_eps(1 << 24), mp, al))
    rows = []
    for name, X, eps, mp, al in cases:
        pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        lab = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
        gb.set_tuning(0, 0.0)
        gb.tuning_clear()
        t = time.perf_counter()
        gb.dbscan_run(pts, eps, mp, algo=al, labels_out=lab)
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t
        entry = gb.tuning_lookup(X.shape[1], X.shape[0], mp, algo=al)
        ms_tuned = timed(lambda: gb.dbscan_run(pts, eps, mp, algo=al, labels_out=lab))
        gb.set_tuning(128, 1.0)
        ms_fixed = timed(lambda: gb.dbscan_run(pts, eps, mp, algo=al, labels_out=lab))
        gb.set_tuning(0, 0.0)
        gb.stream_status()
        rows.append({"workload": name, "n": X.shape[0], "dim": X.shape[1], "min_pts": mp, "algo": al,
                     "block": entry[0], "cell_factor": entry[1], "tuning_call_s": round(tune_s, 3),
                     "ms_tuned": round(ms_tuned, 4), "ms_fixed_128_f1": round(ms_fixed, 4)})
        print(json.dumps(rows[-1]), flush=True)


# ------------------------------------------------------------ batch and serve
SMALL_BATCH = 512
SMALL_SERVE_JOBS = 400
SMALL_SERVE_RATES = (1000.0, 3000.0, 30000.0)
SMALL_SERVE_SIZES = (10_000, 262_144)


def small_job_figures(args, dev) -> dict:
    """Batched and served small jobs on one GPU, at reduced sizes that fit
    the default run (the full batch and serving sweeps are --mode batch and
    --mode serve):
    * batched: SMALL_BATCH instances of the batch family in one fused
      dbscan_run_batch (graph-captured once the shape repeats) against one
      dbscan_run per instance enqueued back to back on one stream;
    * served: Poisson traces of SMALL_SERVE_JOBS jobs of 10K-256K points
      through the server (continuous batching) against one dbscan_run per
      job in arrival order, each waited for (a one-job-at-a-time server).
    Latencies are wall clock, arrival (or call) to labels complete."""
    import torch

    import paper_2103_05162_gb300 as gb
    from workloads import batch_instances, serve_pools, serve_schedule

    out = {}
    # ---- batched
    inst = batch_instances(SMALL_BATCH, args.seed + 1)
    flat = np.concatenate([x.points.ravel() for x in inst]).astype(np.float32)
    offs = np.concatenate([[0], np.cumsum([x.n for x in inst])]).astype(np.int64)
    coffs = np.concatenate([[0], np.cumsum([x.n * x.dim for x in inst])]).astype(np.int64)
    dims, eps, mps = [x.dim for x in inst], [x.eps for x in inst], [x.min_pts for x in inst]
    pts = torch.from_numpy(flat).to(dev)
    total = int(offs[-1])
    labels = torch.empty(total, dtype=torch.int32, device=dev)
    views = [pts[coffs[b]:coffs[b + 1]].view(-1, dims[b]) for b in range(len(inst))]
    outs = [labels[offs[b]:offs[b + 1]] for b in range(len(inst))]

    def fused():
        gb.dbscan_run_batch(pts, offs, dims, eps, mps, algo=gb.ALGO_DENSEBOX, labels_out=labels)

    def sequential():
        for b in range(len(inst)):
            gb.dbscan_run(views[b], eps[b], mps[b], algo=gb.ALGO_DENSEBOX, labels_out=outs[b])

    for _ in range(3):  # direct launch, capture, replay
        fused()
    sequential()
    torch.cuda.synchronize(dev)
    tf, tsq = [], []
    for _ in range(7):
        t = time.perf_counter()
        fused()
        torch.cuda.synchronize(dev)
        tf.append(time.perf_counter() - t)
    for _ in range(3):
        t = time.perf_counter()
        sequential()
        torch.cuda.synchronize(dev)
        tsq.append(time.perf_counter() - t)
    gb.stream_status()
    f50, sq = float(np.median(tf)), float(np.median(tsq))
    out["batched"] = {
        "workload": f"{SMALL_BATCH} instances of the batch family (lognormal sizes, median 20k, sigma 1.2, "
                    "clipped to [1k, 500k]; 2D/3D blobs; eps U[0.01,0.05]; minPts U{2,5,10}), DenseBox, DBSCAN",
        "points": total, "instances": len(inst),
        "p50_ms": 1e3 * f50, "p99_ms": 1e3 * float(np.percentile(tf, 99)),
        "points_per_s": total / f50,
        "sequential": {"ms": 1e3 * sq, "points_per_s": total / sq},
        "ratio": sq / f50,
    }
    del pts, labels, views, outs

    # ---- served
    pool_n = 1 << 20
    pools = {k: torch.from_numpy(v).to(dev) for k, v in serve_pools(pool_n, args.seed + 100).items()}
    scheds = [serve_schedule(SMALL_SERVE_JOBS, lam, args.seed + 2000 + i, pool_n=pool_n,
                             size_range=SMALL_SERVE_SIZES) for i, lam in enumerate(SMALL_SERVE_RATES)]
    cap = max(sum(j.n for j in sc) for sc in scheds)
    arena = torch.empty(cap, dtype=torch.int32, device=dev)
    srv = gb.Server(int(args.serve_budget_gb * (1 << 30)), max_slots=args.serve_slots)

    def views_of(sched):
        res, o = [], 0
        for j in sched:
            res.append((pools[j.pool][j.offset:j.offset + j.n], arena[o:o + j.n]))
            o += j.n
        return res

    def served(sched, vs):
        lag, ids, sub = [], [], []
        t0 = time.perf_counter()
        for j, (x, lab) in zip(sched, vs):
            target = t0 + j.arrival_s
            now = _wait_until(target)
            ids.append(srv.submit(x, j.eps, j.min_pts, algo=j.algo, labels_out=lab))
            lag.append(now - target)
            sub.append(now)
        lat, done_at = [], []
        for jid, lg, ts in zip(ids, lag, sub):
            srv.wait(jid, timeout=600)
            _, l_srv = srv.poll(jid)
            srv.release(jid)
            lat.append(lg + l_srv)
            done_at.append(ts + l_srv)
        return np.asarray(lat), max(done_at) - t0

    def one_at_a_time(sched, vs):
        lat, t0 = [], time.perf_counter()
        done = t0
        for j, (x, lab) in zip(sched, vs):
            target = t0 + j.arrival_s
            _wait_until(max(target, done))
            gb.dbscan_run(x, j.eps, j.min_pts, algo=j.algo, labels_out=lab)
            torch.cuda.synchronize(dev)
            done = time.perf_counter()
            lat.append(done - target)
        return np.asarray(lat), done - t0

    rows = []
    for lam, sched in zip(SMALL_SERVE_RATES, scheds):
        vs = views_of(sched)
        pts_total = sum(j.n for j in sched)
        served(sched, vs)  # warm-up: workspaces, graphs
        one_at_a_time(sched, vs)
        stats0 = srv.stats()
        lat, span = served(sched, vs)
        st = {k: v - stats0[k] for k, v in srv.stats().items()}
        slat, sspan = one_at_a_time(sched, vs)
        rows.append({
            "rate_per_s": lam, "jobs": len(sched), "points": pts_total,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "points_per_s": pts_total / span,
            "sequential": {"p50_ms": 1e3 * float(np.percentile(slat, 50)),
                           "p99_ms": 1e3 * float(np.percentile(slat, 99)), "points_per_s": pts_total / sspan},
            "ratio": sspan / span, "fused_batches": st.get("batches"), "fused_jobs": st.get("batched_jobs"),
        })
    srv.close()
    gb.stream_status()
    out["served"] = {
        "workload": f"Poisson arrivals, {SMALL_SERVE_JOBS} jobs per rate, sizes log-uniform on "
                    f"[{SMALL_SERVE_SIZES[0]}, {SMALL_SERVE_SIZES[1]}], families blobs3/roads/halos/batch "
                    "instance (windows of 1M-point shuffled pools), DBSCAN mode; "
                    f"server: {args.serve_slots} slots, {args.serve_budget_gb} GB budget; sequential: "
                    "one dbscan_run per job in arrival order, each waited for",
        "rates": rows,
    }
    return out


def run_batch_mode(args) -> None:
    """One fused dbscan_run_batch over thousands of independent instances
    against one dbscan_run per instance on one stream (same inputs, same
    outputs)."""
    import torch

    import paper_2103_05162_gb300 as gb
    from workloads import batch_instances

    t0 = time.perf_counter()
    inst = batch_instances(args.batch_count, args.seed + 1, size_scale=args.batch_scale)
    gen_s = time.perf_counter() - t0
    flat = np.concatenate([x.points.ravel() for x in inst]).astype(np.float32)
    offs = np.concatenate([[0], np.cumsum([x.n for x in inst])]).astype(np.int64)
    coffs = np.concatenate([[0], np.cumsum([x.n * x.dim for x in inst])]).astype(np.int64)
    dims = [x.dim for x in inst]
    eps = [x.eps for x in inst]
    mps = [x.min_pts for x in inst]
    pts = torch.from_numpy(flat).cuda()
    total = int(offs[-1])
    labels = torch.empty(total, dtype=torch.int32, device="cuda")
    views = [pts[coffs[b]:coffs[b + 1]].view(-1, dims[b]) for b in range(len(inst))]
    outs = [labels[offs[b]:offs[b + 1]] for b in range(len(inst))]
    for algo_name in args.batch_algos.split(","):
        algo = gb.ALGO_DENSEBOX if algo_name == "densebox" else gb.ALGO_FDBSCAN

        def batch():
            gb.dbscan_run_batch(pts, offs, dims, eps, mps, algo=algo, labels_out=labels)

        def sequential():
            for b in range(len(inst)):
                if offs[b + 1] > offs[b]:
                    gb.dbscan_run(views[b], eps[b], mps[b], algo=algo, labels_out=outs[b])

        for _ in range(max(3, args.warmup)):  # direct, capture, replay
            batch()
        torch.cuda.synchronize()
        launches0 = gb.kernel_launches()
        tb = []
        for _ in range(args.steps):
            t = time.perf_counter()
            batch()
            torch.cuda.synchronize()
            tb.append(time.perf_counter() - t)
        launches = (gb.kernel_launches() - launches0) / args.steps
        sequential()
        torch.cuda.synchronize()
        t = time.perf_counter()
        sequential()
        torch.cuda.synchronize()
        ts = time.perf_counter() - t
        tbm = float(np.median(tb))
        print(json.dumps({
            "metric": "batched points clustered/sec (one fused batch vs one run per instance)",
            "value": total / tbm, "unit": UNIT, "algo": algo_name, "instances": len(inst), "points": total,
            "batch_ms_median": 1e3 * tbm, "batch_ms_min": 1e3 * min(tb), "sequential_ms": 1e3 * ts,
            "sequential_points_per_s": total / ts, "speedup": ts / tbm, "gpu_launches_per_batch": launches,
            "steps": args.steps, "timing": "wall clock around the call and a device synchronize",
            "workload": f"batch_instances({args.batch_count}, seed={args.seed + 1}, size_scale={args.batch_scale}):"
                        f" lognormal sizes, 2D/3D blobs, eps U[0.01,0.05], minPts U{{2,5,10}}",
            "gen_s": round(gen_s, 1)}), flush=True)


def run_sweep_mode(args) -> None:
    """One dbscan_run_multi over several minPts against one dbscan_run per
    minPts, on the benchmark workload (CUDA events, inputs resident)."""
    import torch

    import paper_2103_05162_gb300 as gb

    algo = gb.ALGO_DENSEBOX if args.algo == "densebox" else gb.ALGO_FDBSCAN
    X, eps = workload(args.n, args.seed)
    n = X.shape[0]
    mps = [int(x) for x in args.sweep_min_pts.split(",")]
    pts = torch.from_numpy(X).cuda()
    lab = torch.empty((len(mps), n), dtype=torch.int32, device="cuda")

    def multi():
        gb.dbscan_run_multi(pts, eps, mps, algo=algo, labels_out=lab)

    def singles():
        for k, mp in enumerate(mps):
            gb.dbscan_run(pts, eps, mp, algo=algo, labels_out=lab[k])

    res = {}
    for name, f in (("multi", multi), ("singles", singles)):
        for _ in range(max(3, args.warmup)):
            f()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(args.steps):
            f()
        t1.record()
        torch.cuda.synchronize()
        res[name] = t0.elapsed_time(t1) / args.steps
    print(json.dumps({
        "metric": "minPts sweep: one index and one counting pass vs one run per minPts",
        "min_pts": mps, "algo": args.algo, "n": n, "multi_ms": res["multi"], "singles_ms": res["singles"],
        "speedup": res["singles"] / res["multi"], "value": n * len(mps) / (res["multi"] / 1e3),
        "unit": "point-clusterings/s", "steps": args.steps,
        "workload": f"halos3d: {n} 3D float32 points (the benchmark workload), eps={eps:.6g}, minPts in {mps}, "
                    f"DBSCAN mode"}), flush=True)


def run_slabs_mode(args) -> None:
    """Slab-wise clustering of host points (the out-of-core path): copies of
    the benchmark workload side by side along x, clustered in slabs of
    --slab-points points; wall time of the whole call (host partition and
    merge, copies, both device passes)."""
    import paper_2103_05162_gb300 as gb

    X1, eps = workload(args.n, args.seed)
    X = np.concatenate([X1 + np.array([float(c), 0.0, 0.0], np.float32) for c in range(args.slab_copies)])
    X = np.ascontiguousarray(X, dtype=np.float32)
    algo = gb.ALGO_DENSEBOX if args.algo == "densebox" else gb.ALGO_FDBSCAN
    gb.dbscan_run_slabs(X[: len(X1)], eps, args.min_pts, algo=algo, slab_points=args.slab_points)  # warm-up
    ts = []
    for _ in range(max(1, args.steps)):
        t = time.perf_counter()
        gb.dbscan_run_slabs(X, eps, args.min_pts, algo=algo, slab_points=args.slab_points)
        ts.append(time.perf_counter() - t)
    tm = float(np.median(ts))
    print(json.dumps({
        "metric": "points clustered/sec, slab-wise from host memory", "value": X.shape[0] / tm, "unit": UNIT,
        "points": int(X.shape[0]), "slab_points": args.slab_points, "seconds_median": tm, "steps": len(ts),
        "algo": args.algo, "min_pts": args.min_pts,
        "workload": f"{args.slab_copies} copies of {workload_desc(args.n, eps, args.min_pts)} side by side along x",
        "timing": "wall clock of dbscan_run_slabs (host partition, gathers, copies, two device passes, merge)"}),
        flush=True)


def _wait_until(target: float) -> float:
    while True:
        now = time.perf_counter()
        if now >= target:
            return now
        if target - now > 2e-3:
            time.sleep(target - now - 1e-3)


def run_serve_mode(args) -> None:
    """Replays Poisson arrival schedules in real time through the server
    (continuous batching, several slots) and, on the same schedule, through
    one dbscan_run per job in arrival order on one stream; reports latency
    percentiles (arrival to labels complete) and throughput of both."""
    import torch

    import paper_2103_05162_gb300 as gb
    from workloads import SERVE_POOL_N, serve_pools, serve_schedule

    t0 = time.perf_counter()
    pools = {k: torch.from_numpy(v).cuda() for k, v in serve_pools(SERVE_POOL_N, args.seed + 100).items()}
    gen_s = time.perf_counter() - t0
    rates = [float(x) for x in args.serve_rates.split(",")]
    scheds = [serve_schedule(args.serve_jobs, lam, args.seed + 1000 + i) for i, lam in enumerate(rates)]
    cap = max(sum(j.n for j in sc) for sc in scheds)
    arena = torch.empty(cap, dtype=torch.int32, device="cuda")

    def views(sched):
        out, o = [], 0
        for j in sched:
            out.append((pools[j.pool][j.offset:j.offset + j.n], arena[o:o + j.n]))
            o += j.n
        return out

    # warm-up: every slot (and the sequential arm's stream) grows its
    # workspace to the largest job of each family and algorithm
    from workloads import halo_eps
    warm = [("blobs3", 1, 0.03), ("blobs2", 1, 0.03), ("halos", 1, halo_eps(SERVE_POOL_N)),
            ("roads", 0, float(np.float32(2e-4 * (4194304 / SERVE_POOL_N) ** 0.5)))]
    srv = gb.Server(int(args.serve_budget_gb * (1 << 30)), max_slots=args.serve_slots)
    srv.hold(True)
    wids = [srv.submit(pools[p], e, 10, algo=a, labels_out=arena[:SERVE_POOL_N])
            for _ in range(args.serve_slots) for p, a, e in warm]
    srv.hold(False)
    for w in wids:
        srv.wait(w, timeout=600)
        srv.release(w)
    for p, a, e in warm:
        gb.dbscan_run(pools[p], e, 10, algo=a, labels_out=arena[:SERVE_POOL_N])
    torch.cuda.synchronize()

    for lam, sched in zip(rates, scheds):
        vs = views(sched)
        total = sum(j.n for j in sched)
        stats0 = srv.stats()
        # served
        lag, ids, sub = [], [], []
        t0 = time.perf_counter()
        for j, (x, lab) in zip(sched, vs):
            target = t0 + j.arrival_s
            now = _wait_until(target)
            ids.append(srv.submit(x, j.eps, j.min_pts, algo=j.algo, labels_out=lab))
            lag.append(now - target)
            sub.append(now)
        lat, done_at = [], []
        for jid, lg, ts in zip(ids, lag, sub):
            srv.wait(jid, timeout=600)
            _, l_srv = srv.poll(jid)
            srv.release(jid)
            lat.append(lg + l_srv)
            done_at.append(ts + l_srv)
        span = max(done_at) - t0
        st = {k: v - stats0[k] for k, v in srv.stats().items()}
        # sequential plain runs, arrival order, one stream
        slat, t0 = [], time.perf_counter()
        done = t0
        for j, (x, lab) in zip(sched, vs):
            target = t0 + j.arrival_s
            _wait_until(target)
            gb.dbscan_run(x, j.eps, j.min_pts, algo=j.algo, labels_out=lab)
            torch.cuda.synchronize()
            done = time.perf_counter()
            slat.append(done - target)
        sspan = done - t0
        lat_ms, slat_ms = 1e3 * np.asarray(lat), 1e3 * np.asarray(slat)
        print(json.dumps({
            "metric": "served latency, arrival to labels complete (Poisson arrivals)",
            "rate_per_s": lam, "jobs": len(sched), "points": total, "mean_job_points": total / len(sched),
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "points_per_s": total / span, "span_s": span,
            "sequential": {"p50_ms": float(np.percentile(slat_ms, 50)), "p99_ms": float(np.percentile(slat_ms, 99)),
                           "points_per_s": total / sspan, "span_s": sspan},
            "server": {"slots": args.serve_slots, "budget_gb": args.serve_budget_gb, **st},
            "submit_lag_ms_p99": float(np.percentile(1e3 * np.asarray(lag), 99)),
            "workload": "serve_schedule: sizes log-uniform [1e4, 8e6]; families blobs3 (DenseBox), roads "
                        "(FDbscan), halos (DenseBox), batch instances (DenseBox); each job a window of an "
                        f"8M-point shuffled pool; DBSCAN mode; pools generated in {gen_s:.1f} s"}), flush=True)
    srv.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--min-pts", type=int, default=10)
    ap.add_argument("--algo", choices=["densebox", "fdbscan"], default="densebox")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--ref-side", type=float, default=0.25,
                    help="edge of the cube [0,a)^3 whose points form the CPU sample: each step of the reference "
                         "arm, and the runs of the GPU arm's cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-small-jobs", action="store_true", help="skip the batched / served small-job figures")
    ap.add_argument("--no-two-streams", action="store_true", help="skip the two-runs-in-flight figure")
    ap.add_argument("--block", type=int, default=0, help="traversal block size (0: autotuner)")
    ap.add_argument("--cell-factor", type=float, default=0.0, help="DenseBox cell factor (0: autotuner)")
    ap.add_argument("--border-lists", type=int, choices=[0, 1], default=None,
                    help="border claims from per-point neighbour lists (1) or in the main traversal (0); "
                         "default: the library's default")
    ap.add_argument("--ncu-csv", default=None, help="--mode traffic: the ncu launch CSV to summarise")
    ap.add_argument("--ncu-command", default="", help="--mode traffic: the command that produced the CSV")
    ap.add_argument("--traffic-runs", type=int, default=1, help="--mode traffic: clustering runs captured")
    ap.add_argument("--mode", choices=["step", "batch", "serve", "sweep", "slabs", "counters", "traffic", "tune"],
                    default="step",
                    help="step: the headline line (default); batch: fused batch vs per-instance runs; "
                         "serve: Poisson-arrival serving vs sequential runs; sweep: several minPts over one "
                         "index vs one run each; slabs: slab-wise clustering from host memory "
                         "(these four: 1 GPU, rank 0 only)")
    ap.add_argument("--sweep-min-pts", default="2,5,10,20")
    ap.add_argument("--slab-copies", type=int, default=4)
    ap.add_argument("--slab-points", type=int, default=1 << 24)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--batch-algos", default="densebox,fdbscan")
    ap.add_argument("--serve-rates", default="100,300,1000,3000,5000")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.mode != "step":
        if rank == 0:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            {"batch": run_batch_mode, "serve": run_serve_mode, "sweep": run_sweep_mode,
             "slabs": run_slabs_mode, "counters": run_counters_mode, "traffic": run_traffic_mode,
             "tune": run_tune_mode}[args.mode](args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    run_gb300(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
