#!/usr/bin/env python
"""Benchmark: points clustered per second by FDbscan-DenseBox on 2^24 3D
cosmology-like points on one GB300 (plus the fraction of the HBM roofline).

One step is one complete dbscan_run (bounds, keys, radix sort, gather,
DenseBox cells, LBVH build and refit, union-find init, preprocessing, main
traversal with fused union-find, finalize and relabel) on device-resident
points; the output labels stay on the device.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
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
def bytes_model(n: int, d: int, m: int, key_bytes: int) -> dict:
    """Compulsory device-memory traffic of each stage (each logical array read
    or written once per stage), in bytes per run. n points, d dims, m BVH
    leaves, key_bytes 8 (DenseBox cell keys) or 4 (FDbscan Morton codes)."""
    kv = key_bytes + 4
    return {
        "bounds": 4 * d * n,                              # read coordinates
        "keys": 4 * d * n + kv * n,                       # read coordinates, write key + index
        "sort": 2 * kv * n,                               # read and write (key, index) once
        "gather": 4 * n + 4 * d * n + 4 * d * n,          # read index and coordinates, write sorted coordinates
        "leaves": key_bytes * n + 5 * n + 8 * m,          # read keys, write flags, leaf records
        "lbvh": 4 * d * n + 8 * m + 64 * m + 64 * m,      # leaf boxes from points, keys, node records, refit
        "init": 5 * n,                                    # labels + core flags
        "preprocess": 4 * d * n + 64 * m + n,             # points once, tree once, core flags
        "main": 4 * d * n + 64 * m + n + 4 * n + 4 * n,   # points, tree, core flags, labels read and written
        "finalize": 8 * n + 8 * n,                        # labels + index read, output labels + core written
    }


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


def run_gb300(args, rank: int, world: int) -> None:
    import torch
    import torch.distributed as dist

    import paper_2103_05162_gb300 as gb

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    gb.load()
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
        step()
    torch.cuda.synchronize(dev)
    stats = gb.last_stats(stream)

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
    ms = t0.elapsed_time(t1)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = n * world * args.steps / (ms / 1e3)

    # end to end through the host-buffer entry point: H2D of the points, the
    # clustering, D2H of the labels, every step
    e2e = None
    if not args.no_e2e:
        host_pts = torch.from_numpy(X).pin_memory()
        host_lab = torch.empty(n, dtype=torch.int32).pin_memory()
        hp, hl = host_pts.numpy(), host_lab.numpy()
        for _ in range(max(1, args.warmup // 2)):
            gb.dbscan_run_host(hp, eps, args.min_pts, algo=algo, labels_out=hl, stream=stream)
        barrier()
        te = time.perf_counter()
        e2e_steps = max(3, args.steps // 2)
        for _ in range(e2e_steps):
            gb.dbscan_run_host(hp, eps, args.min_pts, algo=algo, labels_out=hl, stream=stream)
        e2e_s = time.perf_counter() - te
        if world > 1:
            t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": n * world * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(X.nbytes),
               "d2h_bytes_per_step": int(4 * n)}

    # roofline of the dominant stage (its kernels timed with CUDA events on the
    # launching stream over the timed region)
    m = stats["leaves"]
    model = bytes_model(n, d, m, 8 if algo == gb.ALGO_DENSEBOX else 4)
    stage_ms = {k: v[0] / max(1, args.steps) for k, v in prof.items() if v[1] > 0}
    top = max(stage_ms, key=stage_ms.get)
    peak, peak_kind = measured_peak_hbm()
    achieved = model[top] / (stage_ms[top] / 1e3) / 1e9
    path_bytes = sum(model[k] for k in stage_ms)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": top, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": model[top], "launch_ms": stage_ms[top]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        W = cpu_sample(X, args.cpu_side)
        tcpu = time_oracle(W, eps, args.min_pts)
        cpu = {"value": W.shape[0] / tcpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"points of the workload inside [0,{args.cpu_side})^3: {W.shape[0]} points, "
                         f"same eps/minPts, one run ({tcpu:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(n, eps, args.min_pts), "n": n, "dim": d, "eps": eps,
                       "min_pts": args.min_pts, "algo": args.algo, "mode": "dbscan",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (201 MB of points; multi-GB working set per step)"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": int(launches),
            "stages_ms_per_step": {k: round(v, 4) for k, v in stage_ms.items()},
            "hbm_frac_path": path_bytes / (ms / args.steps / 1e3) / 1e9 / peak,
            "features_per_s": value * d,
            "stats": stats,
        }
        print(json.dumps(line), flush=True)


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
    ap.add_argument("--cpu-side", type=float, default=0.6,
                    help="edge of the cube [0,a)^3 whose points form the CPU baseline's sample (one run)")
    ap.add_argument("--ref-side", type=float, default=0.25,
                    help="edge of the cube whose points form each step of the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
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
