"""Host-side parts of bench.py: the reference arm's JSON line, its silence on
ranks other than 0, and the max-over-ranks reduction of the multi-rank path
(world size 2 over gloo on the CPU)."""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          env=env, timeout=600)


def test_reference_arm_prints_one_json_line():
    r = _run_bench(["--impl", "reference", "--n", "20000", "--steps", "2", "--warmup", "3", "--ref-side", "0.5"])
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "points/s"
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["metric"].startswith("points clustered/sec")


def test_reference_arm_is_silent_on_other_ranks():
    r = _run_bench(["--impl", "reference", "--n", "20000", "--steps", "1", "--warmup", "3", "--gpus", "2"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world_2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    del torch


def _load_bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _fake_sources(b, tmp_path):
    import hashlib
    srcs = []
    for i, text in enumerate((b"kernel one\n", b"kernel two\n")):
        f = tmp_path / f"src{i}.cu"
        f.write_bytes(text)
        srcs.append(str(f))
    b.COUNT_SOURCES = srcs
    return hashlib.sha256(b"kernel one\nkernel two\n").hexdigest()


def test_measured_traffic_per_stage_and_source_check(tmp_path):
    """The roofline's traffic comes from the ncu summary in profiles/ (JSON:
    bytes per point per stage), scaled by the points, and only while the
    sources still hash to the recorded value."""
    b = _load_bench()
    digest = _fake_sources(b, tmp_path)
    summary = tmp_path / "traffic.json"
    summary.write_text(json.dumps({"bytes_per_point": {"preprocess": 45.5, "main": 22.25},
                                   "sources_sha256": digest, "capture_n": 8388608}))
    b.TRAFFIC_JSON = str(summary)
    assert b.measured_traffic(1000, "preprocess") == pytest.approx(45500.0)
    assert b.measured_traffic(2000, "main") == pytest.approx(44500.0)
    assert b.measured_traffic(1000, "sort") is None          # no figure for that stage
    (tmp_path / "src1.cu").write_bytes(b"kernel two, changed\n")
    assert b.measured_traffic(1000, "preprocess") is None    # sources changed since the capture


def test_traversal_counts_are_used_only_for_their_workload_and_sources(tmp_path):
    b = _load_bench()
    digest = _fake_sources(b, tmp_path)
    rec = {"n": 1 << 24, "sources_sha256": digest,
           "per_point": {"preprocess": {"distance_tests": 40.0, "box_tests": 12.0}}}
    f = tmp_path / "counts.json"
    f.write_text(json.dumps(rec))
    b.COUNTS_JSON = str(f)
    assert b.traversal_counts(1 << 24)["per_point"]["preprocess"]["distance_tests"] == 40.0
    assert b.traversal_counts(1 << 20) is None
    (tmp_path / "src0.cu").write_bytes(b"other\n")
    assert b.traversal_counts(1 << 24) is None


def test_committed_profiles_belong_to_the_current_sources():
    """The traversal counts and DRAM traffic that the bench line's roofline
    reads from profiles/ were taken on the sources as they are (a kernel
    change makes the bench drop them until they are measured again)."""
    b = _load_bench()
    counts = b.traversal_counts(1 << 24)
    assert counts is not None, "profiles/ counts are stale: python bench.py --mode counters"
    assert counts["algo"] == "densebox" and counts["min_pts"] == 10 and counts["dim"] == 3
    per = counts["per_point"]["preprocess"]
    assert per["distance_tests"] > 0 and per["box_tests"] > 0
    for stage in ("preprocess", "main"):
        t = b.measured_traffic(1 << 24, stage)
        assert t is not None and t > 0, "profiles/ traffic is stale: retake the ncu dram__bytes capture"


def test_fp32_operations_per_test():
    """3D: a distance test is 3 differences, 3 products and 2 sums; a box
    test 3 x (2 differences, 2 maxima, 1 product) + 2 sums."""
    b = _load_bench()
    assert b.fp32_ops(3, 1, 0) == 8 and b.fp32_ops(3, 0, 1) == 17
    assert b.fp32_ops(2, 1, 0) == 5 and b.fp32_ops(2, 0, 1) == 11


def test_traffic_summary_from_an_ncu_csv(tmp_path):
    """--mode traffic sums dram bytes of each stage's kernels from the
    launch CSV (units converted) and divides by the runs and points."""
    b = _load_bench()
    _fake_sources(b, tmp_path)
    csv_path = tmp_path / "launches.csv"
    lines = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    for k, unit, rd, wr in (("void k_pre<3>(DevArgs<T1>)", "Mbyte", "2.5", "0.5"),
                            ("k_list_claims(const int *)", "Kbyte", "500", "500"),
                            ("void k_main<3, 1>(DevArgs<T1>)", "Mbyte", "1", "1"),
                            ("void k_intra<3>(DevArgs<T1>)", "byte", "1000000", "0"),
                            ("k_onesweep", "Mbyte", "9", "9")):
        lines.append(f'"1","{k}","dram__bytes_read.sum","{unit}","{rd}"')
        lines.append(f'"1","{k}","dram__bytes_write.sum","{unit}","{wr}"')
    csv_path.write_text("\n".join(lines) + "\n")
    out = tmp_path / "traffic.json"
    b.TRAFFIC_JSON = str(out)

    class A:
        ncu_csv, n, traffic_runs, ncu_command = str(csv_path), 1000, 1, "ncu ..."
    b.run_traffic_mode(A)
    rec = json.loads(out.read_text())
    assert rec["bytes_per_point"]["preprocess"] == pytest.approx(4e6 / 1000)
    assert rec["bytes_per_point"]["main"] == pytest.approx(3e6 / 1000)


def test_bytes_model_packed_sort_moves_a_third_less():
    """Keys-only sort of packed 64-bit words: 16 bytes per point against 24
    for (64-bit key, 32-bit index) pairs; the gather also writes the
    permutation and the keys."""
    b = _load_bench()
    n, d, m = 1 << 20, 3, 1 << 15
    pairs = b.bytes_model(n, d, m, 8)
    packed = b.bytes_model(n, d, m, 8, packed=True)
    assert pairs["sort"] == 24 * n and packed["sort"] == 16 * n
    assert packed["gather"] - pairs["gather"] == 16 * n
    assert {k: v for k, v in pairs.items() if k not in ("keys", "sort", "gather")} == \
        {k: v for k, v in packed.items() if k not in ("keys", "sort", "gather")}
