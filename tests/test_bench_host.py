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


def test_measured_traffic_per_stage_and_source_check(tmp_path):
    """The roofline's traffic comes from a profile summary per stage, scaled
    by the points, and only while the sources still hash to the recorded
    value."""
    import hashlib
    b = _load_bench()
    srcs = []
    for i, text in enumerate((b"kernel one\n", b"kernel two\n")):
        f = tmp_path / f"src{i}.cu"
        f.write_bytes(text)
        srcs.append(str(f))
    digest = hashlib.sha256(b"kernel one\nkernel two\n").hexdigest()
    summary = tmp_path / "summary.md"
    summary.write_text("# capture\n\ntraffic_bytes_per_point_preprocess: 45.5\n"
                       "traffic_bytes_per_point_main: 22.25\nsources_sha256: %s\n" % digest)
    b.TRAFFIC_SUMMARY, b.TRAFFIC_SOURCES = str(summary), srcs
    assert b.measured_traffic(1000, "preprocess") == pytest.approx(45500.0)
    assert b.measured_traffic(2000, "main") == pytest.approx(44500.0)
    assert b.measured_traffic(1000, "sort") is None          # no figure for that stage
    (tmp_path / "src1.cu").write_bytes(b"kernel two, changed\n")
    assert b.measured_traffic(1000, "preprocess") is None    # sources changed since the capture


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
