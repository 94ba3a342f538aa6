"""Full-size parity: the CUDA path against the complete oracle clustering on
the workloads at the sizes the benchmark runs them.

* 3D halos, 2^24 points (eps = 0.2 x mean spacing), minPts 10 and 2, both
  modes, DenseBox and FDbscan, border claims from lists and in the main
  traversal;
* 2D roads, 4,194,304 points (eps 2e-4, minPts 10), both modes, both
  algorithms;
* the 4096-instance batch (lognormal sizes, 164M points), one fused
  dbscan_run_batch, every 16th instance compared with the oracle run on that
  instance alone.

Every comparison is the one of Sec. 2.1: core set, noise set and the label
of every core point exactly; a border point's label within the set of
clusters of its core neighbours (DBSCAN mode), or -1 (DBSCAN*). The oracle
runs on the host cores in threads (its C calls release the interpreter
lock); nothing here is timed.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from tests.parity import assert_matches_oracle
from workloads import batch_instances, halo_eps, halos, roads

torch = pytest.importorskip("torch")
import paper_2103_05162_gb300 as gb  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ALGOS = [gb.ALGO_DENSEBOX, gb.ALGO_FDBSCAN]
MODES = [gb.MODE_DBSCAN, gb.MODE_DBSCAN_STAR]


def _threads() -> int:
    return max(2, min(16, len(os.sched_getaffinity(0))))


def _reference(X, eps, min_pts):
    """Oracle labels and core flags (DBSCAN mode) plus its border sets. The
    DBSCAN* result shares the core part (Sec. 2.1) and makes every non-core
    point noise, so one oracle run serves both modes."""
    ref = oracle.dbscan(X, eps, min_pts, oracle.MODE_DBSCAN)
    sets = oracle.border_sets(X, eps, ref[1], ref[0])
    return ref, sets


def _gpu(X, eps, mp, mode, algo):
    pts = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    lab, core = gb.dbscan_run(pts, eps, mp, mode=mode, algo=algo, want_core=True)
    torch.cuda.synchronize()
    gb.stream_status()
    out = lab.cpu().numpy(), core.cpu().numpy().astype(bool)
    del pts, lab, core
    return out


# ------------------------------------------------------------ 3D halos, 2^24

@pytest.fixture(scope="module")
def halos16m():
    n = 1 << 24
    X = halos(n, 2)
    eps = halo_eps(n)
    with ThreadPoolExecutor(2) as ex:
        futs = {mp: ex.submit(_reference, X, eps, mp) for mp in (10, 2)}
        refs = {mp: f.result() for mp, f in futs.items()}
    return X, eps, refs


@pytest.mark.parametrize("mp,mode,algo", [
    (10, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX),
    (10, gb.MODE_DBSCAN_STAR, gb.ALGO_DENSEBOX),
    (10, gb.MODE_DBSCAN, gb.ALGO_FDBSCAN),
    (2, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX),
    (2, gb.MODE_DBSCAN_STAR, gb.ALGO_DENSEBOX),
    (2, gb.MODE_DBSCAN, gb.ALGO_FDBSCAN),
])
def test_halos_16m_full_oracle(halos16m, mp, mode, algo):
    """The benchmark workload (2^24 3D points, 50,000 halos + 30% background),
    every point compared with the oracle."""
    X, eps, refs = halos16m
    ref, sets = refs[mp]
    lab, core = _gpu(X, eps, mp, mode, algo)
    assert_matches_oracle(X, eps, mp, mode, lab, core, ref=ref, sets=sets)
    # the case is not degenerate: clusters, noise and (minPts 10) border points
    assert ref[1].any() and (ref[0] == -1).any()
    if mp == 10:
        assert (~ref[1] & (ref[0] >= 0)).any()


def test_halos_16m_full_oracle_without_border_lists(halos16m):
    """The benchmark workload with border claims made in the main traversal
    (no per-point neighbour list), every point compared with the oracle."""
    X, eps, refs = halos16m
    ref, sets = refs[10]
    gb.set_border_lists(False)
    try:
        lab, core = _gpu(X, eps, 10, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX)
    finally:
        gb.set_border_lists(True)
    assert_matches_oracle(X, eps, 10, gb.MODE_DBSCAN, lab, core, ref=ref, sets=sets)


# ------------------------------------------------------------ 2D roads, 4M

@pytest.fixture(scope="module")
def roads4m():
    X = roads(1 << 22, 1)
    return X, _reference(X, 2e-4, 10)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("mode", MODES)
def test_roads_4m_full_oracle(roads4m, mode, algo):
    """The 2D workload at full size (4,194,304 points, eps 2e-4, minPts 10)."""
    X, (ref, sets) = roads4m
    lab, core = _gpu(X, 2e-4, 10, mode, algo)
    assert_matches_oracle(X, 2e-4, 10, mode, lab, core, ref=ref, sets=sets)


# ------------------------------------------------------------ 4096-instance batch

def test_batch_4096_instances_every_16th_against_oracle():
    """The batch workload at full size (4096 instances, sizes lognormal(median
    20k, sigma 1.2) clipped to [1k, 500k], 2D/3D, per-instance eps and minPts)
    in one dbscan_run_batch; every 16th instance (256 of them, about 9.5M
    points) compared with the oracle run on that instance alone."""
    inst = batch_instances(4096, 3)
    offs = np.concatenate([[0], np.cumsum([x.n for x in inst])]).astype(np.int64)
    flat = np.concatenate([x.points.ravel() for x in inst]).astype(np.float32)
    pts = torch.from_numpy(flat).cuda()
    del flat
    total = int(offs[-1])
    labels = torch.empty(total, dtype=torch.int32, device="cuda")
    core = torch.empty(total, dtype=torch.uint8, device="cuda")
    gb.dbscan_run_batch(pts, offs, [x.dim for x in inst], [x.eps for x in inst], [x.min_pts for x in inst],
                        mode=gb.MODE_DBSCAN, algo=gb.ALGO_DENSEBOX, labels_out=labels, core_out=core)
    torch.cuda.synchronize()
    gb.stream_status()
    checked = list(range(0, 4096, 16))
    lab_parts = {b: labels[offs[b]:offs[b + 1]].cpu().numpy() for b in checked}
    core_parts = {b: core[offs[b]:offs[b + 1]].cpu().numpy().astype(bool) for b in checked}
    del pts, labels, core

    def one(b):
        x = inst[b]
        assert_matches_oracle(x.points, x.eps, x.min_pts, gb.MODE_DBSCAN, lab_parts[b], core_parts[b])
        return x.n

    # largest instances first, so that the pool ends together
    order = sorted(checked, key=lambda b: -inst[b].n)
    with ThreadPoolExecutor(_threads()) as ex:
        done = sum(ex.map(one, order))
    assert done == sum(inst[b].n for b in checked)
