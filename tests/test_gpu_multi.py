"""The multi-minPts sweep (one index, one counting pass, one main phase per
minPts): every row must match the oracle for its minPts and agree with a
single dbscan_run for that minPts (core flags, core labels and noise set
identical; border labels valid)."""
import numpy as np
import pytest

import oracle
from tests.parity import assert_matches_oracle
from workloads import blobs, roads

torch = pytest.importorskip("torch")
import paper_2103_05162_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu

ALGOS = [gb.ALGO_FDBSCAN, gb.ALGO_DENSEBOX]
MODES = [gb.MODE_DBSCAN, gb.MODE_DBSCAN_STAR]


def run_multi(X, eps, mps, mode, algo):
    pts = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    lab, core = gb.dbscan_run_multi(pts, eps, mps, mode=mode, algo=algo, want_core=True)
    torch.cuda.synchronize()
    gb.stream_status()
    return lab.cpu().numpy(), core.cpu().numpy().astype(bool)


def run_single(X, eps, mp, mode, algo):
    pts = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    lab, core = gb.dbscan_run(pts, eps, mp, mode=mode, algo=algo, want_core=True)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), core.cpu().numpy().astype(bool)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("mps", [[1, 2, 3, 5, 10], [10, 5, 2], [4], [2, 2, 40], [3, 32, 33]])
def test_sweep_matches_oracle_per_min_pts(mps, mode, algo):
    X = blobs(6000, 3, 3, n_blobs=6, sigma=0.03)
    eps = float(np.float32(0.03))
    lab, core = run_multi(X, eps, mps, mode, algo)
    assert lab.shape == (len(mps), X.shape[0])
    for k, mp in enumerate(mps):
        assert_matches_oracle(X, eps, mp, mode, lab[k], core[k])


@pytest.mark.parametrize("algo", ALGOS)
def test_sweep_agrees_with_single_runs_2d(algo):
    X = roads(60000, 5)
    eps = float(np.float32(2e-4 * (4194304 / 60000) ** 0.5))
    mps = [2, 5, 10, 20]
    lab, core = run_multi(X, eps, mps, gb.MODE_DBSCAN, algo)
    for k, mp in enumerate(mps):
        sl, sc = run_single(X, eps, mp, gb.MODE_DBSCAN, algo)
        np.testing.assert_array_equal(core[k], sc)
        np.testing.assert_array_equal(lab[k][sc], sl[sc])
        np.testing.assert_array_equal(lab[k] == -1, sl == -1)
    # the oracle for the extremes
    for k in (0, len(mps) - 1):
        assert_matches_oracle(X, eps, mps[k], gb.MODE_DBSCAN, lab[k], core[k])


def test_sweep_degenerate_inputs():
    # duplicates (distance 0), a single point, minPts above n
    X = np.zeros((50, 3), np.float32)
    lab, core = run_multi(X, 0.1, [1, 50, 51], gb.MODE_DBSCAN, gb.ALGO_DENSEBOX)
    assert core[0].all() and core[1].all() and not core[2].any()
    assert (lab[0] == 0).all() and (lab[1] == 0).all() and (lab[2] == -1).all()
    one = np.array([[0.5, 0.5]], np.float32)
    lab, core = run_multi(one, 0.1, [1, 2], gb.MODE_DBSCAN, gb.ALGO_FDBSCAN)
    assert lab[:, 0].tolist() == [0, -1] and core[:, 0].tolist() == [True, False]


def test_sweep_equals_oracle_on_lattice_ties():
    # integer lattice with eps exactly 1: many pairs at distance exactly eps
    g = np.stack(np.meshgrid(np.arange(12), np.arange(12), np.arange(3), indexing="ij"), -1).reshape(-1, 3)
    rs = np.random.default_rng(1)
    X = g[rs.random(g.shape[0]) < 0.7].astype(np.float32)
    for algo in ALGOS:
        lab, core = run_multi(X, 1.0, [2, 3, 4, 5, 6, 7], gb.MODE_DBSCAN, algo)
        for k, mp in enumerate([2, 3, 4, 5, 6, 7]):
            ref = oracle.dbscan(X, 1.0, mp, gb.MODE_DBSCAN)
            assert_matches_oracle(X, 1.0, mp, gb.MODE_DBSCAN, lab[k], core[k], ref)
