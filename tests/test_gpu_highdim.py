"""Points of 4 to 8 dimensions (the paper's higher-dimensional sets, Table 1):
parity of both algorithms with the oracle, and of the sweep, the automatic
choice and the host entry point."""
import numpy as np
import pytest

from tests.parity import assert_matches_oracle
from workloads import blobs, uniform

torch = pytest.importorskip("torch")
import paper_2103_05162_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu

ALGOS = [gb.ALGO_FDBSCAN, gb.ALGO_DENSEBOX]
MODES = [gb.MODE_DBSCAN, gb.MODE_DBSCAN_STAR]


def run_gpu(X, eps, mp, mode, algo):
    pts = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    lab, core = gb.dbscan_run(pts, eps, mp, mode=mode, algo=algo, want_core=True)
    torch.cuda.synchronize()
    gb.stream_status()
    return lab.cpu().numpy(), core.cpu().numpy().astype(bool)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("d", [4, 5, 6, 7, 8])
def test_blobs_match_oracle(d, mode, algo):
    X = blobs(4000, d, 10 + d, n_blobs=6, sigma=0.03)
    eps = float(np.float32(0.04 * np.sqrt(d)))
    for mp in (2, 5, 12):
        lab, core = run_gpu(X, eps, mp, mode, algo)
        assert_matches_oracle(X, eps, mp, mode, lab, core)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("d", [5, 7])
def test_lattice_ties_and_duplicates(d, algo):
    # exact distances: pairs at exactly eps, duplicates, minPts = 1 isolated points
    rs = np.random.default_rng(d)
    X = rs.integers(0, 3, size=(2500, d)).astype(np.float32)
    for mp in (1, 3, 8):
        lab, core = run_gpu(X, 1.0, mp, gb.MODE_DBSCAN, algo)
        assert_matches_oracle(X, 1.0, mp, gb.MODE_DBSCAN, lab, core)


@pytest.mark.parametrize("algo", ALGOS)
def test_larger_5d_set_spanning_many_tiles(algo):
    X = np.concatenate([blobs(50_000, 5, 3, n_blobs=20, sigma=0.02), uniform(10_000, 5, 4)]).astype(np.float32)
    eps = float(np.float32(0.05))
    lab, core = run_gpu(X, eps, 10, gb.MODE_DBSCAN, algo)
    assert_matches_oracle(X, eps, 10, gb.MODE_DBSCAN, lab, core)


def test_algorithms_agree_on_400k_5d_points():
    X = np.concatenate([blobs(300_000, 5, 8, n_blobs=40, sigma=0.02), uniform(100_000, 5, 9)]).astype(np.float32)
    eps = float(np.float32(0.03))
    lf, cf = run_gpu(X, eps, 10, gb.MODE_DBSCAN, gb.ALGO_FDBSCAN)
    ld, cd = run_gpu(X, eps, 10, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX)
    np.testing.assert_array_equal(cf, cd)
    np.testing.assert_array_equal(lf[cf], ld[cd])
    np.testing.assert_array_equal(lf == -1, ld == -1)


def test_sweep_auto_and_host_entry_in_high_dims():
    X = blobs(5000, 5, 21, n_blobs=5, sigma=0.03)
    eps = float(np.float32(0.09))
    pts = torch.from_numpy(X).cuda()
    lab, core = gb.dbscan_run_multi(pts, eps, [2, 6, 15], want_core=True)
    torch.cuda.synchronize()
    for k, mp in enumerate([2, 6, 15]):
        assert_matches_oracle(X, eps, mp, gb.MODE_DBSCAN, lab[k].cpu().numpy(), core[k].cpu().numpy())
    Y = blobs(5000, 7, 22, n_blobs=5, sigma=0.03)
    eps7 = float(np.float32(0.11))
    la, ca = run_gpu(Y, eps7, 5, gb.MODE_DBSCAN, gb.ALGO_AUTO)
    assert_matches_oracle(Y, eps7, 5, gb.MODE_DBSCAN, la, ca)
    hl = gb.dbscan_run_host(Y, eps7, 5)
    assert_matches_oracle(Y, eps7, 5, gb.MODE_DBSCAN, hl, ca)


def test_batches_refuse_high_dims():
    X = blobs(100, 5, 1)
    pts = torch.from_numpy(X.ravel().copy()).cuda()
    with pytest.raises(gb.DbscanError):
        gb.dbscan_run_batch(pts, np.array([0, 100]), [5], [0.1], [3])
