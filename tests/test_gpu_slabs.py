"""Slab-wise (out-of-core) clustering: host points cut into slabs along the
widest axis, each clustered with its eps halo, clusters merged across slabs.
Results must match the oracle and the in-memory run."""
import numpy as np
import pytest

from tests.parity import assert_matches_oracle
from workloads import blobs, halo_eps, halos, roads

torch = pytest.importorskip("torch")
import paper_2103_05162_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu

ALGOS = [gb.ALGO_FDBSCAN, gb.ALGO_DENSEBOX]
MODES = [gb.MODE_DBSCAN, gb.MODE_DBSCAN_STAR]


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("mode", MODES)
def test_many_slabs_match_oracle_3d(mode, algo):
    X = blobs(40_000, 3, 5, n_blobs=12, sigma=0.03)
    for mp in (2, 5, 10):
        lab, core = gb.dbscan_run_slabs(X, 0.02, mp, mode=mode, algo=algo, slab_points=3000)
        assert_matches_oracle(X, 0.02, mp, mode, lab, core)


@pytest.mark.parametrize("algo", ALGOS)
def test_many_slabs_match_oracle_2d_and_5d(algo):
    X = roads(60_000, 3)
    eps = float(np.float32(2e-4 * (4194304 / 60_000) ** 0.5))
    lab, core = gb.dbscan_run_slabs(X, eps, 10, algo=algo, slab_points=5000)
    assert_matches_oracle(X, eps, 10, gb.MODE_DBSCAN, lab, core)
    Y = blobs(20_000, 5, 6, n_blobs=6, sigma=0.03)
    lab, core = gb.dbscan_run_slabs(Y, 0.1, 6, algo=algo, slab_points=2000)
    assert_matches_oracle(Y, 0.1, 6, gb.MODE_DBSCAN, lab, core)


@pytest.mark.parametrize("algo", ALGOS)
def test_slabs_agree_with_the_in_memory_run(algo):
    n = 300_000
    X = halos(n, 11, n_halos=900)
    eps = halo_eps(n)
    lab, core = gb.dbscan_run_slabs(X, eps, 10, algo=algo, slab_points=8000)
    pts = torch.from_numpy(X).cuda()
    ml, mc = gb.dbscan_run(pts, eps, 10, algo=algo, want_core=True)
    ml, mc = ml.cpu().numpy(), mc.cpu().numpy().astype(bool)
    np.testing.assert_array_equal(core, mc)
    np.testing.assert_array_equal(lab[mc], ml[mc])
    np.testing.assert_array_equal(lab == -1, ml == -1)


def test_a_cluster_crossing_every_slab():
    # a chain along x with spacing 0.9 eps: one cluster through all slabs
    n = 20_000
    x = np.arange(n, dtype=np.float64) * 0.9
    rs = np.random.default_rng(2)
    X = np.stack([x, rs.uniform(0, 0.01, n), rs.uniform(0, 0.01, n)], axis=1).astype(np.float32)
    X = X[rs.permutation(n)]
    for mp in (2, 3):
        lab, core = gb.dbscan_run_slabs(X, 1.0, mp, slab_points=500)
        assert_matches_oracle(X, 1.0, mp, gb.MODE_DBSCAN, lab, core)
        assert len(np.unique(lab[core])) == 1


def test_one_slab_and_degenerate_sets():
    X = blobs(5000, 3, 9)
    lab, core = gb.dbscan_run_slabs(X, 0.03, 5)  # default slab size: one slab
    assert_matches_oracle(X, 0.03, 5, gb.MODE_DBSCAN, lab, core)
    same = np.full((3000, 2), 0.25, np.float32)  # zero extent: one bin
    lab, core = gb.dbscan_run_slabs(same, 0.01, 10, slab_points=100)
    assert core.all() and (lab == 0).all()
    bad = blobs(100, 3, 1)
    bad[7, 1] = np.inf
    with pytest.raises(gb.DbscanError):
        gb.dbscan_run_slabs(bad, 0.03, 5)
