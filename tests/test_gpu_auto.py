"""The automatic FDbscan / DenseBox choice: the dense-point estimate, the
choice it drives, and parity of the chosen path with the oracle."""
import numpy as np
import pytest

from tests.parity import assert_matches_oracle
from workloads import blobs, roads, uniform

torch = pytest.importorskip("torch")
import paper_2103_05162_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu

WAIT_S = 300.0


@pytest.fixture(autouse=True)
def _default_threshold():
    gb.set_auto_threshold(2)
    gb.set_auto_threshold(3)
    yield
    gb.set_auto_threshold(2)
    gb.set_auto_threshold(3)


def run_auto(X, eps, mp, mode=gb.MODE_DBSCAN):
    pts = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    lab, core = gb.dbscan_run(pts, eps, mp, mode=mode, algo="auto", want_core=True)
    torch.cuda.synchronize()
    algo, frac, _ = gb.last_choice()
    return lab.cpu().numpy(), core.cpu().numpy().astype(bool), algo, frac


def _cells(X, eps):
    """Grid cells of side eps/sqrt(d) from the point-set minimum, as one int64
    per point (float64 cells: points on a boundary may differ from the GPU's
    fp32 cells, hence the tolerances of the tests)."""
    d = X.shape[1]
    c = np.floor((X.astype(np.float64) - X.min(axis=0)) / (eps / np.sqrt(d))).astype(np.int64)
    k = np.zeros(X.shape[0], np.int64)
    for j in range(d):
        k = k * (int(c[:, j].max()) + 1) + c[:, j]
    return k


def exact_dense_share(X, eps, mp):
    """Share of points whose cell holds at least mp points."""
    _, inv, cnt = np.unique(_cells(X, eps), return_inverse=True, return_counts=True)
    return float((cnt[inv.reshape(-1)] >= mp).mean())


def estimator_on_cpu(X, eps, mp, samples=2048):
    """The estimator as the library defines it: strided samples; above 2^22
    points the cells are counted on every (n >> 22)-th point and scaled, the
    sample itself counted once."""
    n = X.shape[0]
    k = _cells(X, eps)
    stride = n >> 22 if n > (1 << 22) else 1
    ck, cc = np.unique(k[::stride], return_counts=True)
    s = min(n, samples)
    idx = (np.arange(s, dtype=np.int64) * n) // s
    pos = np.searchsorted(ck, k[idx])
    hit = (pos < ck.size) & (ck[np.minimum(pos, ck.size - 1)] == k[idx])
    counted = np.where(hit, cc[np.minimum(pos, ck.size - 1)], 0)
    est = 1 + (counted - (idx % stride == 0)) * stride
    return float((est >= mp).mean()), float(est.mean())


def test_dense_blobs_choose_densebox():
    X = blobs(200_000, 3, 4, n_blobs=8, sigma=0.02)
    lab, core, algo, frac = run_auto(X, 0.03, 5)
    assert algo == gb.ALGO_DENSEBOX and frac > 0.5
    assert abs(frac - exact_dense_share(X, 0.03, 5)) < 0.06
    assert_matches_oracle(X, 0.03, 5, gb.MODE_DBSCAN, lab, core)


def test_mean_occupancy_estimate():
    # every point in a cell with exactly 4 points (4 copies of each point of a
    # lattice of pitch 10 eps): the size-biased mean occupancy is 4
    centres = np.stack(np.meshgrid(*[np.arange(20)] * 3, indexing="ij"), -1).reshape(-1, 3) * 1.0
    X = np.repeat(centres, 4, axis=0).astype(np.float32)
    pts = torch.from_numpy(X).cuda()
    gb.dbscan_run(pts, 0.1, 3, algo="auto")
    torch.cuda.synchronize()
    algo, frac, occ = gb.last_choice()
    assert occ == pytest.approx(4.0) and frac == pytest.approx(1.0)


def test_estimate_with_a_subsampled_counting_pass():
    # above 2^22 points the counts come from every stride-th point: uniform
    # data with about 8 points per cell
    n = (1 << 23) + 12345
    X = uniform(n, 3, 8)
    h = (8.0 / n) ** (1 / 3)
    eps = float(np.float32(h * np.sqrt(3.0)))
    pts = torch.from_numpy(X).cuda()
    gb.dbscan_run(pts, eps, 8, algo="auto")
    torch.cuda.synchronize()
    algo, frac, occ = gb.last_choice()
    want_frac, want_occ = estimator_on_cpu(X, eps, 8)
    # the same estimator (cell boundaries may differ by fp32 vs fp64 rounding)
    assert abs(frac - want_frac) < 0.02 and abs(occ - want_occ) < 0.3
    # and an estimate of the exact share (thinning blurs cells near minPts)
    assert abs(frac - exact_dense_share(X, eps, 8)) < 0.2
    assert 7.0 < occ < 11.0  # size-biased mean of 1 + Poisson(8): 9


def test_sparse_uniform_chooses_fdbscan():
    n = 300_000
    X = uniform(n, 3, 5)
    eps = float(np.float32(0.2 * n ** (-1 / 3)))
    lab, core, algo, frac = run_auto(X, eps, 5)
    assert algo == gb.ALGO_FDBSCAN and frac < 0.05
    assert abs(frac - exact_dense_share(X, eps, 5)) < 0.06
    assert_matches_oracle(X, eps, 5, gb.MODE_DBSCAN, lab, core)


@pytest.mark.parametrize("fraction,occupancy,want", [(0.0, 16.0, gb.ALGO_DENSEBOX), (1.0, 1e30, gb.ALGO_FDBSCAN),
                                                     (1.0, 0.0, gb.ALGO_DENSEBOX)])
def test_threshold_extremes(fraction, occupancy, want):
    gb.set_auto_threshold(2, fraction, occupancy)
    X = roads(50_000, 2)
    eps = float(np.float32(2e-4 * (4194304 / 50_000) ** 0.5))
    lab, core, algo, frac = run_auto(X, eps, 10)
    assert algo == want and 0.0 <= frac < 1.0
    assert_matches_oracle(X, eps, 10, gb.MODE_DBSCAN, lab, core)


def test_explicit_algorithm_reports_no_estimate():
    X = blobs(5000, 2, 1)
    pts = torch.from_numpy(X).cuda()
    gb.dbscan_run(pts, 0.03, 5, algo="fdbscan")
    torch.cuda.synchronize()
    assert gb.last_choice() == (gb.ALGO_FDBSCAN, -1.0, -1.0)


def test_auto_jobs_in_the_server_run_alone_and_match():
    jobs = [blobs(3000, 3, s) for s in range(6)]
    with gb.Server(8 << 30, max_slots=2) as srv:
        dev = [torch.from_numpy(x).cuda() for x in jobs]
        torch.cuda.synchronize()
        srv.hold(True)
        ids = [srv.submit(x, 0.03, 5, algo="auto") for x in dev]
        srv.hold(False)
        labs = [srv.wait(j, timeout=WAIT_S).cpu().numpy() for j in ids]
        st = srv.stats()
    assert st["batches"] == 0 and st["single"] == len(jobs)
    for x, lab in zip(jobs, labs):
        import oracle
        olab, ocore = oracle.dbscan(x, 0.03, 5, gb.MODE_DBSCAN)
        np.testing.assert_array_equal(lab[ocore], olab[ocore])
