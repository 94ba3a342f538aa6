"""Pins for the CPU oracle: it is checked against what the paper's definition
(Sec. 2.1) and plain mathematics fix, never against itself.

* an O(n^2) brute force written independently here (numpy fp32 arithmetic,
  scipy connected components) on many small seeded inputs;
* closed forms: chains, isolated points, minPts = 1, minPts > n, duplicates,
  minPts = 2 equals connected components of the eps-graph (Sec. 2.1);
* the bridging hazard of Sec. 3.2 (a border point within eps of two clusters
  must not merge them);
* exactly representable boundary pairs and a rounding witness showing the
  distance test is the fp32 squared form without fused multiply-add.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

import oracle
from workloads import blobs, uniform


# ---------------------------------------------------------------- brute force

def _adjacency(X: np.ndarray, eps: float) -> np.ndarray:
    """All-pairs fp32 squared distances compared with fp32 eps^2 (numpy
    evaluates each elementwise operation with one rounding, no contraction)."""
    X = np.asarray(X, dtype=np.float32)
    e2 = np.float32(eps) * np.float32(eps)
    d = X.shape[1]
    diff = X[:, None, 0] - X[None, :, 0]
    s = diff * diff
    for k in range(1, d):
        diff = X[:, None, k] - X[None, :, k]
        s = s + diff * diff
    return s <= e2


def brute_force(X, eps, min_pts, mode):
    """Returns (core bool[n], core labels int[n] (-1 for non-core), valid
    label sets per non-core point)."""
    n = X.shape[0]
    A = _adjacency(X, eps)
    core = A.sum(axis=1) >= min_pts
    labels = np.full(n, -1, dtype=np.int64)
    idx = np.nonzero(core)[0]
    if idx.size:
        sub = csr_matrix(A[np.ix_(idx, idx)])
        ncomp, comp = connected_components(sub, directed=False)
        first = np.full(ncomp, n, dtype=np.int64)
        np.minimum.at(first, comp, idx)
        labels[idx] = first[comp]
    valid = {}
    for i in np.nonzero(~core)[0]:
        nb = np.nonzero(A[i] & core)[0]
        valid[int(i)] = sorted(set(int(labels[j]) for j in nb))
    return core, labels, valid


def check_against_brute(X, eps, min_pts, mode):
    lab, core = oracle.dbscan(X, eps, min_pts, mode)
    bcore, blab, valid = brute_force(X, eps, min_pts, mode)
    np.testing.assert_array_equal(core, bcore)
    np.testing.assert_array_equal(lab[bcore], blab[bcore])
    for i, v in valid.items():
        if mode == oracle.MODE_DBSCAN_STAR or not v:
            assert lab[i] == -1, (i, v, lab[i])
        else:
            assert lab[i] == min(v), (i, v, lab[i])
    if mode == oracle.MODE_DBSCAN:
        off, sets = oracle.border_sets(X, eps, core, lab)
        for i, v in valid.items():
            assert list(sets[off[i]:off[i + 1]]) == v
        for i in np.nonzero(bcore)[0]:
            assert off[i] == off[i + 1]
    return lab, core


CASES = []
for seed in range(120):
    rs = np.random.default_rng(1000 + seed)
    d = int(rs.choice([2, 3]))
    n = int(rs.integers(1, 500))
    mp = int(rs.choice([1, 2, 3, 5, 10]))
    mode = int(rs.integers(0, 2))
    eps = float(np.float32(rs.uniform(0.01, 0.12)))
    CASES.append((seed, d, n, mp, mode, eps))


@pytest.mark.parametrize("seed,d,n,mp,mode,eps", CASES)
def test_oracle_matches_brute_force_blobs(seed, d, n, mp, mode, eps):
    X = blobs(n, d, seed, n_blobs=4, sigma=0.03)
    check_against_brute(X, eps, mp, mode)


@pytest.mark.parametrize("seed", range(60))
def test_oracle_matches_brute_force_lattice(seed):
    """Integer lattice points with eps = 1: many pairs sit exactly at distance
    eps (adjacent) or sqrt(2) (not), and duplicates are frequent."""
    rs = np.random.default_rng(5000 + seed)
    d = int(rs.choice([2, 3]))
    n = int(rs.integers(2, 400))
    X = rs.integers(0, 8, size=(n, d)).astype(np.float32)
    mp = int(rs.choice([1, 2, 3, 4, 6, 9]))
    for mode in (0, 1):
        check_against_brute(X, 1.0, mp, mode)


HD_CASES = []
for seed in range(40):
    rs = np.random.default_rng(3000 + seed)
    d = int(rs.integers(4, 9))
    n = int(rs.integers(1, 400))
    mp = int(rs.choice([1, 2, 3, 5, 10]))
    mode = int(rs.integers(0, 2))
    # blobs of sigma 0.03 per axis: typical pair distances grow like sqrt(d)
    eps = float(np.float32(rs.uniform(0.02, 0.1) * np.sqrt(d)))
    HD_CASES.append((seed, d, n, mp, mode, eps))


@pytest.mark.parametrize("seed,d,n,mp,mode,eps", HD_CASES)
def test_oracle_matches_brute_force_4_to_8_dims(seed, d, n, mp, mode, eps):
    """Points of 4 to 8 dimensions (the paper's higher-dimensional sets,
    Table 1): the 3^d cells of the oracle's grid against all pairs."""
    X = blobs(n, d, seed, n_blobs=4, sigma=0.03)
    check_against_brute(X, eps, mp, mode)


@pytest.mark.parametrize("seed", range(12))
def test_oracle_matches_brute_force_lattice_5_and_7_dims(seed):
    rs = np.random.default_rng(6000 + seed)
    d = 5 if seed % 2 else 7
    n = int(rs.integers(2, 300))
    X = rs.integers(0, 3, size=(n, d)).astype(np.float32)
    for mode in (0, 1):
        check_against_brute(X, 1.0, int(rs.choice([1, 2, 3, 5])), mode)


@pytest.mark.parametrize("seed", range(20))
def test_oracle_matches_brute_force_offset_coordinates(seed):
    """Coordinates near 1e3 with a small eps: differences are rounded."""
    rs = np.random.default_rng(7000 + seed)
    n = 300
    X = (1000.0 + rs.uniform(0, 0.05, size=(n, 3))).astype(np.float32)
    eps = float(np.float32(rs.uniform(0.002, 0.006)))
    check_against_brute(X, eps, int(rs.choice([2, 4, 7])), int(seed % 2))


# ---------------------------------------------------------------- closed forms

def test_chain_below_eps_is_one_cluster():
    k = 50
    X = np.zeros((k, 3), dtype=np.float32)
    X[:, 0] = np.arange(k, dtype=np.float32) * 0.5
    for mp in (1, 2):
        lab, core = oracle.dbscan(X, 0.6, mp)
        assert (lab == 0).all() and core.all()
    lab, core = oracle.dbscan(X, 0.6, 3)
    # interior points have 3 neighbours (itself + 2), the two ends only 2:
    # the ends are border points of the one cluster, labelled by the smallest
    # core index, 1
    assert core[1:-1].all() and not core[0] and not core[-1]
    assert (lab == 1).all()
    lab, core = oracle.dbscan(X, 0.6, 4)
    assert (lab == -1).all()


def test_isolated_points_are_noise_unless_minpts_is_one():
    X = np.arange(40, dtype=np.float32).reshape(-1, 2) * 10.0
    lab, core = oracle.dbscan(X, 1.0, 2)
    assert (lab == -1).all() and not core.any()
    lab, core = oracle.dbscan(X, 1.0, 1)
    assert core.all()
    np.testing.assert_array_equal(lab, np.arange(X.shape[0]))


def test_minpts_above_n_is_all_noise():
    X = blobs(200, 3, 3)
    lab, core = oracle.dbscan(X, 10.0, 201)
    assert (lab == -1).all() and not core.any()
    lab, core = oracle.dbscan(X, 10.0, 200)
    assert (lab == 0).all() and core.all()


def test_identical_points():
    X = np.full((64, 2), 0.25, dtype=np.float32)
    lab, core = oracle.dbscan(X, 1e-6, 64)
    assert (lab == 0).all() and core.all()
    lab, core = oracle.dbscan(X, 1e-6, 65)
    assert (lab == -1).all()


def test_minpts_two_is_connected_components_of_eps_graph():
    """Sec. 2.1: with minPts = 2 DBSCAN reduces to the components of the
    eps-graph; points without a neighbour are noise, and there are no border
    points."""
    for seed in range(10):
        X = blobs(700, 2 + seed % 2, 40 + seed, sigma=0.05)
        eps = 0.02
        lab, core = oracle.dbscan(X, eps, 2)
        A = _adjacency(X, eps)
        ncomp, comp = connected_components(csr_matrix(A), directed=False)
        sizes = np.bincount(comp)
        single = sizes[comp] == 1
        assert ((lab == -1) == single).all()
        assert (core == ~single).all()
        for c in range(ncomp):
            members = np.nonzero(comp == c)[0]
            if members.size > 1:
                assert (lab[members] == members.min()).all()


def test_dbscan_star_core_part_equals_dbscan():
    X = blobs(1500, 3, 11)
    lab, core = oracle.dbscan(X, 0.03, 5, oracle.MODE_DBSCAN)
    lab2, core2 = oracle.dbscan(X, 0.03, 5, oracle.MODE_DBSCAN_STAR)
    np.testing.assert_array_equal(core, core2)
    np.testing.assert_array_equal(lab[core], lab2[core])
    assert (lab2[~core] == -1).all()
    assert (lab[~core] >= 0).any()  # the case has border points


def test_bridging_border_point_does_not_merge_clusters():
    """Sec. 3.2: a border point within eps of two clusters joins one of them
    and never merges them."""
    a = np.array([[0.0, 0.0], [0.1, 0.0], [0.0, 0.1], [0.1, 0.1]], dtype=np.float32)
    b = a + np.float32(2.0)
    # x is within eps = 1.5 of a[3] = (0.1, 0.1) and of b[0] = (2, 2) only
    x = np.array([[1.05, 1.05]], dtype=np.float32)
    X = np.concatenate([a, b, x])
    lab, core = oracle.dbscan(X, 1.4, 4)
    assert core[:8].all() and not core[8]
    assert (lab[:4] == 0).all() and (lab[4:8] == 4).all()
    assert lab[8] == 0
    off, sets = oracle.border_sets(X, 1.4, core, lab)
    assert list(sets[off[8]:off[9]]) == [0, 4]


def test_labels_are_smallest_core_index():
    X = blobs(3000, 2, 21)
    lab, core = oracle.dbscan(X, 0.02, 6)
    for l in np.unique(lab[lab >= 0]):
        members = np.nonzero((lab == l) & core)[0]
        assert members.min() == l


def test_empty_and_single():
    lab, core = oracle.dbscan(np.zeros((0, 3), np.float32), 0.1, 2)
    assert lab.shape == (0,)
    lab, core = oracle.dbscan(np.zeros((1, 3), np.float32), 0.1, 1)
    assert lab.tolist() == [0] and core.tolist() == [True]
    lab, core = oracle.dbscan(np.zeros((1, 3), np.float32), 0.1, 2)
    assert lab.tolist() == [-1]


def test_rejects_bad_arguments():
    X = uniform(10, 3, 0)
    for eps in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(ValueError):
            oracle.dbscan(X, eps, 2)
    with pytest.raises(ValueError):
        oracle.dbscan(X, 0.1, 0)
    Y = X.copy()
    Y[3, 1] = np.nan
    with pytest.raises(ValueError):
        oracle.dbscan(Y, 0.1, 2)


# ----------------------------------------------------------- distance rounding

def test_exact_boundary_pairs():
    one_up = float(np.nextafter(np.float32(1.0), np.float32(2.0)))
    assert oracle.adjacent([0, 0], [1, 0], 1.0)
    assert not oracle.adjacent([0, 0], [one_up, 0], 1.0)
    assert oracle.adjacent([0, 0, 0], [3, 4, 0], 5.0)  # 9 + 16 = 25 exactly
    assert oracle.adjacent([0, 0, 0], [2, 3, 6], 7.0)  # 4 + 9 + 36 = 49
    below = float(np.nextafter(np.float32(7.0), np.float32(0.0)))
    assert not oracle.adjacent([0, 0, 0], [2, 3, 6], below)
    # symmetry: fl(a - b) = -fl(b - a)
    rs = np.random.default_rng(3)
    for _ in range(200):
        p, q = rs.uniform(-1, 1, size=(2, 3)).astype(np.float32)
        assert oracle.dist2(p, q) == oracle.dist2(q, p)


def _round_f32(q: Fraction) -> np.float32:
    """Correct round-to-nearest-even of a rational to fp32."""
    f = np.float32(float(q))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]

    def key(c):
        return (abs(Fraction(float(c)) - q), int(np.array(c, np.float32).view(np.uint32)) & 1)
    return min(cands, key=key)


def test_distance_is_fp32_squared_form_without_fma():
    """Search pairs near the eps boundary for ones where (a) the stated
    rounded formula and (b) a fused multiply-add of the second term, or (c)
    the exact real distance, give different answers; the oracle must follow
    (a) on all of them, and such witnesses must exist."""
    rs = np.random.default_rng(12345)
    eps = np.float32(0.001)
    e2 = eps * eps
    fma_witness = exact_witness = 0
    for _ in range(20000):
        ang = rs.uniform(0, 2 * np.pi)
        r = eps * (1.0 + rs.uniform(-3e-7, 3e-7))
        p = rs.uniform(0, 1, size=2).astype(np.float32)
        q = (p + np.array([r * np.cos(ang), r * np.sin(ang)])).astype(np.float32)
        d0 = p[0] - q[0]
        d1 = p[1] - q[1]
        t = d0 * d0
        rounded = (t + d1 * d1) <= e2
        fused = _round_f32(Fraction(float(d1)) ** 2 + Fraction(float(t))) <= e2
        exact = (Fraction(float(p[0])) - Fraction(float(q[0]))) ** 2 + \
                (Fraction(float(p[1])) - Fraction(float(q[1]))) ** 2 <= Fraction(float(eps)) ** 2
        if rounded != fused or rounded != exact:
            got = oracle.adjacent(p, q, float(eps))
            assert got == bool(rounded)
            fma_witness += int(rounded != fused)
            exact_witness += int(rounded != exact)
    assert fma_witness > 0 and exact_witness > 0


# ------------------------------------------------- per-point brute-force rows

def _check_point_neighbors(X, eps, queries):
    A = _adjacency(X, eps)
    for q in queries:
        q = int(q)
        got = oracle.point_neighbors(X, eps, q)
        want = np.nonzero(A[q])[0]
        np.testing.assert_array_equal(got, want)
        assert q in got  # x is its own neighbour (Sec. 2.1: N_eps(x) contains x)


@pytest.mark.parametrize("seed", range(30))
def test_point_neighbors_matches_all_pairs_row(seed):
    """point_neighbors (the checker of the sampled large-input tests) equals
    the row of the independent numpy adjacency: blobs in 2D to 8D, the point
    itself included, indices increasing."""
    rs = np.random.default_rng(8000 + seed)
    d = int(rs.integers(2, 9))
    n = int(rs.integers(1, 600))
    X = blobs(n, d, seed, n_blobs=3, sigma=0.03)
    eps = float(np.float32(rs.uniform(0.02, 0.08) * np.sqrt(d)))
    _check_point_neighbors(X, eps, rs.integers(0, n, size=min(n, 25)))


@pytest.mark.parametrize("seed", range(10))
def test_point_neighbors_lattice_ties_duplicates_and_offsets(seed):
    """Pairs exactly at distance eps (adjacent), at sqrt(2) eps (not),
    duplicated points (distance 0), and coordinates near 1e3 whose
    differences are rounded."""
    rs = np.random.default_rng(8500 + seed)
    d = 2 + seed % 2
    X = rs.integers(0, 6, size=(int(rs.integers(20, 300)), d)).astype(np.float32)
    X[1::7] = X[0]  # many copies of one point
    _check_point_neighbors(X, 1.0, range(X.shape[0]))
    Y = (1000.0 + rs.uniform(0, 0.05, size=(250, 3))).astype(np.float32)
    _check_point_neighbors(Y, float(np.float32(0.004)), range(0, 250, 3))


def test_point_neighbors_boundary_pair_and_isolated_point():
    one_up = float(np.nextafter(np.float32(1.0), np.float32(2.0)))
    X = np.array([[0, 0], [1, 0], [0, one_up], [5, 5]], dtype=np.float32)
    assert oracle.point_neighbors(X, 1.0, 0).tolist() == [0, 1]
    assert oracle.point_neighbors(X, 1.0, 2).tolist() == [2]
    assert oracle.point_neighbors(X, 1.0, 3).tolist() == [3]
