"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Small and medium inputs are compared with the full oracle clustering: core
and noise sets and core labels exactly, border labels against their valid
sets (tests/parity.py). The full-size 3D halo workload is checked at sampled
points with brute-force neighbourhoods, and the two GPU algorithms must agree.
"""
import numpy as np
import pytest

import oracle
from tests.parity import assert_matches_oracle, check_properties_at_samples
from workloads import blobs, halo_eps, halos, roads, uniform

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


def check(X, eps, mp, mode, algo, ref=None):
    lab, core = run_gpu(X, eps, mp, mode, algo)
    return assert_matches_oracle(X, eps, mp, mode, lab, core, ref), lab, core


# ------------------------------------------------------------ config 0 family

@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_blobs_16k_3d(seed, mode, algo):
    """16384 3D points: 8 Gaussian blobs (sigma 0.02) + 10% noise, eps 0.03,
    minPts 5 (the small 3D workload)."""
    X = blobs(16384, 3, seed)
    check(X, 0.03, 5, mode, algo)


SMALL = []
for s in range(40):
    rs = np.random.default_rng(900 + s)
    SMALL.append((s, int(rs.choice([2, 3])), int(rs.integers(1, 3000)), int(rs.choice([1, 2, 3, 5, 10])),
                  int(rs.integers(0, 2)), float(np.float32(rs.uniform(0.01, 0.1)))))


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("seed,d,n,mp,mode,eps", SMALL)
def test_small_random(seed, d, n, mp, mode, eps, algo):
    X = blobs(n, d, seed, n_blobs=5, sigma=0.03)
    check(X, eps, mp, mode, algo)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("seed", range(8))
def test_lattice_exact_ties_and_duplicates(seed, algo):
    """Integer lattice, eps = 1: many pairs exactly at distance eps, many
    duplicates, dense cells of identical points."""
    rs = np.random.default_rng(77 + seed)
    d = 2 + seed % 2
    X = rs.integers(0, 12, size=(int(rs.integers(100, 4000)), d)).astype(np.float32)
    for mp in (1, 2, 4, 9):
        for mode in MODES:
            check(X, 1.0, mp, mode, algo)


@pytest.mark.parametrize("algo", ALGOS)
def test_edge_cases(algo):
    for mode in MODES:
        # one point
        check(np.zeros((1, 3), np.float32), 0.1, 1, mode, algo)
        check(np.zeros((1, 2), np.float32), 0.1, 2, mode, algo)
        # two points, adjacent and not
        check(np.array([[0, 0], [1, 0]], np.float32), 1.0, 2, mode, algo)
        check(np.array([[0, 0], [1.0000001, 0]], np.float32), 1.0, 2, mode, algo)
        # minPts above n
        check(blobs(500, 3, 5), 0.05, 501, mode, algo)
        # all identical
        check(np.full((777, 3), 0.5, np.float32), 1e-3, 10, mode, algo)
        check(np.full((777, 2), -3.0, np.float32), 1e-3, 778, mode, algo)
        # collinear 2D chain with spacing below eps
        X = np.zeros((1000, 2), np.float32)
        X[:, 0] = np.arange(1000, dtype=np.float32) * 0.5
        check(X, 0.6, 3, mode, algo)
        # ragged tails around the 32-point tile size
        for n in (31, 32, 33, 63, 65, 1023, 1025):
            check(blobs(n, 3, n), 0.08, 3, mode, algo)


def test_empty_input():
    pts = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    lab = gb.dbscan_run(pts, 0.1, 2)
    assert lab.numel() == 0


@pytest.mark.parametrize("algo", ALGOS)
def test_offset_coordinates_tiny_eps(algo):
    """Coordinates near 1e6 with eps of a few ulps: the grid arithmetic of
    DenseBox loses precision (Sec. 4.2); results must stay exact."""
    rs = np.random.default_rng(5)
    base = np.float32(1e6)
    ulp = np.spacing(base)
    X = (base + ulp * rs.integers(0, 40, size=(3000, 3))).astype(np.float32)
    for eps in (float(ulp), float(2.5 * ulp), float(7 * ulp)):
        for mp in (2, 5, 20):
            check(X, eps, mp, gb.MODE_DBSCAN, algo)


@pytest.mark.parametrize("d", [2, 3])
def test_wide_cell_keys(d):
    """DenseBox cells so small against the extent (about 1000 / 1e-7) that
    the cell key takes (nearly) all 64 bits: the key cannot share a word with
    the point index, so the pairs sort (key, index) runs instead of the
    packed keys-only one. Exact duplicates make dense cells; a few points sit
    one ulp (within eps) from another."""
    rs = np.random.default_rng(11)
    base = rs.integers(0, 1 << 10, size=(600, d)).astype(np.float32)
    base[:, 0] = np.float32(0.5) + rs.integers(0, 2048, size=600).astype(np.float32) / np.float32(4096)
    X = np.repeat(base, rs.integers(1, 12, size=600), axis=0)
    near = X[:200].copy()
    near[:, 0] = np.nextafter(near[:, 0], np.float32(2))
    X = np.concatenate([X, near]).astype(np.float32)
    rs.shuffle(X)
    eps = float(np.spacing(np.float32(1)))
    for mp in (2, 4, 9):
        check(X, eps, mp, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX)


@pytest.mark.parametrize("algo", ALGOS + [gb.ALGO_AUTO])
def test_nonfinite_input_is_rejected(algo):
    """A NaN or infinity is found on the device: dbscan_run returns at once,
    writes no label, and the next sync point reports NONFINITE; the stream
    then serves the next run normally."""
    X = blobs(1000, 3, 1)
    # the first call of a kind runs the autotuner, which waits for the
    # device: it reports the error itself
    gb.tuning_clear()
    Y = X.copy()
    Y[3, 0] = np.inf
    with pytest.raises(gb.DbscanError) as e:
        gb.dbscan_run(torch.from_numpy(Y).cuda(), 0.05, 3, algo=algo)
    assert e.value.name == "NONFINITE"
    gb.dbscan_run(torch.from_numpy(X).cuda(), 0.05, 3, algo=algo, sync=True)  # tunes this kind
    X[17, 2] = np.nan
    pts = torch.from_numpy(X).cuda()
    labels = torch.full((1000,), -7, dtype=torch.int32, device="cuda")
    gb.dbscan_run(pts, 0.05, 3, algo=algo, labels_out=labels)  # enqueued, no error yet
    with pytest.raises(gb.DbscanError) as e:
        gb.stream_status()
    assert e.value.name == "NONFINITE"
    assert (labels.cpu().numpy() == -7).all()
    X[17, 2] = np.inf
    with pytest.raises(gb.DbscanError) as e:
        gb.dbscan_run(torch.from_numpy(X).cuda(), 0.05, 3, algo=algo, sync=True)
    assert e.value.name == "NONFINITE"
    with pytest.raises(gb.DbscanError) as e:
        gb.dbscan_run_host(X, 0.05, 3, algo=algo)
    assert e.value.name == "NONFINITE"
    gb.stream_status()  # cleared
    X[17, 2] = 0.5
    check(X, 0.05, 3, gb.MODE_DBSCAN, algo if algo != gb.ALGO_AUTO else gb.ALGO_DENSEBOX)


# ------------------------------------------------------- medium, full oracle

@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("mp", [2, 10])
def test_halos_256k(mp, algo):
    """The 3D cosmology-like family at 2^18 points (eps = 0.2 x mean
    spacing), full oracle comparison."""
    n = 1 << 18
    X = halos(n, 12, n_halos=800)
    check(X, halo_eps(n), mp, gb.MODE_DBSCAN, algo)


@pytest.mark.parametrize("algo", ALGOS)
def test_roads_512k(algo):
    """The 2D GPS-trace-like family at 2^19 points; eps scaled with the
    density so neighbourhoods keep their size."""
    n = 1 << 19
    X = roads(n, 3)
    eps = float(np.float32(2e-4 * (4194304 / n) ** 0.5))
    for mode in MODES:
        check(X, eps, 10, mode, algo)


def test_uniform_2d_and_3d_many_tiles():
    for d, eps in ((2, 0.004), (3, 0.02)):
        X = uniform(200_000, d, 9)
        for algo in ALGOS:
            check(X, eps, 4, gb.MODE_DBSCAN, algo)


# ----------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def halos16m():
    n = 1 << 24
    return halos(n, 2), halo_eps(n)


@pytest.mark.slow
@pytest.mark.parametrize("mp", [10, 2])
def test_halos_16m_sampled(halos16m, mp):
    """The 3D workload at full size (2^24 points, DenseBox, minPts 10 and 2):
    properties at sampled points with brute-force neighbourhoods, and exact
    agreement of the core set and core labels between DenseBox and FDbscan."""
    X, eps = halos16m
    lab, core = run_gpu(X, eps, mp, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX)
    rs = np.random.default_rng(mp)
    # samples: random points plus points in the densest regions (largest clusters)
    samples = list(rs.choice(X.shape[0], 96, replace=False))
    big = np.bincount(lab[lab >= 0]).argsort()[-8:]
    for b in big:
        members = np.nonzero(lab == b)[0]
        samples += list(rs.choice(members, 4, replace=False))
    check_properties_at_samples(X, eps, mp, gb.MODE_DBSCAN, lab, core, samples)
    lab2, core2 = run_gpu(X, eps, mp, gb.MODE_DBSCAN, gb.ALGO_FDBSCAN)
    assert (core == core2).all()
    assert (lab[core] == lab2[core]).all()
    assert ((lab == -1) == (lab2 == -1)).all()


# ---------------------------------------------------------------- interfaces

def test_repeat_runs_are_identical_on_unique_parts():
    X = halos(1 << 17, 4, n_halos=400)
    eps = halo_eps(1 << 17)
    for algo in ALGOS:
        a_lab, a_core = run_gpu(X, eps, 5, gb.MODE_DBSCAN, algo)
        b_lab, b_core = run_gpu(X, eps, 5, gb.MODE_DBSCAN, algo)
        assert (a_core == b_core).all()
        assert (a_lab[a_core] == b_lab[a_core]).all()
        assert ((a_lab == -1) == (b_lab == -1)).all()


def test_host_entry_point_matches_device_entry_point():
    X = blobs(50_000, 3, 8)
    for algo in ALGOS:
        d_lab, d_core = run_gpu(X, 0.02, 5, gb.MODE_DBSCAN_STAR, algo)
        core = np.empty(X.shape[0], np.uint8)
        h_lab, h_core = gb.dbscan_run_host(X, 0.02, 5, mode=gb.MODE_DBSCAN_STAR, algo=algo, core_out=core)
        assert (h_lab == d_lab).all() and (h_core.astype(bool) == d_core).all()


def test_async_host_entry_point_on_two_streams_matches_the_oracle():
    """dbscan_run_host_async: steps alternating between two streams, each
    with its own pinned label buffer, give the oracle's clustering; pageable
    host buffers are refused before anything is enqueued."""
    X = blobs(50_000, 3, 9)
    eps, mp = 0.02, 5
    hx = torch.from_numpy(X).pin_memory()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for algo in ALGOS:
        for mode in (gb.MODE_DBSCAN, gb.MODE_DBSCAN_STAR):
            ref = oracle.dbscan(X, eps, mp, mode)
            labs = [torch.full((X.shape[0],), -7, dtype=torch.int32).pin_memory() for _ in range(4)]
            cores = [torch.zeros(X.shape[0], dtype=torch.uint8).pin_memory() for _ in range(4)]
            for i in range(4):
                gb.dbscan_run_host_async(hx.numpy(), eps, mp, labs[i].numpy(), mode=mode, algo=algo,
                                         core_out=cores[i].numpy(), stream=streams[i % 2])
            for st in streams:
                st.synchronize()
                gb.stream_status(st)
            for i in range(4):
                assert_matches_oracle(X, eps, mp, mode, labs[i].numpy(), cores[i].numpy(), ref=ref)
    lab = np.empty(X.shape[0], np.int32)
    with pytest.raises(gb.DbscanError, match="pinned"):
        gb.dbscan_run_host_async(X, eps, mp, lab, stream=streams[0])


def test_tuning_does_not_change_results():
    X = halos(1 << 16, 6, n_halos=200)
    eps = halo_eps(1 << 16)
    ref = oracle.dbscan(X, eps, 5, 0)
    try:
        for block, f in ((64, 1.0), (512, 0.5), (128, 0.25)):
            gb.set_tuning(block, f)
            for algo in ALGOS:
                check(X, eps, 5, gb.MODE_DBSCAN, algo, ref=ref)
    finally:
        gb.set_tuning(0, 0.0)


# ---------------------------------------------------------------- components

def test_radix_sort_matches_stable_argsort():
    rs = np.random.default_rng(1)
    # key widths at and across the digit boundaries (9-bit digits: 1 to 8
    # passes, the result in either buffer), tiles with a ragged tail
    for n, bits in ((1, 8), (5000, 9), (5000, 10), (4095, 12), (70_001, 27), (4097, 36), (70_001, 45),
                    (70_001, 63), (100_000, 64), (1 << 20, 30)):
        keys = rs.integers(0, 1 << min(bits, 62), size=n, dtype=np.int64)
        if bits == 64:
            keys = rs.integers(-(1 << 62), 1 << 62, size=n, dtype=np.int64)
        keys[::7] = keys[0]  # many duplicates: stability matters
        vals = np.arange(n, dtype=np.int32)
        k = torch.from_numpy(keys.copy()).cuda()
        v = torch.from_numpy(vals.copy()).cuda()
        gb.sort_pairs_u64(k, v, bits)
        ku = keys.view(np.uint64) & np.uint64((1 << bits) - 1 if bits < 64 else 0xFFFFFFFFFFFFFFFF)
        order = np.argsort(ku, kind="stable")
        assert (v.cpu().numpy() == order).all()
        assert (k.cpu().numpy() == keys[order]).all()


def test_morton_codes_match_bit_interleave():
    rs = np.random.default_rng(2)
    for d, bits in ((3, 10), (2, 16), (3, 21), (2, 31)):
        X = rs.uniform(-1, 3, size=(5000, d)).astype(np.float32)
        lo, hi = X.min(0), X.max(0)
        got = gb.morton_codes(torch.from_numpy(X).cuda(), lo, hi, bits).cpu().numpy().view(np.uint64)
        cells = np.float32(2.0 ** bits)
        for i in range(0, 5000, 37):
            c = []
            for k in range(d):
                scale = cells / (hi[k] - lo[k])
                t = np.floor((X[i, k] - lo[k]) * scale)
                c.append(int(min(max(t, 0), 2 ** bits - 1)))
            key = 0
            for b in range(bits):
                for k in range(d):
                    key |= ((c[k] >> b) & 1) << (b * d + k)
            assert int(got[i]) == key


def test_lbvh_topology_reproduces_the_papers_figure():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pair_traversal_figure.json")))
    keys = torch.tensor(g["leaf_keys"], dtype=torch.int64, device="cuda")
    ch, rg = gb.lbvh_topology(keys)
    ch = ch.cpu().numpy()
    m = len(g["leaf_keys"])

    def ref(r):
        return m - 1 + int(r[1:]) if r[0] == "l" else int(r[1:])

    for i, (a, b) in g["internal_children"].items():
        assert tuple(ch[int(i)]) == (ref(a), ref(b)), i


def test_lbvh_topology_invariants():
    rs = np.random.default_rng(3)
    for m in (2, 3, 17, 1000, 65537):
        keys = np.sort(rs.integers(0, 1 << 20, size=m)).astype(np.int64)
        keys[m // 3: m // 3 + m // 5] = keys[m // 3]  # duplicate run
        ch, rg = gb.lbvh_topology(torch.from_numpy(keys).cuda())
        ch, rg = ch.cpu().numpy(), rg.cpu().numpy()
        seen = np.zeros(2 * m - 1, np.int64)
        for i in range(m - 1):
            for c in ch[i]:
                seen[c] += 1
        assert seen[0] == 0 and (seen[1:] == 1).all()  # every node but the root has one parent
        assert tuple(rg[0]) == (0, m - 1)
        for i in range(m - 1):
            lo, hi = rg[i]
            l, r = ch[i]
            llo, lhi = (l - (m - 1),) * 2 if l >= m - 1 else tuple(rg[l])
            rlo, rhi = (r - (m - 1),) * 2 if r >= m - 1 else tuple(rg[r])
            assert llo == lo and rhi == hi and lhi + 1 == rlo


# ---------------------------------------------------------------- boundary

def test_dbscan_run_returns_before_the_device_finishes():
    """dbscan_run only enqueues: right after it returns, an event recorded
    behind its work is still pending on a 2^22-point input (about 2 ms of
    device work), and the results match a synchronous run."""
    n = 1 << 22
    X = halos(n, 7, n_halos=12000)
    eps = halo_eps(n)
    pts = torch.from_numpy(X).cuda()
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    for algo in (gb.ALGO_DENSEBOX, gb.ALGO_FDBSCAN, gb.ALGO_AUTO):
        gb.dbscan_run(pts, eps, 10, algo=algo, labels_out=labels)  # sizes the workspace
        torch.cuda.synchronize()
        pending = 0
        for _ in range(5):
            gb.dbscan_run(pts, eps, 10, algo=algo, labels_out=labels)
            ev = torch.cuda.Event()
            ev.record()
            pending += 0 if ev.query() else 1
            torch.cuda.synchronize()
        assert pending >= 4, f"algo {algo}: the call waited for the device ({pending} of 5 pending)"
        gb.stream_status()
        ref = gb.dbscan_run(pts, eps, 10, algo=algo, sync=True)
        assert torch.equal(ref, labels)


def test_sort_wait_that_runs_out_is_reported_and_the_next_sort_is_correct():
    """The radix sort's bounded look-back wait, made to run out by a test
    hook (the first tile of each pass publishes nothing, so every later
    tile's wait on it ends at a short limit): the sort returns
    DEVICE_TIMEOUT instead of hanging; with the hooks off the next sort is
    exact and reports nothing."""
    rs = np.random.default_rng(31)
    n, bits = 1 << 20, 40
    keys = rs.integers(0, 1 << bits, size=n, dtype=np.int64)
    vals = np.arange(n, dtype=np.int32)
    k = torch.from_numpy(keys.copy()).cuda()
    v = torch.from_numpy(vals.copy()).cuda()
    gb.sort_test_hooks(wait_limit=2000, stall_first_tile=True)
    try:
        with pytest.raises(gb.DbscanError) as e:
            gb.sort_pairs_u64(k, v, bits)
        assert e.value.name == "DEVICE_TIMEOUT"
    finally:
        gb.sort_test_hooks()
    k = torch.from_numpy(keys.copy()).cuda()
    v = torch.from_numpy(vals.copy()).cuda()
    gb.sort_pairs_u64(k, v, bits)
    order = np.argsort(keys, kind="stable")
    assert (v.cpu().numpy() == order).all() and (k.cpu().numpy() == keys[order]).all()
    gb.stream_status()


# ------------------------------------------------- border claims without lists

@pytest.fixture
def no_border_lists():
    gb.set_border_lists(False)
    try:
        yield
    finally:
        gb.set_border_lists(True)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("mode", MODES)
def test_claims_in_the_main_traversal_without_lists(no_border_lists, mode, algo):
    """Border points claimed by core points during the main traversal, with
    no per-point neighbour list (Algorithm 3 as written): blobs, halos,
    roads and lattice ties against the oracle, for minPts from 3 to 40."""
    assert not gb.border_lists()
    check(blobs(16384, 3, 4), 0.03, 5, mode, algo)
    n = 1 << 18
    check(halos(n, 13, n_halos=800), halo_eps(n), 10, mode, algo)
    X = roads(1 << 19, 5)
    check(X, float(np.float32(2e-4 * (4194304 / (1 << 19)) ** 0.5)), 10, mode, algo)
    rs = np.random.default_rng(8)
    L = rs.integers(0, 12, size=(3000, 2)).astype(np.float32)
    for mp in (3, 4, 9, 40):
        check(L, 1.0, mp, mode, algo)


# ---------------------------------------------------------------- autotuner

def test_autotuner_fills_its_table_and_results_stay_exact():
    """dbscan_set_tuning(0, 0): the first call of a kind measures the block
    sizes and cell factors on its data and keeps the fastest; results match
    the oracle on that call and the next, and the next call does not wait
    for the device."""
    gb.set_tuning(0, 0.0)
    gb.tuning_clear()
    n = 1 << 18
    X = halos(n, 21, n_halos=800)
    eps = halo_eps(n)
    assert gb.tuning_lookup(3, n, 10) is None
    ref = check(X, eps, 10, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX)[0]
    entry = gb.tuning_lookup(3, n, 10)
    assert entry is not None
    block, f, ms = entry
    assert block in (64, 128, 256) and f in (1.0, 0.75, 0.5) and ms > 0
    check(X, eps, 10, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX, ref=ref)
    assert gb.tuning_lookup(3, n, 10) == entry
    # FDbscan: block sizes only
    check(X, eps, 10, gb.MODE_DBSCAN, gb.ALGO_FDBSCAN, ref=ref)
    fb = gb.tuning_lookup(3, n, 10, algo=gb.ALGO_FDBSCAN)
    assert fb is not None and fb[1] == 1.0
    # a fixed knob restricts the search
    gb.set_tuning(0, 0.75)
    gb.tuning_clear()
    check(X, eps, 10, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX, ref=ref)
    assert gb.tuning_lookup(3, n, 10)[1] == 0.75
    gb.set_tuning(0, 0.0)


def test_autotuner_for_batches():
    from tests.test_gpu_batch_serve import _check_batch, _concat, _mixed_instances
    gb.set_tuning(0, 0.0)
    gb.tuning_clear()
    inst = _mixed_instances(77)
    flat, offs = _concat(inst)
    pts = torch.from_numpy(flat).cuda()
    total = int(offs[-1])
    labels = torch.empty(total, dtype=torch.int32, device="cuda")
    core = torch.empty(total, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        gb.dbscan_run_batch(pts, offs, [x.dim for x in inst], [x.eps for x in inst], [x.min_pts for x in inst],
                            algo=gb.ALGO_DENSEBOX, labels_out=labels, core_out=core)
        torch.cuda.synchronize()
        gb.stream_status()
        _check_batch(inst, gb.MODE_DBSCAN, gb.ALGO_DENSEBOX, labels.cpu().numpy(), core.cpu().numpy())
    entry = gb.tuning_lookup(0, total, max(x.min_pts for x in inst), batch=True, count=len(inst))
    assert entry is not None and entry[0] in (64, 128, 256)
