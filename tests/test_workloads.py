"""The seeded input generators: determinism, shapes, and the recipe's
parameters (the serving schedule in particular)."""
import math

import numpy as np

from workloads import (SERVE_FAMILIES, batch_instances, blobs, halo_eps, halos, roads, serve_pools,
                       serve_schedule)


def test_generators_are_seeded_float32_and_in_range():
    for f, args, d in [(blobs, (5000, 3, 1), 3), (blobs, (5000, 2, 1), 2), (roads, (5000, 1), 2),
                       (halos, (5000, 1, 30), 3)]:
        a, b = f(*args), f(*args)
        assert a.dtype == np.float32 and a.shape == (5000, d) and a.flags.c_contiguous
        np.testing.assert_array_equal(a, b)
    r = roads(20000, 3)
    assert r.min() >= -0.01 and r.max() <= 1.01
    h = halos(20000, 3, n_halos=40)
    assert h.min() >= 0.0 and h.max() <= 1.0


def test_halo_eps_is_a_fifth_of_the_mean_spacing():
    assert halo_eps(1 << 24) == float(np.float32(0.2 / 256))


def test_batch_instances_recipe():
    inst = batch_instances(300, 5)
    sizes = np.array([x.n for x in inst])
    assert sizes.min() >= 1000 and sizes.max() <= 500000
    assert {x.dim for x in inst} == {2, 3}
    assert all(0.01 <= x.eps <= 0.05 for x in inst)
    assert {x.min_pts for x in inst} <= {2, 5, 10}


def test_serve_schedule_recipe():
    pool_n = 100_000
    s = serve_schedule(3000, 500.0, 9, pool_n=pool_n, size_range=(1000, 80_000))
    assert s == serve_schedule(3000, 500.0, 9, pool_n=pool_n, size_range=(1000, 80_000))
    t = np.array([j.arrival_s for j in s])
    assert (np.diff(t) > 0).all()
    # Poisson arrivals: mean inter-arrival 1/rate (loose: 3000 samples)
    assert abs(np.mean(np.diff(t)) - 1 / 500.0) < 0.1 / 500.0
    for j in s:
        assert 1000 <= j.n <= 80_000 and 0 <= j.offset and j.offset + j.n <= pool_n
        assert j.family in SERVE_FAMILIES
        if j.family == "roads":
            assert j.algo == 0 and j.min_pts == 10 and j.pool == "roads"
            assert math.isclose(j.eps, 2e-4 * math.sqrt(4194304 / j.n), rel_tol=1e-6)
        elif j.family == "halos":
            assert j.algo == 1 and j.eps == halo_eps(j.n) and j.pool == "halos"
        elif j.family == "blobs3":
            assert j.algo == 1 and j.min_pts == 5 and j.pool == "blobs3"
        else:
            assert j.pool in ("blobs2", "blobs3") and 0.01 <= j.eps <= 0.05 and j.min_pts in (2, 5, 10)
    assert {j.family for j in s} == set(SERVE_FAMILIES)
    # log-uniform sizes: the median is near the geometric mean of the range
    assert abs(math.log(np.median([j.n for j in s])) - 0.5 * math.log(1000 * 80_000)) < 0.3


def test_serve_pools_shapes():
    p = serve_pools(4000, 1)
    assert p["blobs3"].shape == (4000, 3) and p["blobs2"].shape == (4000, 2)
    assert p["roads"].shape == (4000, 2) and p["halos"].shape == (4000, 3)
