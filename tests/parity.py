"""Comparison of a clustering with the oracle's (test helper).

What DBSCAN fixes uniquely is compared exactly: the core set, the noise set
and the label of every core point (labels are canonical: the smallest input
index of a core point of the cluster). A border point may join any cluster
of its core neighbours (Sec. 2.1), so its label is only checked to be one of
those; in DBSCAN* mode border points are noise and everything is exact.
"""
from __future__ import annotations

import numpy as np

import oracle


def assert_matches_oracle(X, eps, min_pts, mode, labels, core, ref=None, sets=None):
    """labels/core: numpy arrays from the CUDA path. ``ref`` (the oracle's
    (labels, core)) and ``sets`` (its border sets, ``oracle.border_sets``) are
    computed when not given. Returns the oracle's (labels, core) for reuse."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    labels = np.asarray(labels, dtype=np.int64)
    core = np.asarray(core).astype(bool)
    if ref is None:
        ref = oracle.dbscan(X, eps, min_pts, mode)
    olab, ocore = ref
    n = X.shape[0]
    assert labels.shape == (n,) and core.shape == (n,)
    bad = np.nonzero(core != ocore)[0]
    assert bad.size == 0, f"core flags differ at {bad.size} points, e.g. {bad[:10].tolist()}"
    bad = np.nonzero(labels[ocore] != olab[ocore])[0]
    assert bad.size == 0, (f"core labels differ at {bad.size} points, e.g. idx "
                           f"{np.nonzero(ocore)[0][bad[:5]].tolist()}")
    noncore = ~ocore
    if mode == oracle.MODE_DBSCAN_STAR:
        assert (labels[noncore] == -1).all(), "DBSCAN*: non-core points must be noise"
        return ref
    bad = np.nonzero((labels[noncore] == -1) != (olab[noncore] == -1))[0]
    assert bad.size == 0, f"noise sets differ at {bad.size} points"
    border = np.nonzero(noncore & (olab >= 0))[0]
    if border.size:
        off, sets = oracle.border_sets(X, eps, ocore, olab) if sets is None else sets
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
        valid = rows * (1 << 32) + sets.astype(np.int64)
        got = border.astype(np.int64) * (1 << 32) + labels[border]
        ok = np.isin(got, valid)
        assert ok.all(), f"{(~ok).sum()} border points got a label outside their valid set"
    return ref


def check_properties_at_samples(X, eps, min_pts, mode, labels, core, samples):
    """Checks that hold at any size, at sampled points, with the oracle's
    brute-force neighbourhoods (for inputs too large to cluster on the CPU):
      * the core flag equals |N_eps| >= minPts;
      * a core point's core neighbours share its label, and its label is the
        label of a core point that labels itself, no larger than its index;
      * a labelled non-core point (DBSCAN) has a core neighbour with the same
        label; a noise point has no core neighbour (DBSCAN) or is non-core
        (DBSCAN*).
    """
    X = np.ascontiguousarray(X, dtype=np.float32)
    labels = np.asarray(labels, dtype=np.int64)
    core = np.asarray(core).astype(bool)
    for q in samples:
        q = int(q)
        nb = oracle.point_neighbors(X, eps, q)
        assert core[q] == (nb.size >= min_pts), f"core flag wrong at {q} ({nb.size} neighbours)"
        cn = nb[core[nb]]
        if core[q]:
            L = labels[q]
            assert L >= 0 and L <= q and core[L] and labels[L] == L, f"bad canonical label at {q}"
            assert (labels[cn] == L).all(), f"core neighbours of {q} carry other labels"
        else:
            if labels[q] == -1:
                if mode == oracle.MODE_DBSCAN:
                    assert cn.size == 0, f"noise point {q} has a core neighbour"
            else:
                assert mode == oracle.MODE_DBSCAN
                assert (labels[cn] == labels[q]).any(), f"border {q} has no core neighbour with its label"
