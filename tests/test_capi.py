"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/gbdbscan.h declares, and argument errors are
reported before anything touches the device."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import paper_2103_05162_gb300 as gb
from paper_2103_05162_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(dbscan_[A-Za-z0-9_]+)\s*\(", text,
                             flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return gb.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dbscan_run", "dbscan_run_batch", "dbscan_run_host", "dbscan_server_create",
                 "dbscan_server_submit", "dbscan_server_poll", "dbscan_server_wait", "dbscan_server_destroy",
                 "dbscan_last_error", "dbscan_set_tuning"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_built_for_sm103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert "--fmad=false" in _build.FLAGS


def _run(lib, pts, n, dim, eps, mp, mode=0, algo=1, labels=1):
    return lib.dbscan_run(ctypes.c_void_p(pts), n, dim, eps, mp, mode, algo,
                          ctypes.c_void_p(labels) if labels else None, None, None)


def test_argument_errors_are_reported_without_device_work(lib):
    P = 0x1000  # never dereferenced: every call below fails its argument check
    assert _run(lib, P, 10, 9, 0.1, 2) == 1
    assert _run(lib, P, 10, 1, 0.1, 2) == 1
    assert b"dim" in lib.dbscan_last_error()
    assert _run(lib, P, 10, 3, 0.0, 2) == 1
    assert _run(lib, P, 10, 3, float("inf"), 2) == 1
    assert _run(lib, P, 10, 3, float("nan"), 2) == 1
    assert _run(lib, P, 10, 3, 0.1, 0) == 1
    assert b"min_pts" in lib.dbscan_last_error()
    assert _run(lib, P, 10, 3, 0.1, 2, mode=7) == 1
    assert _run(lib, P, 10, 3, 0.1, 2, algo=9) == 1
    assert _run(lib, P, -1, 3, 0.1, 2) == 1
    assert _run(lib, P, 1 << 30, 3, 0.1, 2) == 1
    assert _run(lib, 0, 10, 3, 0.1, 2) == 1
    assert _run(lib, P, 10, 3, 0.1, 2, labels=0) == 1
    # n == 0 is a valid no-op
    assert _run(lib, 0, 0, 3, 0.1, 2, labels=0) == 0


def test_tuning_validation(lib):
    assert lib.dbscan_set_tuning(0, 0.0) == 0
    assert lib.dbscan_set_tuning(33, 0.0) == 1
    assert lib.dbscan_set_tuning(2048, 0.0) == 1
    assert lib.dbscan_set_tuning(0, 1.5) == 1
    assert lib.dbscan_set_tuning(128, 0.5) == 0
    assert lib.dbscan_set_tuning(0, 0.0) == 0


def test_auto_choice_arguments(lib):
    assert lib.dbscan_set_auto_threshold(3, -0.1, 16.0) == 1
    assert lib.dbscan_set_auto_threshold(3, 1.5, 16.0) == 1
    assert lib.dbscan_set_auto_threshold(3, float("nan"), 16.0) == 1
    assert lib.dbscan_set_auto_threshold(3, 0.3, -1.0) == 1
    assert lib.dbscan_set_auto_threshold(3, 0.3, float("inf")) == 1
    assert lib.dbscan_set_auto_threshold(9, 0.3, 16.0) == 1
    assert lib.dbscan_set_auto_threshold(5, 0.3, 16.0) == 0
    assert lib.dbscan_set_auto_threshold(2, 0.3, 16.0) == 0
    assert lib.dbscan_set_auto_threshold(3, -1.0, -1.0) == 0  # defaults
    assert lib.dbscan_last_choice(None, None, None) == 1
    # the automatic choice is accepted by single runs, refused by batches
    P = 0x1000
    assert _run(lib, P, 10, 9, 0.1, 2, algo=2) == 1 and b"dim" in lib.dbscan_last_error()
    off = np.array([0, 5], dtype=np.int64)
    dims = np.array([3], dtype=np.int32)
    eps = np.array([0.1], dtype=np.float32)
    mp = np.array([2], dtype=np.int32)
    st = lib.dbscan_run_batch(ctypes.c_void_p(P), off.ctypes.data, dims.ctypes.data, eps.ctypes.data,
                              mp.ctypes.data, 1, 0, 2, ctypes.c_void_p(P), None, None)
    assert st == 1 and b"explicit algorithm" in lib.dbscan_last_error()


def test_batch_argument_errors(lib):
    off = np.array([0, 5, 3], dtype=np.int64)
    dims = np.array([3, 3], dtype=np.int32)
    eps = np.array([0.1, 0.1], dtype=np.float32)
    mp = np.array([2, 2], dtype=np.int32)
    st = lib.dbscan_run_batch(ctypes.c_void_p(0x1000), off.ctypes.data, dims.ctypes.data, eps.ctypes.data,
                              mp.ctypes.data, 2, 0, 1, ctypes.c_void_p(0x1000), None, None)
    assert st == 1 and b"non-decreasing" in lib.dbscan_last_error()
    off = np.array([1, 5, 9], dtype=np.int64)
    st = lib.dbscan_run_batch(ctypes.c_void_p(0x1000), off.ctypes.data, dims.ctypes.data, eps.ctypes.data,
                              mp.ctypes.data, 2, 0, 1, ctypes.c_void_p(0x1000), None, None)
    assert st == 1
    assert lib.dbscan_run_batch(None, None, None, None, None, 0, 0, 1, None, None, None) == 0


def test_multi_argument_errors(lib):
    P = ctypes.c_void_p(0x1000)
    mp = np.array([2, 0, 5], dtype=np.int32)
    st = lib.dbscan_run_multi(P, 10, 3, 0.1, mp.ctypes.data, 3, 0, 1, P, None, None)
    assert st == 1 and b"min_pts[1]" in lib.dbscan_last_error()
    mp = np.array([2, 5], dtype=np.int32)
    assert lib.dbscan_run_multi(P, 10, 9, 0.1, mp.ctypes.data, 2, 0, 1, P, None, None) == 1
    assert lib.dbscan_run_multi(P, 10, 3, 0.1, None, 2, 0, 1, P, None, None) == 1
    assert lib.dbscan_run_multi(P, 10, 3, 0.1, mp.ctypes.data, -1, 0, 1, P, None, None) == 1
    assert lib.dbscan_run_multi(P, 10, 3, 0.1, mp.ctypes.data, 5000, 0, 1, P, None, None) == 1
    # nothing to do
    assert lib.dbscan_run_multi(P, 10, 3, 0.1, None, 0, 0, 1, P, None, None) == 0
    assert lib.dbscan_run_multi(None, 0, 3, 0.1, mp.ctypes.data, 2, 0, 1, None, None, None) == 0


def test_slab_argument_errors(lib):
    H = np.zeros(30, np.float32)
    lab = np.zeros(10, np.int32)
    core = np.zeros(10, np.uint8)
    run = lambda n, dim, pts, l, c, sp: lib.dbscan_run_slabs(  # noqa: E731
        pts, n, dim, 0.1, 3, 0, 1, l, c, sp, None)
    assert run(1 << 31, 3, H.ctypes.data, lab.ctypes.data, core.ctypes.data, 0) == 1
    assert run(10, 9, H.ctypes.data, lab.ctypes.data, core.ctypes.data, 0) == 1
    assert run(10, 3, H.ctypes.data, lab.ctypes.data, None, 0) == 1 and b"core" in lib.dbscan_last_error()
    assert run(10, 3, H.ctypes.data, lab.ctypes.data, core.ctypes.data, -5) == 1
    assert run(0, 3, None, None, None, 0) == 0


def test_server_argument_errors(lib):
    h = ctypes.c_void_p()
    assert lib.dbscan_server_create(0, 4, ctypes.byref(h)) == 1
    assert lib.dbscan_server_create(1 << 30, 0, ctypes.byref(h)) == 1
    assert lib.dbscan_server_poll(None, 1, None, None) == 1


def test_async_host_entry_point_refuses_bad_arguments_and_pageable_buffers(lib):
    """dbscan_run_host_async: argument errors, and host buffers that are not
    page-locked (plain numpy arrays), are returned before anything is
    enqueued."""
    pts = np.zeros((16, 3), np.float32)
    lab = np.zeros(16, np.int32)
    vp = ctypes.c_void_p

    def run(n, dim, eps, mp, labels=True):
        return lib.dbscan_run_host_async(vp(pts.ctypes.data), n, dim, eps, mp, 0, 1,
                                         vp(lab.ctypes.data) if labels else None, None, None)

    assert run(16, 9, 0.1, 2) == 1
    assert run(16, 3, 0.0, 2) == 1
    assert run(16, 3, 0.1, 0) == 1
    assert run(16, 3, 0.1, 2, labels=False) == 1
    assert run(0, 3, 0.1, 2) == 0  # nothing to do
    assert run(16, 3, 0.1, 2) == 1
    assert b"pinned" in lib.dbscan_last_error()


def test_component_argument_errors(lib):
    assert lib.dbscan_sort_pairs_u64(None, None, 10, 8, None) == 1
    assert lib.dbscan_sort_pairs_u64(None, None, 10, 65, None) == 1
    assert lib.dbscan_lbvh_topology(None, 1, None, None, None) == 1
    lo = np.zeros(3, np.float32)
    assert lib.dbscan_morton_codes(None, 10, 3, lo.ctypes.data, lo.ctypes.data, 22, None, None) == 1


def test_pair_mask_rule_on_the_papers_figure():
    """Sec. 4.1, Figure 'pair traversal': with the rule 'never enter a subtree
    whose leaves all have index <= i', the thread of leaf 4 visits internal
    nodes 0, 4, 5, 6 and sees leaves 5, 6, 7 only."""
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "pair_traversal_figure.json")))
    ch = {int(k): v for k, v in g["internal_children"].items()}

    def last_leaf(ref):
        if ref[0] == "l":
            return int(ref[1:])
        return max(last_leaf(c) for c in ch[int(ref[1:])])

    i = g["query_leaf"]
    seen, visited, stack = [], [], ["n0"]
    while stack:
        ref = stack.pop()
        if last_leaf(ref) <= i:
            continue
        if ref[0] == "l":
            seen.append(int(ref[1:]))
        else:
            visited.append(int(ref[1:]))
            stack.extend(reversed(ch[int(ref[1:])]))
    assert sorted(seen) == g["visible_leaves"]
    assert sorted(visited) == g["visited_internal_nodes"]
