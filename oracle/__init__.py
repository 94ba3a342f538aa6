"""CPU DBSCAN oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library in
``paper_2103_05162_gb300``) never imports it and shares no code with it.

The computation lives in ``dbscan_oracle.c`` (plain C, fp32 distance test with
no contraction): DBSCAN as defined in Sec. 2.1 of the paper, with canonical
labels (smallest input index of a core point per cluster, -1 for noise).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dbscan_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_DBSCAN = 0
MODE_DBSCAN_STAR = 1


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, i32, f32 = ctypes.c_int64, ctypes.c_int, ctypes.c_float
            vp = ctypes.c_void_p
            lib.oracle_dbscan.argtypes = [vp, i64, i32, f32, i32, i32, vp, vp]
            lib.oracle_dbscan.restype = i32
            lib.oracle_border_sets.argtypes = [vp, i64, i32, f32, vp, vp, vp, vp, i64]
            lib.oracle_border_sets.restype = i64
            lib.oracle_point_neighbors.argtypes = [vp, i64, i32, f32, i64, vp, i64]
            lib.oracle_point_neighbors.restype = i64
            lib.oracle_adjacent.argtypes = [vp, vp, i32, f32]
            lib.oracle_adjacent.restype = i32
            lib.oracle_dist2.argtypes = [vp, vp, i32]
            lib.oracle_dist2.restype = f32
            _lib = lib
    return _lib


def _points(X) -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
    if X.ndim != 2:
        raise ValueError("points must be an (n, d) array")
    return X


def dbscan(X, eps: float, min_pts: int, mode: int = MODE_DBSCAN):
    """Returns ``(labels int32[n], core bool[n])``."""
    X = _points(X)
    n, d = X.shape
    labels = np.empty(n, dtype=np.int32)
    core = np.empty(n, dtype=np.uint8)
    rc = _load().oracle_dbscan(X.ctypes.data, n, d, float(eps), int(min_pts), int(mode),
                               labels.ctypes.data, core.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_dbscan failed ({rc})")
    return labels, core.astype(bool)


def border_sets(X, eps: float, core, labels):
    """CSR ``(offsets int64[n+1], sets int32[...])``: for each non-core point
    the sorted labels of the clusters it may join."""
    X = _points(X)
    n, d = X.shape
    core8 = np.ascontiguousarray(np.asarray(core, dtype=np.uint8))
    lab = np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    offsets = np.zeros(n + 1, dtype=np.int64)
    lib = _load()
    total = lib.oracle_border_sets(X.ctypes.data, n, d, float(eps), core8.ctypes.data, lab.ctypes.data,
                                   offsets.ctypes.data, None, 0)
    if total < 0:
        raise ValueError(f"oracle_border_sets failed ({total})")
    sets = np.zeros(max(int(total), 1), dtype=np.int32)
    lib.oracle_border_sets(X.ctypes.data, n, d, float(eps), core8.ctypes.data, lab.ctypes.data,
                           offsets.ctypes.data, sets.ctypes.data, int(total))
    return offsets, sets[: int(total)]


def point_neighbors(X, eps: float, q: int) -> np.ndarray:
    """Brute force: indices of all points adjacent to point ``q`` (q included)."""
    X = _points(X)
    n, d = X.shape
    lib = _load()
    k = lib.oracle_point_neighbors(X.ctypes.data, n, d, float(eps), int(q), None, 0)
    if k < 0:
        raise ValueError("oracle_point_neighbors failed")
    out = np.empty(max(int(k), 1), dtype=np.int64)
    lib.oracle_point_neighbors(X.ctypes.data, n, d, float(eps), int(q), out.ctypes.data, int(k))
    return out[: int(k)]


def adjacent(a, b, eps: float) -> bool:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float32))
    return bool(_load().oracle_adjacent(a.ctypes.data, b.ctypes.data, a.shape[0], float(eps)))


def dist2(a, b) -> float:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float32))
    return float(_load().oracle_dist2(a.ctypes.data, b.ctypes.data, a.shape[0]))
