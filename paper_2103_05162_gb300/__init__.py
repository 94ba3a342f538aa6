"""gbdbscan: DBSCAN (FDbscan / FDbscan-DenseBox) for 2D/3D fp32 points on GB300.

A thin ctypes binding over the C ABI of ``lib/libgbdbscan.so`` (declared in
``include/gbdbscan.h``). It only marshals arguments: every stage of the
clustering runs in the library's CUDA kernels. Device memory and streams come
from PyTorch tensors and ``torch.cuda`` streams. There is no CPU fallback: if
the library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "DbscanError", "MODE_DBSCAN", "MODE_DBSCAN_STAR", "ALGO_FDBSCAN", "ALGO_DENSEBOX", "ALGO_AUTO",
    "load", "library_path", "dbscan_run", "dbscan_run_host", "dbscan_run_host_async", "dbscan_run_batch", "dbscan_run_multi", "dbscan_run_slabs", "Server",
    "sort_pairs_u64", "sort_pairs_u64_noalloc", "morton_codes", "lbvh_topology", "set_tuning",
    "set_auto_threshold", "last_choice", "stream_status", "release_workspaces", "profile_enable",
    "profile_collect", "kernel_launches", "last_stats",
]

MODE_DBSCAN = 0
MODE_DBSCAN_STAR = 1
ALGO_FDBSCAN = 0
ALGO_DENSEBOX = 1
ALGO_AUTO = 2

_STATUS = {
    0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NONFINITE", 5: "DEVICE_TIMEOUT", 6: "BUSY",
    7: "NOT_FOUND",
}

_MODES = {"dbscan": MODE_DBSCAN, "dbscan*": MODE_DBSCAN_STAR, "dbscan_star": MODE_DBSCAN_STAR}
_ALGOS = {"fdbscan": ALGO_FDBSCAN, "densebox": ALGO_DENSEBOX, "auto": ALGO_AUTO}


class DbscanError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = _STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libgbdbscan.so (building it first if it is missing and nvcc is
    available). Raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"libgbdbscan.so is not built ({_build.LIB})")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        i64, i32, f32, vp, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_uint64
        sz = ctypes.c_size_t
        sig = {
            "dbscan_run": [vp, i64, i32, f32, i32, i32, i32, vp, vp, vp],
            "dbscan_run_sync": [vp, i64, i32, f32, i32, i32, i32, vp, vp, vp],
            "dbscan_run_host": [vp, i64, i32, f32, i32, i32, i32, vp, vp, vp],
            "dbscan_run_host_async": [vp, i64, i32, f32, i32, i32, i32, vp, vp, vp],
            "dbscan_run_batch": [vp, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp],
            "dbscan_run_multi": [vp, i64, i32, f32, vp, i32, i32, i32, vp, vp, vp],
            "dbscan_run_slabs": [vp, i64, i32, f32, i32, i32, i32, vp, vp, i64, vp],
            "dbscan_server_create": [sz, i32, ctypes.POINTER(vp)],
            "dbscan_server_submit": [vp, vp, i64, i32, f32, i32, i32, i32, vp, vp, ctypes.POINTER(u64)],
            "dbscan_server_poll": [vp, u64, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)],
            "dbscan_server_wait": [vp, u64],
            "dbscan_server_release": [vp, u64],
            "dbscan_server_destroy": [vp],
            "dbscan_server_set_batching": [vp, i64, i64, i32],
            "dbscan_server_stats": [vp, vp],
            "dbscan_server_hold": [vp, i32],
            "dbscan_stream_status": [vp],
            "dbscan_release_workspaces": [],
            "dbscan_set_tuning": [i32, f32],
            "dbscan_set_auto_threshold": [i32, f32, f32],
            "dbscan_last_choice": [vp, ctypes.POINTER(i32), vp],
            "dbscan_sort_pairs_u64": [vp, vp, i64, i32, vp],
            "dbscan_sort_pairs_u64_noalloc": [vp, vp, i64, i32, vp],
            "dbscan_morton_codes": [vp, i64, i32, vp, vp, i32, vp, vp],
            "dbscan_lbvh_topology": [vp, i64, vp, vp, vp],
            "dbscan_profile_enable": [i32],
            "dbscan_profile_collect": [vp, vp, vp],
            "dbscan_last_stats": [vp, vp],
            "dbscan_test_sort_hooks": [i64, i32],
            "dbscan_set_border_lists": [i32],
            "dbscan_tuning_lookup": [i32, i32, i64, i32, i32, i32, i64, ctypes.POINTER(i32),
                                     ctypes.POINTER(f32), ctypes.POINTER(f32)],
            "dbscan_tuning_clear": [],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = i32
        lib.dbscan_last_error.argtypes = []
        lib.dbscan_last_error.restype = ctypes.c_char_p
        lib.dbscan_profile_stage_name.argtypes = [i32]
        lib.dbscan_profile_stage_name.restype = ctypes.c_char_p
        lib.dbscan_border_lists.argtypes = []
        lib.dbscan_border_lists.restype = i32
        lib.dbscan_kernel_launches.argtypes = []
        lib.dbscan_kernel_launches.restype = i64
        _lib = lib
        return lib


def _check(status: int):
    if status != 0:
        msg = _lib.dbscan_last_error().decode(errors="replace") if _lib is not None else ""
        raise DbscanError(status, msg)


def _mode(mode) -> int:
    return _MODES[mode.lower()] if isinstance(mode, str) else int(mode)


def _algo(algo) -> int:
    return _ALGOS[algo.lower()] if isinstance(algo, str) else int(algo)


def _stream_handle(stream, device=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def dbscan_run(points, eps: float, min_pts: int, mode="dbscan", algo="densebox", labels_out=None,
               core_out=None, want_core: bool = False, stream=None, sync: bool = False):
    """Clusters ``points`` (a CUDA float32 tensor of shape (n, d), 2 <= d <= 8).

    Returns ``labels`` (int32, -1 = noise, else the smallest input index of a
    core point of the cluster) or ``(labels, core)`` when ``want_core`` or
    ``core_out`` is given. Work is enqueued on ``stream`` (default: the
    current torch stream) and the call returns without waiting for it;
    errors found on the device (non-finite input, a bounded wait that gave
    up) are raised by ``stream_status()``, or by this call with ``sync``.
    """
    import torch
    lib = load()
    if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dtype == torch.float32):
        raise TypeError("points must be a CUDA float32 tensor")
    if points.dim() != 2:
        raise ValueError("points must have shape (n, dim)")
    points = points.contiguous()
    n, d = points.shape
    if labels_out is None:
        labels_out = torch.empty(n, dtype=torch.int32, device=points.device)
    if core_out is None and want_core:
        core_out = torch.empty(n, dtype=torch.uint8, device=points.device)
    fn = lib.dbscan_run_sync if sync else lib.dbscan_run
    with torch.cuda.device(points.device):
        _check(fn(_ptr(points), n, d, float(eps), int(min_pts), _mode(mode), _algo(algo),
                  _ptr(labels_out), _ptr(core_out), _stream_handle(stream, points.device)))
    return (labels_out, core_out) if core_out is not None else labels_out


def dbscan_run_slabs(points: np.ndarray, eps: float, min_pts: int, mode="dbscan", algo="densebox",
                     slab_points: int = 0, stream=None):
    """Clusters host ``points`` (float32 (n, d)) slab by slab, for sets larger
    than device memory. Returns (labels int32[n], core bool[n])."""
    lib = load()
    pts = np.ascontiguousarray(points, dtype=np.float32)
    if pts.ndim != 2:
        raise TypeError("points must have shape (n, dim)")
    n, d = pts.shape
    labels = np.empty(n, dtype=np.int32)
    core = np.empty(n, dtype=np.uint8)
    _check(lib.dbscan_run_slabs(ctypes.c_void_p(pts.ctypes.data), n, d, float(eps), int(min_pts), _mode(mode),
                                _algo(algo), ctypes.c_void_p(labels.ctypes.data), ctypes.c_void_p(core.ctypes.data),
                                int(slab_points), _stream_handle(stream)))
    return labels, core.astype(bool)


def dbscan_run_multi(points, eps: float, min_pts, mode="dbscan", algo="densebox", labels_out=None,
                     core_out=None, want_core: bool = False, stream=None):
    """Clusters CUDA ``points`` (n, d) once per value of ``min_pts`` over one
    index. Returns labels of shape (len(min_pts), n) (and core flags of the
    same shape if ``want_core`` or ``core_out`` is given); row k is what
    dbscan_run gives for min_pts[k]."""
    import torch
    lib = load()
    points = points.contiguous()
    n, d = points.shape
    mps = np.ascontiguousarray(np.asarray(min_pts, dtype=np.int32).reshape(-1))
    count = int(mps.shape[0])
    if labels_out is None:
        labels_out = torch.empty((count, n), dtype=torch.int32, device=points.device)
    if core_out is None and want_core:
        core_out = torch.empty((count, n), dtype=torch.uint8, device=points.device)
    _check(lib.dbscan_run_multi(_ptr(points), n, d, float(eps), ctypes.c_void_p(mps.ctypes.data), count,
                                _mode(mode), _algo(algo), _ptr(labels_out), _ptr(core_out),
                                _stream_handle(stream, points.device)))
    return (labels_out, core_out) if core_out is not None else labels_out


def dbscan_run_host(points: np.ndarray, eps: float, min_pts: int, mode="dbscan", algo="densebox",
                    labels_out: np.ndarray | None = None, core_out: np.ndarray | None = None, stream=None):
    """The same clustering on host arrays (copies in, clusters, copies out,
    waits). ``points`` is a float32 (n, d) array (pinned memory is faster)."""
    lib = load()
    pts = np.asarray(points)
    if pts.dtype != np.float32 or pts.ndim != 2 or not pts.flags.c_contiguous:
        raise TypeError("points must be a C-contiguous float32 array of shape (n, dim)")
    n, d = pts.shape
    if labels_out is None:
        labels_out = np.empty(n, dtype=np.int32)
    _check(lib.dbscan_run_host(ctypes.c_void_p(pts.ctypes.data), n, d, float(eps), int(min_pts), _mode(mode),
                               _algo(algo), ctypes.c_void_p(labels_out.ctypes.data),
                               ctypes.c_void_p(core_out.ctypes.data) if core_out is not None else None,
                               _stream_handle(stream)))
    return (labels_out, core_out) if core_out is not None else labels_out


def dbscan_run_host_async(points: np.ndarray, eps: float, min_pts: int, labels_out: np.ndarray, mode="dbscan",
                          algo="densebox", core_out: np.ndarray | None = None, stream=None):
    """dbscan_run_host without the wait: enqueues copy in, clustering and
    copy out on ``stream`` and returns. ``points``, ``labels_out`` (and
    ``core_out``) must live in page-locked memory (e.g. the numpy view of a
    pinned torch tensor) and stay alive until the stream is done; read them
    after a stream synchronize or ``stream_status``."""
    lib = load()
    pts = np.asarray(points)
    if pts.dtype != np.float32 or pts.ndim != 2 or not pts.flags.c_contiguous:
        raise TypeError("points must be a C-contiguous float32 array of shape (n, dim)")
    n, d = pts.shape
    if labels_out.dtype != np.int32 or labels_out.shape != (n,) or not labels_out.flags.c_contiguous:
        raise TypeError("labels_out must be a C-contiguous int32 array of n entries")
    if core_out is not None and (core_out.dtype != np.uint8 or core_out.shape != (n,)
                                 or not core_out.flags.c_contiguous):
        raise TypeError("core_out must be a C-contiguous uint8 array of n entries")
    _check(lib.dbscan_run_host_async(ctypes.c_void_p(pts.ctypes.data), n, d, float(eps), int(min_pts), _mode(mode),
                                     _algo(algo), ctypes.c_void_p(labels_out.ctypes.data),
                                     ctypes.c_void_p(core_out.ctypes.data) if core_out is not None else None,
                                     _stream_handle(stream)))
    return (labels_out, core_out) if core_out is not None else labels_out


def dbscan_run_batch(points, offsets, dims, eps, min_pts, mode="dbscan", algo="densebox", labels_out=None,
                     core_out=None, stream=None):
    """Clusters independent instances concatenated in ``points`` (a flat CUDA
    float32 tensor of coordinates). ``offsets`` (count+1 row offsets), ``dims``,
    ``eps``, ``min_pts`` are host sequences. Labels are relative to each
    instance."""
    import torch
    lib = load()
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    dm = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
    ep = np.ascontiguousarray(np.asarray(eps, dtype=np.float32))
    mp = np.ascontiguousarray(np.asarray(min_pts, dtype=np.int32))
    count = len(dm)
    total = int(off[-1]) if count else 0
    if labels_out is None:
        labels_out = torch.empty(total, dtype=torch.int32, device=points.device)
    with torch.cuda.device(points.device):
        _check(lib.dbscan_run_batch(_ptr(points), ctypes.c_void_p(off.ctypes.data), ctypes.c_void_p(dm.ctypes.data),
                                    ctypes.c_void_p(ep.ctypes.data), ctypes.c_void_p(mp.ctypes.data), count,
                                    _mode(mode), _algo(algo), _ptr(labels_out), _ptr(core_out),
                                    _stream_handle(stream, points.device)))
    return (labels_out, core_out) if core_out is not None else labels_out


class Server:
    """A serving loop: jobs are admitted against a device-memory budget and a
    slot limit and run concurrently on the slots' streams."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.dbscan_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, points, eps: float, min_pts: int, mode="dbscan", algo="densebox", labels_out=None,
               core_out=None) -> int:
        import torch
        points = points.contiguous()
        n, d = points.shape
        if labels_out is None:
            labels_out = torch.empty(n, dtype=torch.int32, device=points.device)
        jid = ctypes.c_uint64()
        _check(_lib.dbscan_server_submit(self._h, _ptr(points), n, d, float(eps), int(min_pts), _mode(mode),
                                         _algo(algo), _ptr(labels_out), _ptr(core_out), ctypes.byref(jid)))
        self._keep[jid.value] = (points, labels_out, core_out)
        return jid.value

    def set_batching(self, max_job_points: int = 1 << 18, max_batch_points: int = 1 << 24,
                     max_batch_jobs: int = 4096):
        """Continuous batching limits (max_job_points=0 turns it off)."""
        _check(_lib.dbscan_server_set_batching(self._h, int(max_job_points), int(max_batch_points),
                                               int(max_batch_jobs)))

    def hold(self, on: bool = True):
        """Pauses (True) or resumes (False) admission of queued jobs."""
        _check(_lib.dbscan_server_hold(self._h, 1 if on else 0))

    def stats(self) -> dict:
        out = (ctypes.c_int64 * 4)()
        _check(_lib.dbscan_server_stats(self._h, out))
        return {"done": out[0], "single": out[1], "batches": out[2], "batched_jobs": out[3]}

    def poll(self, job_id: int):
        done = ctypes.c_int()
        lat = ctypes.c_double()
        _check(_lib.dbscan_server_poll(self._h, job_id, ctypes.byref(done), ctypes.byref(lat)))
        return bool(done.value), lat.value

    def wait(self, job_id: int, timeout: float | None = None):
        """Blocks until the job is done (at most ``timeout`` seconds, then
        TimeoutError) and returns its labels; raises DbscanError if it
        failed."""
        if timeout is None:
            _check(_lib.dbscan_server_wait(self._h, job_id))
        else:
            import time
            deadline = time.monotonic() + timeout
            while not self.poll(job_id)[0]:
                if time.monotonic() > deadline:
                    raise TimeoutError(f"job {job_id} not done after {timeout} s")
                time.sleep(1e-4)
        return self._keep[job_id][1]

    def release(self, job_id: int):
        _check(_lib.dbscan_server_release(self._h, job_id))
        return self._keep.pop(job_id, None)

    def close(self):
        if self._h is not None:
            _check(_lib.dbscan_server_destroy(self._h))
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def sort_pairs_u64(keys, values, key_bits: int, stream=None):
    """Stable radix sort in place of CUDA int64 ``keys`` (viewed as uint64)
    and int32 ``values`` by the low ``key_bits`` bits."""
    lib = load()
    _check(lib.dbscan_sort_pairs_u64(_ptr(keys), _ptr(values), keys.numel(), int(key_bits),
                                     _stream_handle(stream, keys.device)))


SORT_NOALLOC_MAX_PAIRS = 1 << 20


def sort_pairs_u64_noalloc(keys, values, key_bits: int, stream=None):
    """sort_pairs_u64 without any device allocation (scratch in a static
    device array; n <= SORT_NOALLOC_MAX_PAIRS; overlapping calls race)."""
    lib = load()
    _check(lib.dbscan_sort_pairs_u64_noalloc(_ptr(keys), _ptr(values), keys.numel(), int(key_bits),
                                             _stream_handle(stream, keys.device)))


def morton_codes(points, lo, hi, bits: int, out=None, stream=None):
    import torch
    lib = load()
    points = points.contiguous()
    n, d = points.shape
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=points.device)
    lo = np.ascontiguousarray(np.asarray(lo, dtype=np.float32))
    hi = np.ascontiguousarray(np.asarray(hi, dtype=np.float32))
    _check(lib.dbscan_morton_codes(_ptr(points), n, d, ctypes.c_void_p(lo.ctypes.data),
                                   ctypes.c_void_p(hi.ctypes.data), int(bits), _ptr(out),
                                   _stream_handle(stream, points.device)))
    return out


def lbvh_topology(leaf_keys, stream=None):
    """Karras LBVH topology over sorted keys: returns (children (m-1, 2),
    ranges (m-1, 2)) int32 CUDA tensors."""
    import torch
    lib = load()
    m = leaf_keys.numel()
    ch = torch.empty((max(m - 1, 1), 2), dtype=torch.int32, device=leaf_keys.device)
    rg = torch.empty((max(m - 1, 1), 2), dtype=torch.int32, device=leaf_keys.device)
    _check(lib.dbscan_lbvh_topology(_ptr(leaf_keys), m, _ptr(ch), _ptr(rg), _stream_handle(stream, leaf_keys.device)))
    return ch, rg


PROFILE_STAGES = 10


def profile_enable(on: bool = True):
    """Per-stage CUDA-event timing of every run (process-wide switch)."""
    _check(load().dbscan_profile_enable(1 if on else 0))


def profile_collect(stream=None) -> dict:
    """{stage name: (total ms, executions)} since the last collect."""
    lib = load()
    ms = (ctypes.c_double * PROFILE_STAGES)()
    cnt = (ctypes.c_int64 * PROFILE_STAGES)()
    _check(lib.dbscan_profile_collect(_stream_handle(stream), ms, cnt))
    return {lib.dbscan_profile_stage_name(i).decode(): (ms[i], cnt[i]) for i in range(PROFILE_STAGES)}


def kernel_launches() -> int:
    """Number of CUDA kernels the library has launched since it was loaded."""
    return int(load().dbscan_kernel_launches())


def last_stats(stream=None) -> dict:
    """Statistics of the last run on the stream: BVH leaves m, dense cells."""
    out = (ctypes.c_int64 * 2)()
    _check(load().dbscan_last_stats(_stream_handle(stream), out))
    return {"leaves": int(out[0]), "dense_cells": int(out[1])}


def set_border_lists(on: bool):
    """Border claims from preprocessing's per-point neighbour lists (True,
    the default) or by core points in the main traversal with no per-point
    list (False); see dbscan_set_border_lists."""
    _check(load().dbscan_set_border_lists(1 if on else 0))


def border_lists() -> bool:
    return bool(load().dbscan_border_lists())


def sort_test_hooks(wait_limit: int = -1, stall_first_tile: bool = False):
    """Test hooks of the radix sort's bounded wait (see dbscan_test_sort_hooks);
    (-1, False) restores the defaults."""
    _check(load().dbscan_test_sort_hooks(int(wait_limit), 1 if stall_first_tile else 0))


def tuning_lookup(dim: int, n: int, min_pts: int, mode="dbscan", algo="densebox", batch: bool = False,
                  count: int = 0):
    """The autotuner's (block size, cell factor, ms per call) for a kind of
    call, or None if that kind has not been tuned (see dbscan_tuning_lookup)."""
    lib = load()
    b, f, ms = ctypes.c_int(), ctypes.c_float(), ctypes.c_float()
    st = lib.dbscan_tuning_lookup(1 if batch else 0, int(dim), int(n), int(min_pts), _mode(mode), _algo(algo),
                                  int(count), ctypes.byref(b), ctypes.byref(f), ctypes.byref(ms))
    if st == 7:  # NOT_FOUND
        return None
    _check(st)
    return b.value, f.value, ms.value


def tuning_clear():
    _check(load().dbscan_tuning_clear())


def set_tuning(block_size: int = 0, cell_factor: float = 0.0):
    _check(load().dbscan_set_tuning(int(block_size), float(cell_factor)))


def set_auto_threshold(dim: int, dense_fraction: float = -1.0, occupancy: float = -1.0):
    """For data of dimension ``dim``, algo="auto" takes DenseBox when the
    estimated share of points in dense cells or the estimated mean cell
    occupancy reaches its threshold (both negative: the defaults)."""
    _check(load().dbscan_set_auto_threshold(int(dim), float(dense_fraction), float(occupancy)))


def last_choice(stream=None):
    """(algorithm used by the last call on the stream, estimated dense-point
    share, estimated mean cell occupancy); the estimates are -1 when the
    algorithm was not chosen automatically."""
    a = ctypes.c_int()
    f = (ctypes.c_float * 2)()
    _check(load().dbscan_last_choice(_stream_handle(stream), ctypes.byref(a), f))
    return a.value, f[0], f[1]


def stream_status(stream=None):
    _check(load().dbscan_stream_status(_stream_handle(stream)))


def release_workspaces():
    _check(load().dbscan_release_workspaces())
