"""The radix sort entry point that allocates nothing (dbscan_sort_pairs_u64_noalloc).

Some callers may not call cudaMalloc: real-time loops, where an allocation can
synchronise the device or fail at a bad moment, and applications that hand
the GPU's memory to their own pool or budget. This entry point serves them
from a static device array. Through the C ABI, on two and more calls in a
row (each reusing the array the one before left behind), it must give
exactly the pairs of the allocating entry point and of numpy's stable
argsort, leave the device's free memory unchanged, and reject sizes beyond
its capacity. This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2103_05162_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, k, v, bits):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.dbscan_sort_pairs_u64_noalloc(ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                             k.numel(), bits, stream)


def _keys(rs, n, bits):
    if bits == 64:
        keys = rs.integers(-(1 << 62), 1 << 62, size=n, dtype=np.int64)
    else:
        keys = rs.integers(0, 1 << bits, size=n, dtype=np.int64)
    keys[::5] = keys[3]  # duplicates: stability matters
    return keys


def test_noalloc_sort_matches_allocating_sort_and_argsort_on_consecutive_calls():
    lib = gb.load()
    rs = np.random.default_rng(2024)
    # calls in a row with different sizes and key widths: each one runs on
    # the scratch the one before left behind
    for n, bits in ((300_001, 40), (gb.SORT_NOALLOC_MAX_PAIRS, 64), (77_777, 13), (4097, 21)):
        keys = _keys(rs, n, bits)
        vals = rs.permutation(n).astype(np.int32)
        k_ref = torch.from_numpy(keys.copy()).cuda()
        v_ref = torch.from_numpy(vals.copy()).cuda()
        gb.sort_pairs_u64(k_ref, v_ref, bits)
        k = torch.from_numpy(keys.copy()).cuda()
        v = torch.from_numpy(vals.copy()).cuda()
        assert _call_noalloc(lib, k, v, bits) == 0, lib.dbscan_last_error()
        assert lib.dbscan_last_error() == b""
        torch.cuda.synchronize()
        assert torch.equal(k, k_ref) and torch.equal(v, v_ref)
        # and the definition: a stable order of the low `bits` bits
        mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        order = np.argsort(keys.view(np.uint64) & mask, kind="stable")
        assert (v.cpu().numpy() == vals[order]).all()
        assert (k.cpu().numpy() == keys[order]).all()


def test_noalloc_sort_leaves_free_device_memory_unchanged():
    lib = gb.load()
    gb.release_workspaces()
    rs = np.random.default_rng(7)
    n, bits = 500_000, 48
    k = torch.from_numpy(_keys(rs, n, bits)).cuda()
    v = torch.arange(n, dtype=torch.int32, device="cuda")
    assert _call_noalloc(lib, k, v, bits) == 0, lib.dbscan_last_error()  # may set up the array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _call_noalloc(lib, k, v, bits) == 0, lib.dbscan_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_sort_rejects_sizes_beyond_its_capacity():
    lib = gb.load()
    n = gb.SORT_NOALLOC_MAX_PAIRS + 1
    k = torch.zeros(n, dtype=torch.int64, device="cuda")
    v = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert _call_noalloc(lib, k, v, 8) == 1
    assert b"capacity" in lib.dbscan_last_error()
    # a later good call clears the message
    k = torch.zeros(10, dtype=torch.int64, device="cuda")
    v = torch.zeros(10, dtype=torch.int32, device="cuda")
    assert _call_noalloc(lib, k, v, 8) == 0
    assert lib.dbscan_last_error() == b""
