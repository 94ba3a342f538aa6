"""The radix sort entry point that allocates nothing (dbscan_sort_pairs_u64_noalloc).

It exists for callers that cannot call cudaMalloc (graph capture, real-time
loops, pool-managed memory); its scratch is a static device array. It must
give exactly the same pairs as the allocating entry point, on consecutive
calls that reuse the array, and reject sizes beyond its capacity. This file is
named so that pytest collects it last.
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


def test_noalloc_sort_matches_allocating_sort_on_consecutive_calls():
    lib = gb.load()
    rs = np.random.default_rng(2024)
    # two calls in a row with different sizes and key widths: the second one
    # runs on the scratch the first one left behind
    for n, bits in ((300_001, 40), (gb.SORT_NOALLOC_MAX_PAIRS, 64), (77_777, 13)):
        if bits == 64:
            keys = rs.integers(-(1 << 62), 1 << 62, size=n, dtype=np.int64)
        else:
            keys = rs.integers(0, 1 << bits, size=n, dtype=np.int64)
        keys[::5] = keys[3]  # duplicates: stability matters
        vals = rs.permutation(n).astype(np.int32)
        k_ref = torch.from_numpy(keys.copy()).cuda()
        v_ref = torch.from_numpy(vals.copy()).cuda()
        gb.sort_pairs_u64(k_ref, v_ref, bits)
        k = torch.from_numpy(keys.copy()).cuda()
        v = torch.from_numpy(vals.copy()).cuda()
        assert _call_noalloc(lib, k, v, bits) == 0, lib.dbscan_last_error()
        torch.cuda.synchronize()
        assert torch.equal(k, k_ref) and torch.equal(v, v_ref)


def test_noalloc_sort_rejects_sizes_beyond_its_capacity():
    lib = gb.load()
    n = gb.SORT_NOALLOC_MAX_PAIRS + 1
    k = torch.zeros(n, dtype=torch.int64, device="cuda")
    v = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert _call_noalloc(lib, k, v, 8) == 1
    assert b"capacity" in lib.dbscan_last_error()
