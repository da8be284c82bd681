"""GPU: the no-allocation radix sort gives exactly the result of the allocating sort.

Some callers cannot call cudaMalloc: code running during CUDA graph capture, or inside a
framework that owns all device memory through its own pool.  The entry point serves them
with a scratch array inside the library, shared by every call.  Each case below makes
two calls in a row through the C ABI, so the second one runs on the scratch the first
one left behind.  This file is collected last on purpose: its scratch array stays
resident for the rest of the process."""
import ctypes as C

import numpy as np
import pytest

from paper_2311_04648_gb300 import dem

pytestmark = pytest.mark.gpu

MAX_KEYS = 1 << 20          # DEM_NOALLOC_SORT_MAX in include/dem.h


def _device_u32(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def _keys(n, bits, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 1 << bits, size=n, dtype=np.uint64).astype(np.uint32)
    keys[: n // 4] = keys[0]                 # equal keys: the order must stay stable
    return keys, np.arange(n, dtype=np.uint32)


@pytest.mark.parametrize("n,bits,seed", [(300_000, 23, 1), (65_537, 32, 2), (200_003, 8, 3), (MAX_KEYS, 20, 4)],
                         ids=["3pass", "4pass", "1pass", "max_n"])
def test_no_alloc_sort_matches_the_allocating_sort_on_two_calls(n, bits, seed):
    torch = pytest.importorskip("torch")
    L = dem.load()
    keys, vals = _keys(n, bits, seed)
    want_k, want_v = dem.radix_sort_u32(keys, vals, bits)
    dk, dv = _device_u32(torch, keys), _device_u32(torch, vals)
    for _ in range(2):
        ok, ov = torch.empty_like(dk), torch.empty_like(dv)
        st = L.dem_util_radix_sort_u32_noalloc(n, dk.data_ptr(), dv.data_ptr(), bits, ok.data_ptr(),
                                               ov.data_ptr(), None)
        assert st == dem.OK, L.dem_util_noalloc_error()
        assert L.dem_util_noalloc_error() == b""
        torch.cuda.synchronize()
        assert np.array_equal(ok.cpu().numpy().view(np.uint32), want_k)
        assert np.array_equal(ov.cpu().numpy().view(np.uint32), want_v)
        # the inputs are left untouched
        assert np.array_equal(dk.cpu().numpy().view(np.uint32), keys)


def test_no_alloc_sort_on_a_caller_stream():
    """Queued on a torch stream of the caller's (not the legacy default stream)."""
    torch = pytest.importorskip("torch")
    L = dem.load()
    keys, vals = _keys(123_457, 32, 5)
    want_k, want_v = dem.radix_sort_u32(keys, vals, 32)
    s = torch.cuda.Stream()
    dk, dv = _device_u32(torch, keys), _device_u32(torch, vals)
    torch.cuda.synchronize()
    for _ in range(2):
        with torch.cuda.stream(s):
            ok, ov = torch.empty_like(dk), torch.empty_like(dv)
            st = L.dem_util_radix_sort_u32_noalloc(len(keys), dk.data_ptr(), dv.data_ptr(), 32, ok.data_ptr(),
                                                   ov.data_ptr(), C.c_void_p(s.cuda_stream))
            assert st == dem.OK, L.dem_util_noalloc_error()
        s.synchronize()
        assert np.array_equal(ok.cpu().numpy().view(np.uint32), want_k)
        assert np.array_equal(ov.cpu().numpy().view(np.uint32), want_v)


def test_no_alloc_sort_rejects_more_keys_than_its_array_holds():
    torch = pytest.importorskip("torch")
    L = dem.load()
    a = torch.zeros(16, dtype=torch.int32, device="cuda")
    b = torch.zeros(16, dtype=torch.int32, device="cuda")
    st = L.dem_util_radix_sort_u32_noalloc(MAX_KEYS + 1, a.data_ptr(), a.data_ptr(), 32, b.data_ptr(),
                                           b.data_ptr() + 4, None)
    assert st == dem.ERR_CAPACITY
    assert b"DEM_NOALLOC_SORT_MAX" in L.dem_util_noalloc_error()


def test_no_alloc_sort_rejects_overlapping_buffers():
    """Rejected on the host before any work: nothing is launched."""
    torch = pytest.importorskip("torch")
    L = dem.load()
    n = 1000
    buf = torch.zeros(4 * n + 8, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    k, v, ko, vo = p, p + 4 * n, p + 8 * n, p + 12 * n
    cases = [(k, v, v, vo),            # keys_out is the values' input
             (k, v, ko, k),            # vals_out is the keys' input
             (k, v, ko, ko + 4),       # the outputs overlap by all but one word
             (k, v, k + 8, vo),        # keys_out overlaps the keys in part
             (k, v, ko, v - 4)]        # vals_out straddles the end of the keys
    for kk, vv, oo, pp in cases:
        st = L.dem_util_radix_sort_u32_noalloc(n, kk, vv, 32, oo, pp, None)
        assert st == dem.ERR_ARG
        assert b"overlap" in L.dem_util_noalloc_error()
    torch.cuda.synchronize()
