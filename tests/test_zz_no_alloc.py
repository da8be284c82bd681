"""GPU: the no-allocation radix sort (for callers that cannot call cudaMalloc, e.g. code
running during CUDA graph capture or inside a framework that owns device memory) gives
exactly the result of the allocating sort, on two calls in a row that share its
internal scratch array.  Collected last on purpose: its scratch array stays resident."""
import ctypes as C

import numpy as np
import pytest

from paper_2311_04648_gb300 import dem

pytestmark = pytest.mark.gpu

MAX_KEYS = 1 << 20          # DEM_NOALLOC_SORT_MAX in include/dem.h


def _device_u32(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def test_no_alloc_sort_matches_the_allocating_sort_on_two_calls():
    torch = pytest.importorskip("torch")
    L = dem.load()
    for n, bits, seed in ((300_000, 23, 1), (65_537, 32, 2)):
        rng = np.random.default_rng(seed)
        keys = rng.integers(0, 1 << bits, size=n, dtype=np.uint64).astype(np.uint32)
        keys[: n // 4] = keys[0]                 # equal keys: the order must stay stable
        vals = np.arange(n, dtype=np.uint32)
        want_k, want_v = dem.radix_sort_u32(keys, vals, bits)
        dk, dv = _device_u32(torch, keys), _device_u32(torch, vals)
        ok, ov = torch.empty_like(dk), torch.empty_like(dv)
        st = L.dem_util_radix_sort_u32_noalloc(n, dk.data_ptr(), dv.data_ptr(), bits, ok.data_ptr(), ov.data_ptr(),
                                               None)
        assert st == dem.OK, L.dem_util_noalloc_error()
        torch.cuda.synchronize()
        assert np.array_equal(ok.cpu().numpy().view(np.uint32), want_k)
        assert np.array_equal(ov.cpu().numpy().view(np.uint32), want_v)
        # the inputs are left untouched
        assert np.array_equal(dk.cpu().numpy().view(np.uint32), keys)


def test_no_alloc_sort_rejects_more_keys_than_its_array_holds():
    torch = pytest.importorskip("torch")
    L = dem.load()
    a = torch.zeros(16, dtype=torch.int32, device="cuda")
    b = torch.zeros(16, dtype=torch.int32, device="cuda")
    st = L.dem_util_radix_sort_u32_noalloc(MAX_KEYS + 1, a.data_ptr(), a.data_ptr(), 32, b.data_ptr(),
                                           b.data_ptr() + 4, None)
    assert st == dem.ERR_CAPACITY
    assert b"DEM_NOALLOC_SORT_MAX" in L.dem_util_noalloc_error()
