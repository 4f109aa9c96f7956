"""The allocation-free radix sort entry point, for callers that cannot allocate
device memory while sorting (memory held by another allocator, or a loop that
must not block on an allocation).  It must give the same result as the
allocating entry point, call after call, since every call reuses the same
fixed scratch array inside the library.  This file is collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LIMIT = 1 << 18


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_sort_matches_allocating_sort_twice():
    import paper_2609_13397_b300 as cg
    from paper_2609_13397_b300._lib import lib
    L = lib()
    ctx = cg.Context(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, bits) in enumerate([(200003, 32), (LIMIT, 17)]):
        rng = np.random.default_rng(100 + call)
        keys = rng.integers(0, 1 << bits, n, dtype=np.uint64).astype(np.uint32)
        keys[: n // 4] = keys[n // 2]                      # many equal keys: stability matters
        vals = rng.permutation(n).astype(np.uint32)
        ka = torch.from_numpy(keys.view(np.int32)).cuda()
        va = torch.from_numpy(vals.view(np.int32)).cuda()
        kb, vb = ka.clone(), va.clone()
        cg.radix_sort_pairs(ctx, ka, va, 0, bits)           # the allocating entry point
        st = L.conegs_radix_sort_pairs_noalloc(_p(kb), _p(vb), n, 0, bits, stream)
        assert st == 0, L.conegs_last_error()
        torch.cuda.synchronize()
        assert torch.equal(ka, kb) and torch.equal(va, vb)
        order = np.argsort(keys, kind="stable")
        assert np.array_equal(kb.cpu().numpy().view(np.uint32), keys[order])


def _pool_reset_high(rt, pool):
    attr = rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh
    from cuda.bindings import driver as dr
    try:
        (err,) = rt.cudaMemPoolSetAttribute(pool, attr, dr.cuuint64_t(0))
    except TypeError:
        (err,) = rt.cudaMemPoolSetAttribute(pool, attr, 0)
    assert err == rt.cudaError_t.cudaSuccess, err


def _pool_get(rt, pool, name):
    err, val = rt.cudaMemPoolGetAttribute(pool, getattr(rt.cudaMemPoolAttr, name))
    assert err == rt.cudaError_t.cudaSuccess, err
    return int(val)


def test_noalloc_sort_allocates_nothing():
    """Around calls after the first (which only looks up the array's address),
    nothing is allocated: the device's default pool (which the library's other
    entry points draw from with cudaMallocAsync) neither reserves more nor
    reaches a higher use than before the calls, torch's allocator makes no
    allocation, and the device's free memory does not shrink."""
    from cuda.bindings import runtime as rt
    from paper_2609_13397_b300._lib import lib
    L = lib()
    dev = torch.cuda.current_device()
    n = 150001
    rng = np.random.default_rng(7)
    keys = torch.from_numpy(rng.integers(0, 1 << 31, n, dtype=np.int64).astype(np.int32)).cuda()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.conegs_radix_sort_pairs_noalloc(_p(keys), _p(vals), n, 0, 31, stream) == 0   # set-up call
    torch.cuda.synchronize()
    err, pool = rt.cudaDeviceGetDefaultMemPool(dev)
    assert err == rt.cudaError_t.cudaSuccess, err
    used0 = _pool_get(rt, pool, "cudaMemPoolAttrUsedMemCurrent")
    reserved0 = _pool_get(rt, pool, "cudaMemPoolAttrReservedMemCurrent")
    _pool_reset_high(rt, pool)
    inputs = [torch.from_numpy(rng.integers(0, 1 << 31, n, dtype=np.int64).astype(np.int32)).cuda()
              for _ in range(3)]
    torch.cuda.synchronize()
    torch_allocs0 = torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0)
    free0 = torch.cuda.mem_get_info(dev)[0]
    for k in range(3):
        keys.copy_(inputs[k])
        torch.cuda.synchronize()
        allocs_k = torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0)
        assert L.conegs_radix_sort_pairs_noalloc(_p(keys), _p(vals), n, 0, 31, stream) == 0
        torch.cuda.synchronize()
        assert torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0) == allocs_k
    assert _pool_get(rt, pool, "cudaMemPoolAttrUsedMemHigh") <= used0
    assert _pool_get(rt, pool, "cudaMemPoolAttrReservedMemCurrent") <= reserved0
    assert torch.cuda.mem_get_info(dev)[0] >= free0
    assert torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0) == torch_allocs0
    k_sorted = keys.cpu().numpy()
    assert (np.diff(k_sorted.astype(np.int64)) >= 0).all()


def test_noalloc_sort_rejects_sizes_beyond_its_limit():
    from paper_2609_13397_b300._lib import lib
    L = lib()
    k = torch.zeros(LIMIT + 1, dtype=torch.int32, device="cuda")
    v = torch.zeros(LIMIT + 1, dtype=torch.int32, device="cuda")
    st = L.conegs_radix_sort_pairs_noalloc(_p(k), _p(v), LIMIT + 1, 0, 32, None)
    assert st == 1
    assert b"262144" in L.conegs_last_error()
