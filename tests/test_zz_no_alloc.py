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


def test_noalloc_sort_rejects_sizes_beyond_its_limit():
    from paper_2609_13397_b300._lib import lib
    L = lib()
    k = torch.zeros(LIMIT + 1, dtype=torch.int32, device="cuda")
    v = torch.zeros(LIMIT + 1, dtype=torch.int32, device="cuda")
    st = L.conegs_radix_sort_pairs_noalloc(_p(k), _p(v), LIMIT + 1, 0, 32, None)
    assert st == 1
    assert b"262144" in L.conegs_last_error()
