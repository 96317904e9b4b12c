"""The allocation-free sort entry point, airgs_sort_pairs_noalloc.

It serves callers that cannot allocate device memory while they run (an
allocation can synchronise the device; engine plug-ins and real-time loops
often live under a fixed memory budget).  Its scratch is a fixed device array,
so it needs no context.  This file is collected last so that a run stopping
at its first failure has run every other test; it passes alone in a fresh
process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _inputs(n, seed, bits):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 1 << min(bits, 12), n, dtype=np.int64).astype(np.uint32)  # many equal keys
    if bits > 12:
        keys |= (rng.integers(0, 1 << (bits - 12), n, dtype=np.int64).astype(np.uint32) << np.uint32(12))
    vals = rng.permutation(n).astype(np.uint32)
    to = lambda a: torch.from_numpy(a.view(np.int32)).cuda()
    return to(keys), to(vals)


def test_noalloc_sort_matches_allocating_sort_twice():
    from paper_2512_20943_b300 import Rasterizer, _abi
    lib = _abi.load_library()
    rast = Rasterizer()
    stream = torch.cuda.current_stream()
    for call, (n, bits) in enumerate([(300_001, 24), (1 << 20, 17)]):  # two calls in a row, different sizes
        keys, vals = _inputs(n, 10 + call, bits)
        ref_k, ref_v = rast.sort_pairs(keys, vals, bits)  # existing entry point (allocates from its pool)
        out_k, out_v = torch.empty_like(keys), torch.empty_like(vals)
        rc = lib.airgs_sort_pairs_noalloc(_ptr(keys), _ptr(vals), _ptr(out_k), _ptr(out_v), n, bits,
                                          ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        # integer results: bit-exact
        assert torch.equal(out_k, ref_k), call
        assert torch.equal(out_v, ref_v), call
        # inputs untouched
        k2, v2 = _inputs(n, 10 + call, bits)
        assert torch.equal(keys, k2) and torch.equal(vals, v2)


def test_noalloc_sort_rejects_oversize_and_bad_arguments():
    from paper_2512_20943_b300 import _abi
    lib = _abi.load_library()
    n = _abi.AIRGS_NOALLOC_SORT_MAX_PAIRS + 1
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = lib.airgs_sort_pairs_noalloc(_ptr(x), _ptr(x), _ptr(x), _ptr(x), n, 32, None)
    assert rc == _abi.AIRGS_E_CAPACITY
    assert lib.airgs_sort_pairs_noalloc(_ptr(x), _ptr(x), _ptr(x), _ptr(x), 8, 0, None) == _abi.AIRGS_E_ARG
    assert lib.airgs_sort_pairs_noalloc(None, _ptr(x), _ptr(x), _ptr(x), 8, 8, None) == _abi.AIRGS_E_ARG
