"""The allocation-free sort entry point, airgs_sort_pairs_noalloc.

It serves callers that cannot allocate device memory while they run (an
allocation can synchronise the device; engine plug-ins and real-time loops
often live under a fixed memory budget).  Its scratch is a fixed device array,
so it needs no context.  This file is collected last so that a run stopping
at its first failure has run every other test; it passes alone in a fresh
process as well.

The key widths cover every ping-pong order of the entry point: 8 bits (one
pass, inputs -> outputs), 16 (two: inputs -> scratch -> outputs), 17 and 24
(three: inputs -> outputs -> scratch -> outputs) and 32 (four, with the
outputs as an intermediate buffer).  Keys carry random bits above key_bits,
which the sort must ignore.
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
    if bits < 32:  # bits the sort must not look at
        keys |= (rng.integers(0, 1 << (32 - bits), n, dtype=np.int64).astype(np.uint32) << np.uint32(bits))
    vals = rng.permutation(n).astype(np.uint32)
    return keys, vals


def _dev(a):
    return torch.from_numpy(a.view(np.int32)).cuda()


def _noalloc(lib, keys, vals, n, bits, stream):
    out_k, out_v = torch.empty_like(keys), torch.empty_like(vals)
    rc = lib.airgs_sort_pairs_noalloc(_ptr(keys), _ptr(vals), _ptr(out_k), _ptr(out_v), n, bits,
                                      ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    return out_k, out_v


@pytest.mark.parametrize("n,bits", [(70_001, 8), (300_001, 16), (300_001, 17), (1 << 20, 24), (524_289, 32)])
def test_noalloc_sort_matches_stable_argsort_and_allocating_sort(n, bits):
    from paper_2512_20943_b300 import Rasterizer, _abi
    lib = _abi.load_library()
    rast = Rasterizer()
    stream = torch.cuda.current_stream()
    hk, hv = _inputs(n, 10 + bits, bits)
    keys, vals = _dev(hk), _dev(hv)
    ref_k, ref_v = rast.sort_pairs(keys, vals, bits)  # the existing entry point (allocates from its pool)
    out_k, out_v = _noalloc(lib, keys, vals, n, bits, stream)
    torch.cuda.synchronize()
    order = np.argsort(hk & np.uint32((1 << bits) - 1 if bits < 32 else 0xFFFFFFFF), kind="stable")
    got_k, got_v = out_k.cpu().numpy().view(np.uint32), out_v.cpu().numpy().view(np.uint32)
    # integer results: bit-exact against an independent stable sort and the allocating sort
    assert np.array_equal(got_k, hk[order])
    assert np.array_equal(got_v, hv[order])
    assert torch.equal(out_k, ref_k) and torch.equal(out_v, ref_v)
    # inputs untouched
    assert np.array_equal(keys.cpu().numpy().view(np.uint32), hk)
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), hv)


def test_noalloc_sort_two_calls_in_a_row():
    """Consecutive calls share the scratch array; the second (smaller, other
    width) must not see the first's leftovers."""
    from paper_2512_20943_b300 import Rasterizer, _abi
    lib = _abi.load_library()
    rast = Rasterizer()
    stream = torch.cuda.current_stream()
    for call, (n, bits) in enumerate([(1 << 20, 24), (300_001, 17)]):
        hk, hv = _inputs(n, 40 + call, bits)
        keys, vals = _dev(hk), _dev(hv)
        ref_k, ref_v = rast.sort_pairs(keys, vals, bits)
        out_k, out_v = _noalloc(lib, keys, vals, n, bits, stream)
        torch.cuda.synchronize()
        assert torch.equal(out_k, ref_k), call
        assert torch.equal(out_v, ref_v), call


def test_noalloc_sort_rejects_oversize_and_bad_arguments():
    from paper_2512_20943_b300 import _abi
    lib = _abi.load_library()
    n = _abi.AIRGS_NOALLOC_SORT_MAX_PAIRS + 1
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = lib.airgs_sort_pairs_noalloc(_ptr(x), _ptr(x), _ptr(x), _ptr(x), n, 32, None)
    assert rc == _abi.AIRGS_E_CAPACITY
    assert lib.airgs_sort_pairs_noalloc(_ptr(x), _ptr(x), _ptr(x), _ptr(x), 8, 0, None) == _abi.AIRGS_E_ARG
    assert lib.airgs_sort_pairs_noalloc(_ptr(x), _ptr(x), _ptr(x), _ptr(x), 8, 33, None) == _abi.AIRGS_E_ARG
    assert lib.airgs_sort_pairs_noalloc(None, _ptr(x), _ptr(x), _ptr(x), 8, 8, None) == _abi.AIRGS_E_ARG
