"""The allocation-free lookup entry point, sbbf_multi_find_noalloc.

It exists for callers that must not allocate device memory while looking
keys up: a serving loop that admits work against a fixed device-memory
budget, a framework whose caching allocator owns the device memory, or a
latency-critical caller that cannot pay for the device-wide synchronisation
of cudaFree.  Its only scratch is a static device array inside the library.

These tests call it through the C ABI and compare it with the allocating
entry point (sbbf_multi_find) bit for bit -- the tolerance of every parity
test here, since all results are integers -- on two calls in a row, the
second on a smaller set so that directory entries left over from the first
call would show up as wrong answers.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2101_01719_gb300 as sb
from paper_2101_01719_gb300 import sbbf as abi
import sbbf_inputs as inp
from gpu_util import bits_np, dev, to_dev

pytestmark = pytest.mark.gpu


def _arena_ptr(m):
    p, nbytes = ctypes.c_void_p(), ctypes.c_size_t()
    assert abi.lib().sbbf_multi_device_words(m._h, ctypes.byref(p), ctypes.byref(nbytes)) == 0
    return p.value


def _one_call(sizes, cfg, n_keys, n_queries):
    """Build a set with the allocating API, then look up the same queries
    through both entry points; returns (noalloc bits, reference bits,
    noalloc invalid count, reference invalid count)."""
    sizes = np.asarray(sizes, np.uint32)
    m = sb.MultiFilter(sizes)
    keys = inp.stream(cfg, 0, n_keys)
    ids = (inp.stream(cfg, 4, n_keys) % np.uint64(sizes.size)).astype(np.uint32)
    m.insert(to_dev(keys), ids=torch.from_numpy(ids.view(np.int32)).to(dev()))
    q = np.concatenate([inp.stream(cfg, 1, n_queries - n_keys // 2), keys[: n_keys // 2]])
    qid = (inp.stream(cfg, 5, q.size) % np.uint64(sizes.size + 2)).astype(np.uint32)
    d_q = to_dev(q)
    d_qid = torch.from_numpy(qid.view(np.int32)).to(dev())
    ref = m.find(d_q, ids=d_qid)
    ref_invalid = m.invalid_count()

    d_sizes = torch.from_numpy(sizes.view(np.int32)).to(dev())
    out = torch.full((sb.out_words(q.size),), -1, dtype=torch.int32, device=dev())
    count = torch.full((1,), -1, dtype=torch.int64, device=dev())
    rc = abi.lib().sbbf_multi_find_noalloc(
        _arena_ptr(m), d_sizes.data_ptr(), sizes.size, d_q.data_ptr(), d_qid.data_ptr(), q.size,
        out.data_ptr(), count.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == abi.SBBF_OK, abi.lib().sbbf_status_string(rc)
    torch.cuda.synchronize()
    return bits_np(out), bits_np(ref), int(count.item()), ref_invalid


def test_noalloc_lookup_matches_allocating_lookup_twice():
    got1, ref1, inv1, ref_inv1 = _one_call([1, 3, 64, 4096, 777, 100_003, 5, 2, 31_250],
                                           cfg=60, n_keys=400_000, n_queries=1_000_003)
    assert np.array_equal(got1, ref1)
    assert inv1 == ref_inv1 and inv1 > 0
    # second call: fewer filters; ids 3.. must now count as invalid even though
    # the first call left directory entries for them in the shared scratch
    got2, ref2, inv2, ref_inv2 = _one_call([50, 7, 2000], cfg=61, n_keys=50_000,
                                           n_queries=300_001)
    assert np.array_equal(got2, ref2)
    assert inv2 == ref_inv2 and inv2 > 0


def test_noalloc_limits_and_empty_batch():
    L = abi.lib()
    m = sb.MultiFilter([8, 8])
    d_sizes = torch.tensor([8, 8], dtype=torch.int32, device=dev())
    count = torch.full((1,), -1, dtype=torch.int64, device=dev())
    s = torch.cuda.current_stream().cuda_stream
    too_many = L.sbbf_multi_find_noalloc(_arena_ptr(m), d_sizes.data_ptr(), 65537,
                                         None, None, 0, None, None, s)
    assert too_many == abi.SBBF_ERANGE
    assert L.sbbf_multi_find_noalloc(_arena_ptr(m), d_sizes.data_ptr(), 0, None, None, 0, None,
                                     None, s) == abi.SBBF_EINVAL
    # an empty batch still reports a zero count
    assert L.sbbf_multi_find_noalloc(_arena_ptr(m), d_sizes.data_ptr(), 2, None, None, 0, None,
                                     count.data_ptr(), s) == abi.SBBF_OK
    torch.cuda.synchronize()
    assert int(count.item()) == 0
