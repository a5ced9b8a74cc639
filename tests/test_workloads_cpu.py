"""Host-side logic of the seeded workloads (no GPU): the configurations match
the paper's sizes and the readings of them, and the host generators of filter
sizes, multi-filter offsets and serving requests are deterministic and have
the stated distributions."""
import numpy as np
import pytest
import torch

from paper_2101_01719_gb300 import sbbf
from paper_2101_01719_gb300 import workloads as wl


def test_single_filter_configs_match_the_paper_sizes():
    # the benchmark table's 100k / 1M / 100M elements in 131,072 B / 1 MiB /
    # 134,217,728 B filters, and the two readings of the 3e9-hash filter
    assert (wl.C0.filter_bytes, wl.C0.n_insert) == (131_072, 100_000)
    assert (wl.C1.filter_bytes, wl.C1.n_insert, wl.C1.n_lookup) == (2**20, 10**6, 2**28)
    assert (wl.C2.filter_bytes, wl.C2.n_insert, wl.C2.insert_batch) == (2**27, 10**8, 16 * 10**6)
    assert wl.C2_BIG.num_blocks == 2**30 and wl.C2_BIG.n_insert == 3 * 10**9
    assert abs(wl.C2_11BPK.num_blocks * 256 / wl.C2_11BPK.n_insert - 11.0) < 1e-9
    assert wl.C1.member_frac == 0.5 and wl.C2.member_frac == 0.1
    assert wl.member_threshold(0.1) == 429_496_730  # round(0.1 * 2^32)
    assert wl.seed(3, wl.ROLE_SIZES) == 0x5BBF000000000303


def test_multi_filter_sizes_and_offsets():
    w = wl.C3
    n_keys, blocks = w.sizes()
    n2, b2 = w.sizes()
    assert np.array_equal(n_keys, n2) and np.array_equal(blocks, b2)  # deterministic
    assert n_keys.size == 4096 and n_keys.min() >= 1000 and n_keys.max() <= 4_000_000
    assert np.array_equal(blocks, np.maximum(np.ceil(n_keys * 10.5 / 256.0), 1))
    # log-uniform: the mean of log(n) sits at the middle of [log 1e3, log 4e6]
    mid = 0.5 * (np.log(1e3) + np.log(4e6))
    assert abs(np.log(n_keys).mean() - mid) < 0.1
    ins, qo = w.offsets()
    assert ins[0] == 0 and np.array_equal(np.diff(ins), n_keys)
    q = np.diff(qo)
    assert (q % 64 == 0).all() and (q >= 4 * n_keys).all() and (q < 4 * n_keys + 64).all()


def test_serving_requests_are_deterministic_with_the_stated_distribution():
    w = wl.C4
    n = 200_000
    op, filt, size, off, arr = w.requests(n, 1e5)
    op2, filt2, size2, off2, arr2 = w.requests(n, 1e5)
    for a, b in ((op, op2), (filt, filt2), (size, size2), (off, off2), (arr, arr2)):
        assert np.array_equal(a, b)
    lookups = (op == sbbf.OP_FIND).mean()
    assert abs(lookups - 0.7) < 5 * np.sqrt(0.21 / n)
    assert filt.max() < w.n_filters and np.unique(filt).size == w.n_filters
    assert size.min() >= 1 and size.max() <= w.req_hi
    assert (off + size <= w.pool_hashes).all()
    # log-uniform sizes on [1, 1e6]: mean (1e6 - 1) / ln(1e6) = 72,382
    assert abs(size.mean() / 72_382 - 1) < 0.05
    gaps = np.diff(arr.astype(np.int64))
    assert (gaps >= 0).all() and abs(gaps.mean() / 1e4 - 1) < 0.02  # 1e5 requests/s
    _, _, _, _, at_once = w.requests(1000, float("inf"))
    assert not at_once.any()


def test_serving_filter_sizes_and_prefill():
    w = wl.C4
    blocks = w.filter_blocks()
    assert blocks.size == 256
    assert blocks.min() * 32 >= 128 * 2**10 - 32 and blocks.max() * 32 <= 2**30 + 32
    assert np.array_equal(w.prefill_counts(), np.floor(blocks * 256.0 / 10.5).astype(np.int64))


def test_request_records_give_lookups_aligned_outputs():
    w = wl.C4_SMALL
    op, filt, size, off, _ = w.requests(5000, float("inf"))
    pool = torch.zeros(w.pool_hashes, dtype=torch.int64)
    ring = 1 << 16
    out = torch.zeros(ring + (1 << 12), dtype=torch.int32)
    rec, start, words = wl.request_records(op, filt, size, off, pool, out, ring)
    look = op == sbbf.OP_FIND
    assert (rec["out"][~look] == 0).all() and (words[~look] == 0).all()
    assert (rec["hashes"] == pool.data_ptr() + off * 8).all()
    o = (rec["out"][look] - out.data_ptr())
    assert (o % 32 == 0).all()  # 32-byte aligned slices
    assert (start[look] + words[look] <= ring).all()
    assert (words[look] * 32 >= size[look]).all()
    # before the ring first wraps, lookups get consecutive, disjoint slices
    total = np.cumsum(words.astype(np.int64)) - words.astype(np.int64)
    first = look & (total + words.astype(np.int64) <= ring)
    assert first.sum() > 10 and (start[first] == total[first]).all()
