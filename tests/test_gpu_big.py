"""Full-size parity for the HBM-resident filters with 3e9 inserted hashes:
2^30 blocks (32 GiB) and 128,906,250 blocks (11 bits/key), 1e9 lookups with
10% members, in the batches the benchmark uses.  The oracle rebuilds each
filter whole on the host (all cores, each thread owning a block range), and
every word and every one of the 1e9 answers must match; the random and the
slice-ordered lookup paths must give the same answers; the device's
block-range digest must equal the oracle's; the whole output is
also checked statistically (members always hit; the false positive count of
the non-members within a Poisson interval of the formula)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2101_01719_gb300 as sb
from paper_2101_01719_gb300 import workloads as wl
import sbbf_inputs as inp
from gpu_util import (bit_at, bits_np, compare_all_lookups, compare_words, dev,
                      oracle_filter_of_stream, to_dev, u64_np)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("w", [wl.C2_BIG, wl.C2_11BPK], ids=lambda w: w.name)
def test_three_billion_inserts_full_parity(w):
    f = sb.Filter(w.num_blocks)
    buf = torch.empty(w.insert_batch, dtype=torch.int64, device=dev())
    wl.build_filter(w, f, scratch=buf)
    del buf
    q = wl.gen_queries(w, 0, w.n_lookup)
    bits = f.find(q)
    other = sb.PARTITION_OFF if f.partition_applies(w.n_lookup, lookup=True) else sb.PARTITION_ON
    f.set_partitioning(other)
    assert torch.equal(f.find(q), bits)  # the other lookup path, the same answers
    f.set_partitioning(sb.PARTITION_AUTO)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    ref = oracle_filter_of_stream(w)
    compare_words(f.words, ref)
    compare_all_lookups(w, ref, q, bits)
    # the block-range digest in one device pass, against the oracle's over
    # its rebuilt filter; no block has a zero lane beside a non-zero one
    R = 1 << 20
    got = [t.cpu().numpy().view(np.uint64) for t in f.range_digest(R)]
    exp = oracle.range_digest(ref, 8, R, threads=oracle.num_cores())
    for g, e in zip(got, exp):
        assert np.array_equal(g, e)
    assert not exp[2].any()
    del ref

    # statistics over all 1e9 answers
    r = torch.empty(w.n_lookup, dtype=torch.int64, device=dev())
    sb.fill_splitmix64(r, wl.seed(w.cfg, wl.ROLE_MEMBER), 0)
    members = int((((r >> 32) & 0xFFFFFFFF) < wl.member_threshold(w.member_frac)).sum().item())
    del r
    hits = int(sb.count_bits(bits, w.n_lookup).item())
    p = oracle.fpr_poisson(w.n_insert / w.num_blocks)
    lam = p * (w.n_lookup - members)
    assert hits >= members
    assert abs((hits - members) - lam) <= 6 * np.sqrt(lam) + 0.02 * lam + 10
    del f, q, bits
    torch.cuda.empty_cache()


@pytest.mark.parametrize("slices", [1600, 3000])
def test_partitioned_paths_with_small_scatter_tiles(slices):
    """Filters of 1600 slices (50 GiB) and 3000 slices (94 GiB) take the
    scatter's 4096-key tiles: for lookups past ~1578 slices and for inserts
    past ~2944 (8192-key tiles, positions and slice tables no longer fit in
    shared memory together).  A few million keys are inserted and looked up
    partitioned; the touched blocks are rebuilt by the oracle, every member
    hits, and every answer equals the unpartitioned lookup of the same
    filter."""
    B, n = slices * 2**20 + 17, 4_000_001
    keys = inp.stream(160, 0, n)
    f = sb.Filter(B).set_partitioning(sb.PARTITION_ON)
    f.insert(to_dev(keys))
    blocks = np.unique(np.array([oracle.block_index(int(h), B) for h in keys[::97]], np.uint64))
    got = f.words.view(-1, 8)[torch.from_numpy(blocks.astype(np.int64)).to(dev())]
    exp = oracle.insert_block_ranges(np.zeros(8 * blocks.size, np.uint32), B, keys, blocks,
                                     blocks + np.uint64(1))
    assert np.array_equal(got.cpu().numpy().view(np.uint32).ravel(), exp)
    q = np.concatenate([inp.stream(160, 1, n), keys[: n // 4]])
    dq = to_dev(q)
    part = bits_np(f.find(dq))
    f.set_partitioning(sb.PARTITION_OFF)
    assert np.array_equal(part, bits_np(f.find(dq)))
    tail = np.unpackbits(part.view(np.uint8), bitorder="little")[n: n + n // 4]
    assert tail.all()
    del f
    torch.cuda.empty_cache()


def test_partitioned_lookup_over_two_billion_keys():
    """A partitioned lookup of 2^31 + 4103 hashes runs in two pieces (the
    scatter's positions are 32-bit): every answer equals the unpartitioned
    lookup's, and the answers on both sides of the piece boundary and at
    sampled positions equal the oracle's."""
    B, n = 2**23 + 5, 2**31 + 4103
    keys = inp.stream(180, 0, 4_000_000)
    ref = oracle.new_filter(B)
    oracle.insert_mt(ref, B, keys, oracle.num_cores())
    f = sb.Filter(B)
    f.words.copy_(torch.from_numpy(ref.view(np.int32)).to(dev()))
    q = sb.fill_splitmix64(torch.empty(n, dtype=torch.int64, device=dev()),
                           inp.stream_seed(180, 1))
    dk = to_dev(keys)
    q[: 509 * keys.size: 509] = dk                # members spread over the first piece
    q[2**31 - 2000: 2**31 + 2000] = dk[:4000]     # and across the boundary
    f.set_partitioning(sb.PARTITION_ON)
    part = f.find(q)
    f.set_partitioning(sb.PARTITION_OFF)
    assert torch.equal(part, f.find(q))
    pos = np.concatenate([np.arange(2**31 - 3000, 2**31 + 3000),
                          np.random.default_rng(180).integers(0, n, 20000), [n - 1]])
    hq = u64_np(q[torch.from_numpy(pos).to(dev())])
    exp = oracle.find(ref, B, hq)
    got = bit_at(bits_np(part), pos)
    assert np.array_equal(got, bit_at(exp, np.arange(pos.size)))
    assert got[1000:5000].all()                   # the members across the boundary
    del q, part
    torch.cuda.empty_cache()
