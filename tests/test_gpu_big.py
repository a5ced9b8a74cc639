"""Full-size parity for the HBM-resident filters with 3e9 inserted hashes:
2^30 blocks (32 GiB) and 128,906,250 blocks (11 bits/key), 1e9 lookups with
10% members, in the batches the benchmark uses.  Filters this size cannot be
rebuilt on the host quickly, so the oracle rebuilds exactly the blocks that a
sample of lookups land in (plus two contiguous block ranges) from all 3e9
hashes, and every sampled lookup and every rebuilt block must match; the
whole output is also checked statistically (members always hit; the false
positive count of the non-members within a Poisson interval of the formula)."""
import concurrent.futures

import numpy as np
import pytest
import torch

import oracle
import paper_2101_01719_gb300 as sb
from paper_2101_01719_gb300 import workloads as wl
import sbbf_inputs as inp
from gpu_util import bit_at, bits_np, dev, to_dev, u64_np

pytestmark = pytest.mark.gpu


def _oracle_blocks(w, lo, hi, chunk=1 << 25, threads=8):
    """Blocks [lo[r], hi[r]) of w's filter after all its inserts, by the
    oracle, scanning the insert stream in chunks on several threads."""
    size = 8 * int((hi - lo).sum())
    sd = wl.seed(w.cfg, wl.ROLE_INSERT)
    starts = list(range(0, w.n_insert, chunk))

    def part(s0):
        keys = oracle.splitmix64_fill(sd, s0, min(chunk, w.n_insert - s0))
        out = np.zeros(size, np.uint32)
        return oracle.insert_block_ranges(out, w.num_blocks, keys, lo, hi)

    total = np.zeros(size, np.uint32)
    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        for p in ex.map(part, starts):
            total |= p
    return total


@pytest.mark.parametrize("w", [wl.C2_BIG, wl.C2_11BPK], ids=lambda w: w.name)
def test_three_billion_inserts_sampled_parity(w):
    f = sb.Filter(w.num_blocks)
    buf = torch.empty(w.insert_batch, dtype=torch.int64, device=dev())
    wl.build_filter(w, f, scratch=buf)
    del buf
    q = wl.gen_queries(w, 0, w.n_lookup)
    bits = f.find(q)
    torch.cuda.synchronize()

    rng = np.random.default_rng(w.cfg)
    idx = np.sort(rng.choice(w.n_lookup, size=512, replace=False)).astype(np.uint64)
    qs = inp.sampled_queries(w.cfg, w.n_insert, w.member_frac, 0, idx)
    assert np.array_equal(q[torch.from_numpy(idx.astype(np.int64)).to(dev())].cpu().numpy()
                          .view(np.uint64), qs)
    qb = np.array([oracle.block_index(int(h), w.num_blocks) for h in qs], np.uint64)
    blocks = np.unique(qb)
    lo = np.concatenate([blocks, [0, w.num_blocks - 2048]]).astype(np.uint64)
    hi = np.concatenate([blocks + 1, [2048, w.num_blocks]]).astype(np.uint64)
    order = np.argsort(lo, kind="stable")
    lo, hi = lo[order], hi[order]
    keep = np.ones(lo.size, bool)  # drop single blocks inside the two ranges
    for i in range(1, lo.size):
        if lo[i] < hi[:i][keep[:i]].max(initial=0):
            keep[i] = False
    lo, hi = lo[keep], hi[keep]
    expect = _oracle_blocks(w, lo, hi)

    words = f.words.view(-1, 8)
    got = torch.cat([words[int(a): int(b)] for a, b in zip(lo, hi)]).cpu().numpy()
    assert np.array_equal(got.view(np.uint32).reshape(-1), expect)

    # every sampled lookup against its rebuilt block
    first = np.concatenate([[0], np.cumsum(hi - lo)[:-1]]).astype(np.uint64)
    ans = bit_at(bits.cpu().numpy().view(np.uint32), idx.astype(np.int64))
    for j, (h, b) in enumerate(zip(qs, qb)):
        r = int(np.searchsorted(lo, b, side="right") - 1)
        off = int(first[r] + (b - lo[r]))
        blk = expect[8 * off: 8 * off + 8].copy()
        assert bool(ans[j]) == oracle.find_one(blk, 1, int(h) & 0xFFFFFFFF), j

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
