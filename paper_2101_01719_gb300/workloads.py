"""Seeded synthetic workloads at the paper's sizes, generated on the device.

Hash streams are splitmix64 in counter form (``fill_splitmix64``); query
streams mix previously inserted hashes with fresh ones (``fill_queries``).
Stream seeds are ``0x5BBF000000000000 | (cfg << 8) | role`` with roles
0 = inserted hashes, 1 = fresh lookups, 2 = member selector, 3 = filter sizes,
4 = order/shuffles, 5 = arrivals, 6 = request sizes.

Sizes follow the paper's benchmark table (100k / 1M / 100M elements in
131,072 B / 1 MiB / 134,217,728 B filters) and the larger cases built on them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import sbbf

ROLE_INSERT, ROLE_FRESH, ROLE_MEMBER, ROLE_SIZES, ROLE_ORDER = 0, 1, 2, 3, 4
ROLE_ARRIVAL, ROLE_REQSIZE = 5, 6


def seed(cfg: int, role: int) -> int:
    return 0x5BBF000000000000 | (cfg << 8) | role


def member_threshold(frac: float) -> int:
    return int(round(frac * 2.0**32))


@dataclass(frozen=True)
class SingleFilterWorkload:
    name: str
    cfg: int                # seed namespace
    num_blocks: int
    n_insert: int
    insert_batch: int       # inserts are issued in batches of this many
    n_lookup: int
    member_frac: float      # fraction of mixed lookups drawn from the inserted set
    member_prefix: int = 0  # the first lookups are inserted hashes 0.. in order

    @property
    def filter_bytes(self) -> int:
        return self.num_blocks * 32

    @property
    def keys_per_block(self) -> float:
        return self.n_insert / self.num_blocks


# 100k hashes into 4096 blocks (131,072 B); 100k member lookups then 1M fresh.
C0 = SingleFilterWorkload("sbbf_4096blk_100k_ins_1.1M_lookup", 0, 4096, 100_000, 100_000,
                          1_100_000, 0.0, member_prefix=100_000)
# 1M hashes into 32768 blocks (1 MiB, L2-resident); 256M lookups, half members.
C1 = SingleFilterWorkload("sbbf_32768blk_1M_ins_256M_lookup", 1, 32768, 1_000_000, 1_000_000,
                          256 * 2**20, 0.5)
# 100M hashes into 4,194,304 blocks (134,217,728 B) in 16M batches; 1B lookups, 10% members.
C2 = SingleFilterWorkload("sbbf_4194304blk_100M_ins_1G_lookup", 2, 4_194_304, 100_000_000,
                          16_000_000, 1_000_000_000, 0.1)
# 3B hashes into 2^30 blocks (32 GiB) in one batch; 1B lookups, 10% members.
C2_BIG = SingleFilterWorkload("sbbf_2^30blk_3G_ins_1G_lookup", 12, 2**30, 3_000_000_000,
                              3_000_000_000, 1_000_000_000, 0.1)
# 3B hashes at 11 bits/key: 128,906,250 blocks (4.125 GB), one batch.
C2_11BPK = SingleFilterWorkload("sbbf_128906250blk_3G_ins_1G_lookup", 22,
                                math.ceil(3_000_000_000 * 11 / 256), 3_000_000_000,
                                3_000_000_000, 1_000_000_000, 0.1)

# The 134,217,728-byte filter with a 64M-lookup batch: a profiling-sized case
# (about 1.5 GB on the device) of the same kernels.
C2_PROFILE = SingleFilterWorkload("sbbf_4194304blk_100M_ins_64M_lookup", 2, 4_194_304,
                                  100_000_000, 16_000_000, 64 * 2**20, 0.1)

# A 2 GiB filter (64 slices) with 128M inserts in one batch and 128M lookups:
# both take the partitioned path in automatic mode (2 keys per block), with
# about 5.5 GB on the device -- a profiling-sized case of the partition,
# scatter and slice-ordered kernels the 32 GiB and 11 bits/key filters use.
C2_PART_PROFILE = SingleFilterWorkload("sbbf_2^26blk_128M_ins_128M_lookup", 32, 2**26,
                                       128 * 2**20, 128 * 2**20, 128 * 2**20, 0.1)

# The same filter with 256M lookups (about 3.2 GB on the device): with the
# 64M case, separates the per-key DRAM traffic of a lookup by region passes
# from the per-pass part (each pass loads its region into L2).
C2_PROFILE_256M = SingleFilterWorkload("sbbf_4194304blk_100M_ins_256M_lookup", 2, 4_194_304,
                                       100_000_000, 16_000_000, 256 * 2**20, 0.1)

WORKLOADS = {w.name: w for w in (C0, C1, C2, C2_BIG, C2_11BPK, C2_PROFILE, C2_PROFILE_256M,
                                 C2_PART_PROFILE)}


def gen_inserts(w: SingleFilterWorkload, start: int, n: int, out: torch.Tensor | None = None,
                device=None, stream=None) -> torch.Tensor:
    """Inserted hashes start..start+n-1 of workload w (device int64)."""
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=device or "cuda")
    sbbf.fill_splitmix64(out[:n], seed(w.cfg, ROLE_INSERT), start, stream)
    return out


def gen_queries(w: SingleFilterWorkload, start: int, n: int, out: torch.Tensor | None = None,
                device=None, stream=None) -> torch.Tensor:
    """Lookup hashes start..start+n-1 of workload w (device int64): lookups
    below member_prefix are inserted hashes in order, the rest follow the
    member/fresh recipe indexed from member_prefix."""
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=device or "cuda")
    p = max(0, min(w.member_prefix - start, n))
    if p > 0:
        sbbf.fill_splitmix64(out[:p], seed(w.cfg, ROLE_INSERT), start, stream)
    if n > p:
        sbbf.fill_queries(out[p:n], start + p - w.member_prefix, seed(w.cfg, ROLE_INSERT), 0,
                          w.n_insert, seed(w.cfg, ROLE_FRESH), seed(w.cfg, ROLE_MEMBER),
                          member_threshold(w.member_frac), stream)
    return out


def build_filter(w: SingleFilterWorkload, f: sbbf.Filter, scratch: torch.Tensor | None = None,
                 stream=None) -> sbbf.Filter:
    """Insert all of w's hashes into f in batches of w.insert_batch."""
    b = min(w.insert_batch, w.n_insert)
    if scratch is None or scratch.numel() < b:
        scratch = torch.empty(b, dtype=torch.int64, device=f.device)
    for s in range(0, w.n_insert, w.insert_batch):
        cnt = min(w.insert_batch, w.n_insert - s)
        gen_inserts(w, s, cnt, scratch, stream=stream)
        f.insert(scratch[:cnt], stream=stream)
    return f


# ---- many filters ------------------------------------------------------------

@dataclass(frozen=True)
class MultiFilterWorkload:
    """n_filters filters with key counts log-uniform in [lo, hi] (role 3),
    sized at bits_per_key rounded up to whole 32-byte blocks.  Inserted keys
    are the role-0 stream, concatenated in filter order; filter t gets
    lookup_factor * n_t lookups rounded up to a multiple of 64 (so each
    filter's answers start a fresh output word), a member_frac share of them
    drawn from filter t's inserted keys."""
    name: str
    cfg: int
    n_filters: int
    lo: float
    hi: float
    bits_per_key: float
    lookup_factor: int
    member_frac: float

    def sizes(self):
        import numpy as np
        u = _uniform01_host(seed(self.cfg, ROLE_SIZES), self.n_filters)
        n_keys = np.rint(np.exp(np.log(self.lo) + u * (np.log(self.hi) - np.log(self.lo))))
        n_keys = n_keys.astype(np.int64)
        blocks = np.maximum(np.ceil(n_keys * self.bits_per_key / 256.0), 1).astype(np.int64)
        return n_keys, blocks

    def offsets(self):
        """(insert offsets, lookup offsets), each n_filters + 1 int64 on the host."""
        import numpy as np
        n_keys, _ = self.sizes()
        q = ((self.lookup_factor * n_keys + 63) // 64) * 64
        ins = np.concatenate([[0], np.cumsum(n_keys)]).astype(np.int64)
        qo = np.concatenate([[0], np.cumsum(q)]).astype(np.int64)
        return ins, qo


def _uniform01_host(sd: int, n: int):
    """Uniform doubles in [0,1) from the top 53 bits of a splitmix64 stream."""
    import numpy as np
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(sd) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * 2.0**-53


# 4096 filters, 1k..4M keys each at 10.5 bits/key; 4x lookups, half members.
C3 = MultiFilterWorkload("sbbf_4096filters_1k-4M_keys_10.5bpk_4x_lookup", 3, 4096, 1e3, 4e6,
                         10.5, 4, 0.5)
# A smaller instance of the same recipe for quick checks.
C3_SMALL = MultiFilterWorkload("sbbf_256filters_1k-200k_keys_10.5bpk_4x_lookup", 13, 256, 1e3,
                               2e5, 10.5, 4, 0.5)
MULTI_WORKLOADS = {w.name: w for w in (C3, C3_SMALL)}


def gen_multi(w: MultiFilterWorkload, device=None, stream=None):
    """Device tensors for workload w: inserted hashes, insert offsets, lookup
    hashes, lookup offsets (offsets int64, n_filters + 1)."""
    ins_off, q_off = w.offsets()
    dev = device or "cuda"
    d_ins_off = torch.from_numpy(ins_off).to(dev)
    d_q_off = torch.from_numpy(q_off).to(dev)
    ins = torch.empty(int(ins_off[-1]), dtype=torch.int64, device=dev)
    sbbf.fill_splitmix64(ins, seed(w.cfg, ROLE_INSERT), 0, stream)
    q = torch.empty(int(q_off[-1]), dtype=torch.int64, device=dev)
    sbbf.fill_segment_queries(q, d_q_off, d_ins_off, seed(w.cfg, ROLE_INSERT),
                              seed(w.cfg, ROLE_FRESH), seed(w.cfg, ROLE_MEMBER),
                              member_threshold(w.member_frac), stream)
    return ins, d_ins_off, q, d_q_off


# ---- serving -------------------------------------------------------------------

@dataclass(frozen=True)
class ServingWorkload:
    """n_filters resident filters with byte sizes log-uniform in
    [size_lo, size_hi] (role 3), each pre-filled to prefill_bits_per_key with
    role-0 hashes (filter t takes the next m_t outputs); requests with sizes
    log-uniform in [req_lo, req_hi] (role 6), a lookup_frac share lookups
    (role 2), filters uniform (role 4), payloads slices of a pool of
    pool_hashes role-1 hashes at uniform offsets (role 1 again, separate
    index range) and Poisson arrivals (role 5)."""
    name: str
    cfg: int
    n_filters: int
    size_lo: float
    size_hi: float
    budget_bytes: int
    n_requests: int
    lookup_frac: float
    req_lo: float
    req_hi: float
    prefill_bits_per_key: float
    pool_hashes: int

    def filter_blocks(self):
        import numpy as np
        u = _uniform01_host(seed(self.cfg, ROLE_SIZES), self.n_filters)
        b = np.exp(np.log(self.size_lo) + u * (np.log(self.size_hi) - np.log(self.size_lo)))
        return np.maximum(np.rint(b / 32.0), 1).astype(np.int64)

    def prefill_counts(self):
        import numpy as np
        return np.floor(self.filter_blocks() * 256.0 / self.prefill_bits_per_key).astype(np.int64)

    def requests(self, n: int, rate_per_s: float):
        """(op, filter, size, pool offset, arrival ns) for the first n
        requests at `rate_per_s` requests per second (inf: all at t=0)."""
        import numpy as np
        from . import sbbf as _s
        sizes = np.rint(np.exp(np.log(self.req_lo) + _uniform01_host(
            seed(self.cfg, ROLE_REQSIZE), n) * (np.log(self.req_hi) - np.log(self.req_lo))))
        sizes = np.clip(sizes, 1, self.pool_hashes).astype(np.uint64)
        op = np.where(_uniform01_host(seed(self.cfg, ROLE_MEMBER), n) < self.lookup_frac,
                      _s.OP_FIND, _s.OP_INSERT).astype(np.uint32)
        filt = np.floor(_uniform01_host(seed(self.cfg, ROLE_ORDER), n)
                        * self.n_filters).astype(np.uint32)
        span = (self.pool_hashes - sizes + 1).astype(np.float64)
        off = np.floor(_uniform01_host(seed(self.cfg, ROLE_FRESH) ^ 0x5A5A, n) * span)
        off = off.astype(np.uint64)
        if np.isinf(rate_per_s):
            arrival = np.zeros(n, np.uint64)
        else:
            gaps = -np.log1p(-_uniform01_host(seed(self.cfg, ROLE_ARRIVAL), n)) / rate_per_s
            arrival = np.rint(np.cumsum(gaps) * 1e9).astype(np.uint64)
        return op, filt, sizes, off, arrival


C4 = ServingWorkload("sbbf_serve_256filters_128KiB-1GiB_70pct_lookup", 4, 256, 128 * 2**10,
                     2**30, 80 * 10**9, 10_000_000, 0.7, 1, 1e6, 10.5, 1 << 27)
C4_SMALL = ServingWorkload("sbbf_serve_32filters_4KiB-4MiB_70pct_lookup", 14, 32, 4 * 2**10,
                           4 * 2**20, 64 * 2**20, 20_000, 0.7, 1, 2e4, 10.5, 1 << 22)
SERVING_WORKLOADS = {w.name: w for w in (C4, C4_SMALL)}


def request_records(op, filt, sizes, off, pool: torch.Tensor, out: torch.Tensor,
                    ring_words: int | None = None):
    """REQUEST_DTYPE records pointing into the hash pool and an output area:
    lookups get consecutive 32-byte-aligned output slices (wrapping around
    after ring_words words when given)."""
    import numpy as np
    from . import sbbf as _s
    n = len(op)
    rec = np.zeros(n, dtype=_s.REQUEST_DTYPE)
    rec["op"], rec["filter"], rec["n"] = op, filt, sizes
    rec["hashes"] = np.uint64(pool.data_ptr()) + off * np.uint64(8)
    words = ((sizes + np.uint64(31)) // np.uint64(32) + np.uint64(7)) // np.uint64(8) * np.uint64(8)
    words = np.where(op == _s.OP_FIND, words, 0).astype(np.uint64)
    start = np.concatenate([[0], np.cumsum(words)[:-1]]).astype(np.uint64)
    if ring_words:
        start = start % np.uint64(ring_words)
        over = start + words > np.uint64(ring_words)
        start[over] = 0
    rec["out"] = np.where(op == _s.OP_FIND, np.uint64(out.data_ptr()) + start * np.uint64(4), 0)
    return rec, start, words


def gen_inserts_seeded(sd: int, start: int, n: int, device=None, out=None, stream=None):
    """splitmix64 outputs start..start+n-1 of seed sd (device int64)."""
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=device or "cuda")
    sbbf.fill_splitmix64(out[:n], sd, start, stream)
    return out[:n]


def prefill_server(w: ServingWorkload, srv, chunk: int = 1 << 28, device=None):
    """Register w's filters on srv and pre-fill each one; returns the blocks."""
    import numpy as np
    blocks = w.filter_blocks()
    counts = w.prefill_counts()
    start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    buf = torch.empty(min(chunk, int(counts.max()) or 1), dtype=torch.int64,
                      device=device or "cuda")
    for t, b in enumerate(blocks):
        fid = srv.add_filter(int(b))
        for s0 in range(0, int(counts[t]), chunk):
            c = min(chunk, int(counts[t]) - s0)
            srv.prefill(fid, gen_inserts_seeded(seed(w.cfg, ROLE_INSERT), int(start[t]) + s0, c,
                                                out=buf))
    return blocks
