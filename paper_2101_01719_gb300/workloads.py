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
# 3B hashes into 2^30 blocks (32 GiB); 1B lookups, 10% members.
C2_BIG = SingleFilterWorkload("sbbf_2^30blk_3G_ins_1G_lookup", 12, 2**30, 3_000_000_000,
                              256 * 2**20, 1_000_000_000, 0.1)
# 3B hashes at 11 bits/key: 128,906,250 blocks (4.125 GB).
C2_11BPK = SingleFilterWorkload("sbbf_128906250blk_3G_ins_1G_lookup", 22,
                                math.ceil(3_000_000_000 * 11 / 256), 3_000_000_000,
                                256 * 2**20, 1_000_000_000, 0.1)

WORKLOADS = {w.name: w for w in (C0, C1, C2, C2_BIG, C2_11BPK)}


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
