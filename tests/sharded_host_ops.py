"""Host stand-ins for the sharded filter's device steps (tests only): the
route, local insert / lookup and answer reassembly of
paper_2101_01719_gb300.sharded.DeviceOps, written on numpy, with the local
shard's arithmetic done by the oracle.  They let the exchange logic of
ShardedFilter run on CPU ranks (gloo), where no kernel can run."""
import numpy as np
import torch

import oracle
from paper_2101_01719_gb300 import sbbf

PAD_PERM = 0xFFFFFFFF


def block_index_np(h: np.ndarray, num_blocks: int) -> np.ndarray:
    return ((h >> np.uint64(32)) * np.uint64(num_blocks)) >> np.uint64(32)


class HostOps:
    device = torch.device("cpu")

    def shard_range(self, num_blocks, n_shards, shard):
        return sbbf.shard_range(num_blocks, n_shards, shard)  # arithmetic only, no device

    def new_local(self, n_blocks):
        return oracle.new_filter(n_blocks)

    def route(self, hashes, num_blocks, n_shards, pad):
        h = hashes.numpy().view(np.uint64)
        per = -(-num_blocks // n_shards)
        owner = (block_index_np(h, num_blocks) // np.uint64(per)).astype(np.int64)
        order = np.argsort(owner, kind="stable")
        routed, perm, counts = [], [], []
        for g in range(n_shards):
            idx = order[owner[order] == g]
            keys = h[idx]
            pos = idx.astype(np.uint32)
            if pad and keys.size % 32:
                lo = g * per
                x = ((lo << 32) + num_blocks - 1) // num_blocks  # a hash of block lo
                extra = 32 - keys.size % 32
                keys = np.concatenate([keys, np.full(extra, x << 32, np.uint64)])
                pos = np.concatenate([pos, np.full(extra, PAD_PERM, np.uint32)])
            routed.append(keys)
            perm.append(pos)
            counts.append(int(keys.size))
        routed = np.concatenate(routed) if routed else np.zeros(0, np.uint64)
        perm = np.concatenate(perm) if perm else np.zeros(0, np.uint32)
        return (torch.from_numpy(routed.view(np.int64).copy()),
                torch.from_numpy(perm.view(np.int32).copy()), counts)

    def empty_keys(self, n):
        return torch.empty(n, dtype=torch.int64)

    def empty_words(self, n):
        return torch.empty(n, dtype=torch.int32)

    def local_insert(self, local, num_blocks, lo, keys):
        hi = lo + local.size // 8
        oracle.insert_block_range(local, num_blocks, keys.numpy().view(np.uint64), lo, hi)

    def local_find(self, local, num_blocks, lo, keys):
        full = oracle.new_filter(num_blocks)
        full[8 * lo: 8 * lo + local.size] = local
        bits = oracle.find(full, num_blocks, keys.numpy().view(np.uint64))
        return torch.from_numpy(bits.view(np.int32).copy())

    def unpermute(self, words, perm, n_routed, n):
        w = words.numpy().view(np.uint32)
        p = perm.numpy().view(np.uint32)[:n_routed]
        bit = ((w[np.arange(n_routed) // 32] >> (np.arange(n_routed) % 32).astype(np.uint32))
               & np.uint32(1)).astype(bool)
        out = np.zeros((n + 31) // 32, np.uint32)
        hits = p[bit & (p != PAD_PERM)].astype(np.int64)
        np.bitwise_or.at(out, hits // 32, (np.uint32(1) << (hits % 32).astype(np.uint32)))
        return torch.from_numpy(out.view(np.int32))

    def local_words(self, local):
        return local.copy()
