"""One split block Bloom filter sharded by block range over the ranks of a
process group (one GPU per rank).

The appendix's block_index sends every hash to exactly one block; shard s of
G owns global blocks [s P, min(B, (s + 1) P)), P = ceil(B / G)
(sbbf_shard_range), so the shards together are the unsharded filter bit for
bit.  Every rank brings its own batch:

- insert: group the batch by owner shard (sbbf_shard_route), exchange the
  per-owner counts and then the hashes with an all-to-all, and insert the
  hashes received into the local shard (sbbf_shard_insert);
- find: route with each owner's group padded to whole 32-bit answer words,
  exchange as for inserts, look the received hashes up in the local shard
  (sbbf_shard_find), send the answer words back with the reverse all-to-all
  and put them in query order (sbbf_shard_unpermute).

The device steps are the library's kernels (``DeviceOps``); the exchanges go
through a communicator (``TorchComm``: torch.distributed, NCCL between GPUs).
Both are parameters, so the exchange logic can run with other transports.
"""
from __future__ import annotations

import torch

from . import sbbf


class TorchComm:
    """all-to-all exchanges over a torch.distributed process group; tensors
    live on `device` (CUDA tensors for NCCL, CPU tensors for gloo)."""

    def __init__(self, group=None, device=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device = torch.device(device) if device is not None else torch.device("cpu")

    def exchange_counts(self, send: list[int]) -> list[int]:
        """recv[r] = what rank r sends to this rank (send[r] from this rank to r)."""
        t = torch.tensor(send, dtype=torch.int64, device=self.device)
        out = torch.empty_like(t)
        self.dist.all_to_all_single(out, t, group=self.group)
        return [int(v) for v in out.tolist()]

    def all_to_all(self, out: torch.Tensor, inp: torch.Tensor, out_splits, in_splits):
        self.dist.all_to_all_single(out, inp, list(out_splits), list(in_splits), group=self.group)


class DeviceOps:
    """The device steps, on the library's kernels (see sbbf.h)."""

    def __init__(self, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)

    def shard_range(self, num_blocks: int, n_shards: int, shard: int):
        return sbbf.shard_range(num_blocks, n_shards, shard)

    def new_local(self, n_blocks: int):
        return sbbf.Filter(n_blocks, device=self.device)

    def route(self, hashes: torch.Tensor, num_blocks: int, n_shards: int, pad: bool):
        routed, perm, counts = sbbf.shard_route(hashes, num_blocks, n_shards, pad)
        return routed, perm, [int(c) for c in counts.tolist()]  # the counts size the exchange

    def empty_keys(self, n: int) -> torch.Tensor:
        return torch.empty(n, dtype=torch.int64, device=self.device)

    def empty_words(self, n: int) -> torch.Tensor:
        return torch.empty(n, dtype=torch.int32, device=self.device)

    def local_insert(self, local, num_blocks: int, lo: int, keys: torch.Tensor):
        sbbf.shard_insert(local, num_blocks, lo, keys)

    def local_find(self, local, num_blocks: int, lo: int, keys: torch.Tensor) -> torch.Tensor:
        return sbbf.shard_find(local, num_blocks, lo, keys)

    def unpermute(self, words: torch.Tensor, perm: torch.Tensor, n_routed: int,
                  n: int) -> torch.Tensor:
        return sbbf.shard_unpermute(words, perm, n_routed, n)

    def local_words(self, local):
        return local.to_numpy()


class ShardedFilter:
    """This rank's shard of a num_blocks-block filter split over the ranks of
    `comm` (see the module docstring).  insert() and find() are collective:
    every rank calls them, each with its own batch (possibly empty)."""

    def __init__(self, num_blocks: int, comm=None, ops=None, device=None):
        self.ops = ops if ops is not None else DeviceOps(device)
        self.comm = comm if comm is not None else TorchComm(
            device=getattr(self.ops, "device", None))
        self.num_blocks = int(num_blocks)
        self.world, self.rank = self.comm.world, self.comm.rank
        self.lo, self.hi = self.ops.shard_range(self.num_blocks, self.world, self.rank)
        self.local = self.ops.new_local(self.hi - self.lo) if self.hi > self.lo else None

    def _exchange(self, routed, counts):
        send = list(counts)
        recv = self.comm.exchange_counts(send)
        keys = self.ops.empty_keys(sum(recv))
        self.comm.all_to_all(keys, routed[: sum(send)], recv, send)
        return keys, send, recv

    def insert(self, hashes: torch.Tensor):
        routed, _, counts = self.ops.route(hashes, self.num_blocks, self.world, False)
        keys, _, _ = self._exchange(routed, counts)
        if self.local is not None and keys.numel():
            self.ops.local_insert(self.local, self.num_blocks, self.lo, keys)
        return self

    def find(self, hashes: torch.Tensor) -> torch.Tensor:
        """Packed answers ((n + 31) // 32 int32 words, bit k for hashes[k])."""
        n = hashes.numel()
        routed, perm, counts = self.ops.route(hashes, self.num_blocks, self.world, True)
        keys, send, recv = self._exchange(routed, counts)
        if self.local is not None and keys.numel():
            answers = self.ops.local_find(self.local, self.num_blocks, self.lo, keys)
        else:
            answers = self.ops.empty_words(0)
        # every group is a whole number of answer words: what came from rank r
        # (recv[r] hashes) goes back to r as recv[r] / 32 words
        back = self.ops.empty_words(sum(send) // 32)
        self.comm.all_to_all(back, answers[: sum(recv) // 32], [c // 32 for c in send],
                             [c // 32 for c in recv])
        return self.ops.unpermute(back, perm, sum(send), n)

    def local_words(self):
        """This shard's words (global blocks [lo, hi)) on the host."""
        return None if self.local is None else self.ops.local_words(self.local)
