"""The sharded filter's device steps on one GPU: G virtual shards, one host
thread each, run ShardedFilter with the library's kernels (route, shard
insert / lookup, answer reassembly) and exchange through a host-side
loopback that copies the all-to-all segments between the threads' tensors
(no kernel waits on another).  The shards together must equal the oracle's
filter of all hashes, and every shard's answers the oracle's lookups and the
unsharded filter's."""
import threading

import numpy as np
import pytest
import torch

import oracle
import paper_2101_01719_gb300 as sb
from paper_2101_01719_gb300 import sbbf
from paper_2101_01719_gb300.sharded import DeviceOps, ShardedFilter
import sbbf_inputs as inp
from gpu_util import bits_np, dev, to_dev

pytestmark = pytest.mark.gpu


class LoopbackHub:
    def __init__(self, world):
        self.world = world
        self.barrier = threading.Barrier(world, timeout=120)
        self.slots = [None] * world


class LoopbackComm:
    """all-to-all between the threads of one process, by device copies."""

    def __init__(self, hub, rank):
        self.hub, self.rank, self.world = hub, rank, hub.world

    def _publish(self, payload):
        self.hub.slots[self.rank] = payload
        self.hub.barrier.wait()  # every slot written
        view = list(self.hub.slots)
        self.hub.barrier.wait()  # every slot read before the next exchange writes
        return view

    def exchange_counts(self, send):
        view = self._publish(list(send))
        return [view[r][self.rank] for r in range(self.world)]

    def all_to_all(self, out, inp_, out_splits, in_splits):
        torch.cuda.synchronize()
        view = self._publish((inp_, list(in_splits)))
        off = 0
        for r in range(self.world):
            src, splits = view[r]
            start, cnt = sum(splits[: self.rank]), splits[self.rank]
            assert cnt == out_splits[r]
            out[off: off + cnt].copy_(src[start: start + cnt])
            off += cnt
        torch.cuda.synchronize()
        self.hub.barrier.wait()  # sources stay untouched until every copy is done


@pytest.mark.parametrize("world,num_blocks", [(1, 4096), (3, 100_003), (8, 2**20 + 7), (5, 4)])
def test_sharded_filter_kernels_equal_oracle(world, num_blocks):
    cfg = 90 + world
    device = dev()
    sizes = [300_000 * (r + 1) // world for r in range(world)]
    sizes[-1] = 0 if world > 2 else sizes[-1]  # an empty batch takes part too
    keys = [inp.stream(cfg, 0, n, start=r * 10**7) for r, n in enumerate(sizes)]
    all_keys = np.concatenate(keys)
    queries = [np.concatenate([inp.stream(cfg, 1, 50_001 + 33 * r, start=r * 10**6),
                               all_keys[r::world]]) for r in range(world)]
    hub = LoopbackHub(world)
    results, errors = [None] * world, []

    def rank_main(r):
        try:
            torch.cuda.set_device(device)
            sf = ShardedFilter(num_blocks, comm=LoopbackComm(hub, r), ops=DeviceOps(device))
            sf.insert(to_dev(keys[r]))
            bits = sf.find(to_dev(queries[r]))
            torch.cuda.synchronize()
            results[r] = (sf.lo, sf.hi, sf.local_words(), bits_np(bits))
        except BaseException as e:  # noqa: BLE001 - reported below
            errors.append("rank %d: %r" % (r, e))
            hub.barrier.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    ref = oracle.new_filter(num_blocks)
    oracle.insert(ref, num_blocks, all_keys)
    covered = 0
    for lo, hi, words, _ in results:
        got = np.zeros(8 * (hi - lo), np.uint32) if words is None else words
        assert np.array_equal(got, ref[8 * lo: 8 * hi]), (lo, hi)
        covered += hi - lo
    assert covered == num_blocks
    whole = sb.Filter(num_blocks)
    whole.insert(to_dev(all_keys))
    for r in range(world):
        exp = oracle.find(ref, num_blocks, queries[r])
        assert np.array_equal(results[r][3], exp), "answers of shard %d" % r
        assert np.array_equal(bits_np(whole.find(to_dev(queries[r]))), exp)


def test_route_groups_and_pads_by_owner():
    """sbbf_shard_route: every hash appears once in its owner's group with its
    index, groups come in owner order with the counts reported, and padding
    entries (lookups) are hashes of the owner's first block marked 0xFFFFFFFF."""
    B, G, n = 1_000_003, 6, 200_001
    h = inp.stream(97, 0, n)
    h[:1000] = h[:1000] >> np.uint64(8)  # crowd owner 0 a little
    for pad in (False, True):
        routed, perm, counts = sbbf.shard_route(to_dev(h), B, G, pad)
        counts = counts.cpu().numpy()
        routed = routed.cpu().numpy().view(np.uint64)
        perm = perm.cpu().numpy().view(np.uint32)
        per = -(-B // G)
        owner = np.array([oracle.block_index(int(x), B) for x in h], np.int64) // per
        start = 0
        seen = np.zeros(n, bool)
        for g in range(G):
            c = int(counts[g])
            seg_h, seg_p = routed[start: start + c], perm[start: start + c]
            real = seg_p != 0xFFFFFFFF
            assert int(real.sum()) == int((owner == g).sum())
            assert np.array_equal(h[seg_p[real]], seg_h[real])
            assert (owner[seg_p[real]] == g).all()
            seen[seg_p[real]] = True
            if pad:
                assert c % 32 == 0 and (~real).sum() < 32
                lo, _ = sbbf.shard_range(B, G, g)
                assert all(oracle.block_index(int(x), B) == lo for x in seg_h[~real])
            else:
                assert real.all()
            start += c
        assert seen.all()


def test_sharded_filter_over_nccl_with_one_rank():
    """The sharded filter through its default communicator -- NCCL
    all-to-alls over a one-process group -- and the library's kernels:
    words and answers equal the oracle's (the exchanges move every hash and
    answer word through NCCL even with one rank)."""
    import socket

    import torch.distributed as dist
    from paper_2101_01719_gb300.sharded import TorchComm

    if dist.is_initialized():
        pytest.skip("a process group is already initialised in this process")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    torch.cuda.set_device(dev())
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=0,
                            world_size=1)
    try:
        B = 1_000_003
        keys = inp.stream(99, 0, 700_001)
        q = np.concatenate([inp.stream(99, 1, 300_000), keys[::5]])
        sf = ShardedFilter(B, comm=TorchComm(device=dev()), ops=DeviceOps(dev()))
        assert (sf.lo, sf.hi) == (0, B)
        sf.insert(to_dev(keys[:350_000]))
        sf.insert(to_dev(keys[350_000:]))
        bits = bits_np(sf.find(to_dev(q)))
        ref = oracle.new_filter(B)
        oracle.insert(ref, B, keys)
        assert np.array_equal(sf.local_words(), ref)
        assert np.array_equal(bits, oracle.find(ref, B, q))
        assert bits_np(sf.find(to_dev(q[:0]))).size == 0  # an empty batch
    finally:
        dist.destroy_process_group()


def test_sharded_shards_take_region_passes():
    """Two 128 MiB shards of a 256 MiB filter and over 8Mi routed lookups per
    shard: each shard looks its hashes up in two region passes over its own
    block range.  Every answer equals the oracle's and the unsharded
    filter's."""
    world, B = 2, 2**23
    assert sb.Filter(B // world).region_passes(9_000_000) == 2  # a shard-sized filter
    keys = inp.stream(96, 0, 2_000_000)
    queries = [np.concatenate([inp.stream(96, 1 + r, 9_000_000), keys[r::world]])
               for r in range(world)]
    hub = LoopbackHub(world)
    results, errors = [None] * world, []

    def rank_main(r):
        try:
            torch.cuda.set_device(dev())
            sf = ShardedFilter(B, comm=LoopbackComm(hub, r), ops=DeviceOps(dev()))
            sf.insert(to_dev(keys[r::world]))
            bits = sf.find(to_dev(queries[r]))
            torch.cuda.synchronize()
            results[r] = bits_np(bits)
        except BaseException as e:  # noqa: BLE001 - reported below
            errors.append("rank %d: %r" % (r, e))
            hub.barrier.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    ref = oracle.new_filter(B)
    oracle.insert_mt(ref, B, keys, oracle.num_cores())
    whole = sb.Filter(B).set_partitioning(sb.PARTITION_OFF)
    whole.insert(to_dev(keys))
    for r in range(world):
        exp, _ = oracle.find_mt(ref, B, queries[r], oracle.num_cores())
        assert np.array_equal(results[r], exp), "answers of shard %d" % r
        assert np.array_equal(bits_np(whole.find(to_dev(queries[r]))), exp)
