"""The sharded filter's exchange logic on CPU ranks (gloo, world size 2 and
4): every rank inserts its own batch and looks up its own queries through
ShardedFilter (all-to-all of hashes, local work, reverse all-to-all of
answer words, reassembly); the shards put together must equal the oracle's
filter of all ranks' hashes, and every rank's answers the oracle's lookups.
The device steps are the host stand-ins of sharded_host_ops (no GPU here);
the same exchange code drives the library's kernels on GPUs."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, num_blocks, n_per_rank, errq):
    sys.path[:0] = [ROOT, HERE]
    try:
        import torch
        import torch.distributed as dist

        import oracle
        import sbbf_inputs as inp
        from paper_2101_01719_gb300.sharded import ShardedFilter, TorchComm
        from sharded_host_ops import HostOps

        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        cfg = 70 + world
        sf = ShardedFilter(num_blocks, comm=TorchComm(), ops=HostOps())
        # uneven batches, one rank possibly empty
        n = n_per_rank * (rank + 1) // world if rank != world - 1 or world == 2 else 0
        keys = inp.stream(cfg, 0, n, start=rank * 10**7)
        sf.insert(torch.from_numpy(keys.view(np.int64).copy()))
        all_keys = np.concatenate([
            inp.stream(cfg, 0, (n_per_rank * (r + 1) // world
                                if r != world - 1 or world == 2 else 0), start=r * 10**7)
            for r in range(world)])
        q = np.concatenate([inp.stream(cfg, 1, 3001 + 17 * rank, start=rank * 10**6),
                            all_keys[rank::world]])
        if world == 4 and rank == 1:
            q = q[:0]  # a rank with no queries still takes part in the exchanges
        bits = sf.find(torch.from_numpy(q.view(np.int64).copy())).numpy().view(np.uint32)

        ref = oracle.new_filter(num_blocks)
        oracle.insert(ref, num_blocks, all_keys)
        local = sf.local_words()
        shards = [None] * world
        dist.all_gather_object(shards, (sf.lo, sf.hi, None if local is None else local.tolist()))
        for lo, hi, words in shards:
            got = np.zeros(8 * (hi - lo), np.uint32) if words is None else np.array(words, np.uint32)
            assert np.array_equal(got, ref[8 * lo: 8 * hi]), "shard [%d, %d)" % (lo, hi)
        covered = sum(hi - lo for lo, hi, _ in shards)
        assert covered == num_blocks
        exp = oracle.find(ref, num_blocks, q)
        assert np.array_equal(bits, exp), "answers of rank %d" % rank
        dist.barrier()
        dist.destroy_process_group()
    except BaseException as e:  # report to the parent; never hang the others
        import traceback
        errq.put("rank %d: %s\n%s" % (rank, e, traceback.format_exc()))
        raise


@pytest.mark.parametrize("world,num_blocks", [(2, 5003), (4, 4096), (4, 3)])
def test_sharded_filter_on_gloo_ranks_equals_oracle(world, num_blocks):
    ctx = mp.get_context("spawn")
    errq = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, num_blocks, 40_000, errq))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    errors = []
    while not errq.empty():
        errors.append(errq.get())
    assert not alive, "ranks did not finish"
    assert not errors, "\n".join(errors)
    assert all(p.exitcode == 0 for p in procs)


def test_shard_ranges_cover_the_filter_without_overlap():
    from paper_2101_01719_gb300 import sbbf
    for nb in (1, 3, 4096, 5003, 2**30, 2**32 - 1):
        for g in (1, 2, 3, 4, 7, 8, 1024):
            ranges = [sbbf.shard_range(nb, g, s) for s in range(g)]
            assert ranges[0][0] == 0 and ranges[-1][1] == nb
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and a <= b
            per = -(-nb // g)
            assert all(b - a <= per for a, b in ranges)
    with pytest.raises(sbbf.SbbfError):
        sbbf.shard_range(10, 0, 0)
    with pytest.raises(sbbf.SbbfError):
        sbbf.shard_range(10, 2, 2)
