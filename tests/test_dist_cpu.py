"""Multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1).

bench.py runs one process per GPU; ranks shard the lookup stream and time
independently, and rank 0 reports the whole job's units over the slowest
rank's time.  This exercises that logic without GPUs."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    bench.barrier(dist)
    seconds = [1.5, 2.5][rank]
    slowest = bench.max_over_ranks(dist, seconds)
    start = bench.lookup_slice_start(r, 1000)
    q.put((r, slowest, start, bench.aggregate([1000] * w, slowest)))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [2.5, 2.5]          # both see the slowest rank
    assert [r[2] for r in res] == [0, 1000]           # disjoint lookup slices
    assert res[0][3] == pytest.approx(2000 / 2.5)     # all units / slowest time
