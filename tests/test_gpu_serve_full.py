"""The serving workload at full size: 256 resident filters (128 KiB to 1 GiB,
pre-filled to 10.5 bits/key, ~35 GB) and 10M requests (70% lookups, 1 to 1M
hashes each, ~7.2e11 keys) submitted at once, so that the server batches as
much as it can.  The answers of every lookup on 8 sampled filters are kept
(the rest go to a scratch ring), and the oracle replays those filters'
requests serially in arrival order: every kept answer and the sampled
filters' final words must equal the replay's."""
import concurrent.futures

import numpy as np
import pytest
import torch

import oracle
import paper_2101_01719_gb300 as sb
from paper_2101_01719_gb300 import workloads as wl
import sbbf_inputs as inp
from gpu_util import dev

pytestmark = pytest.mark.gpu

W = wl.C4
N_SAMPLED = 8
RING_WORDS = 1 << 24  # answers of the unchecked lookups (wrapping)


def _words(size):
    """Result words of a lookup of `size` hashes, rounded to 32 bytes."""
    return ((size + np.uint64(31)) // np.uint64(32) + np.uint64(7)) // np.uint64(8) * np.uint64(8)


def test_config_c4_full_run_sampled_filters_replayed():
    blocks, counts = W.filter_blocks(), W.prefill_counts()
    pre_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    srv = sb.Server(W.budget_bytes, max_window_requests=4096, max_inflight_windows=2,
                    max_window_keys=1 << 26, max_pending_requests=1 << 25, device=dev())
    wl.prefill_server(W, srv, device=dev())
    pool = torch.empty(W.pool_hashes, dtype=torch.int64, device=dev())
    sb.fill_splitmix64(pool, wl.seed(W.cfg, wl.ROLE_FRESH), 0)

    n = W.n_requests
    op, filt, size, off, arr = W.requests(n, float("inf"))
    sampled = np.sort(np.random.default_rng(W.cfg).choice(W.n_filters, N_SAMPLED, replace=False))
    look = op == sb.OP_FIND
    kept = look & np.isin(filt, sampled)
    words = np.where(look, _words(size), 0).astype(np.uint64)
    start = np.zeros(n, np.uint64)
    start[kept] = np.concatenate([[0], np.cumsum(words[kept])[:-1]]).astype(np.uint64)
    ring = np.concatenate([[0], np.cumsum(words[look & ~kept])[:-1]]).astype(np.uint64)
    ring %= np.uint64(RING_WORDS)
    ring[ring + words[look & ~kept] > np.uint64(RING_WORDS)] = 0
    out_kept = torch.full((int(words[kept].sum()) + 8,), -1, dtype=torch.int32, device=dev())
    out_ring = torch.empty(RING_WORDS, dtype=torch.int32, device=dev())
    rec = np.zeros(n, dtype=sb.REQUEST_DTYPE)
    rec["op"], rec["filter"], rec["n"] = op, filt, size
    rec["hashes"] = np.uint64(pool.data_ptr()) + off * np.uint64(8)
    out_addr = np.zeros(n, np.uint64)
    out_addr[kept] = np.uint64(out_kept.data_ptr()) + start[kept] * np.uint64(4)
    out_addr[look & ~kept] = np.uint64(out_ring.data_ptr()) + ring * np.uint64(4)
    rec["out"] = out_addr

    lat = srv.replay(rec, arr)
    torch.cuda.synchronize()
    assert (lat > 0).all()
    st = srv.stats()
    assert st["requests"] == n and st["windows"] < n // 10  # requests were batched
    got = out_kept.cpu().numpy().view(np.uint32)
    final = {int(t): srv.filter_words(int(t)) for t in sampled}
    srv.close()
    del pool, out_kept, out_ring
    torch.cuda.empty_cache()

    pool_h = inp.fast_stream(W.cfg, inp.ROLE_FRESH, W.pool_hashes)
    per = max(1, oracle.num_cores() // N_SAMPLED)

    def replay(t):
        """Serial replay of filter t's requests in arrival order."""
        b = int(blocks[t])
        f = oracle.new_filter(b)
        oracle.insert_mt(f, b, inp.fast_stream(W.cfg, inp.ROLE_INSERT, int(counts[t]),
                                               int(pre_off[t]), threads=per), per)
        for i in np.nonzero(filt == t)[0]:
            keys = pool_h[int(off[i]): int(off[i]) + int(size[i])]
            big = keys.size >= (1 << 16)
            if op[i] == sb.OP_INSERT:
                if big:
                    oracle.insert_mt(f, b, keys, per)
                else:
                    oracle.insert(f, b, keys)
            else:
                exp = oracle.find_mt(f, b, keys, per)[0] if big else oracle.find(f, b, keys)
                a = int(start[i])
                if not np.array_equal(got[a: a + exp.size], exp):
                    return "request %d (filter %d)" % (i, t)
        if not np.array_equal(final[t], f):
            return "final words of filter %d" % t
        return None

    with concurrent.futures.ThreadPoolExecutor(N_SAMPLED) as ex:
        errors = [e for e in ex.map(replay, [int(t) for t in sampled]) if e]
    assert not errors, errors
