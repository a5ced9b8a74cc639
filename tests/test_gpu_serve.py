"""GPU tests of the serving form: continuous batching over resident filters
must give every request exactly the result of serial replay in arrival order
(computed by the CPU oracle), with and without evictions, for Poisson and
all-at-once arrivals, with device and pinned-host payloads; a request's
answer alone equals its answer in the mix."""
import numpy as np
import pytest
import torch

import oracle
import paper_2101_01719_gb300 as sb
from paper_2101_01719_gb300 import workloads as wl
import sbbf_inputs as inp
from gpu_util import dev

pytestmark = pytest.mark.gpu

W = wl.C4_SMALL


class Setup:
    """A server with W's filters, pre-filled, plus the request table."""

    def __init__(self, budget, n_req, rate, pinned=False, **cfg):
        self.srv = sb.Server(budget, **cfg)
        self.blocks = W.filter_blocks()
        self.counts = W.prefill_counts()
        self.pre_off = np.concatenate([[0], np.cumsum(self.counts)]).astype(np.int64)
        for t, b in enumerate(self.blocks):
            assert self.srv.add_filter(int(b)) == t
            keys = wl.gen_inserts_seeded(wl.seed(W.cfg, 0), int(self.pre_off[t]),
                                         int(self.counts[t]), device=dev())
            self.srv.prefill(t, keys)
        pool = torch.empty(W.pool_hashes, dtype=torch.int64, device=dev())
        sb.fill_splitmix64(pool, wl.seed(W.cfg, 1), 0)
        self.op, self.filt, self.size, self.off, self.arr = W.requests(n_req, rate)
        words = int(sum(((int(s) + 31) // 32 + 7) // 8 * 8 for s, o in zip(self.size, self.op)
                        if o == sb.OP_FIND)) + 8
        if pinned:
            self.pool = pool.cpu().pin_memory()
            self.out = torch.full((words,), -1, dtype=torch.int32).pin_memory()
        else:
            self.pool = pool
            self.out = torch.full((words,), -1, dtype=torch.int32, device=dev())
        self.rec, self.start, self.words = wl.request_records(
            self.op, self.filt, self.size, self.off, self.pool, self.out)

    def results(self):
        torch.cuda.synchronize()
        return self.out.cpu().numpy().view(np.uint32)

    def close(self):
        self.srv.close()


def _oracle_replay(s: Setup, upto=None):
    """Serial replay in arrival order on the CPU: final filters and the
    expected answer words of every lookup."""
    n = len(s.op) if upto is None else upto
    filt = []
    for t, b in enumerate(s.blocks):
        f = oracle.new_filter(int(b))
        oracle.insert(f, int(b), inp.stream(W.cfg, 0, int(s.counts[t]), int(s.pre_off[t])))
        filt.append(f)
    pool = inp.stream(W.cfg, 1, W.pool_hashes)
    expect = {}
    for i in range(n):
        t, b = int(s.filt[i]), int(s.blocks[int(s.filt[i])])
        keys = pool[int(s.off[i]): int(s.off[i]) + int(s.size[i])]
        if s.op[i] == sb.OP_INSERT:
            oracle.insert(filt[t], b, keys)
        else:
            expect[i] = oracle.find(filt[t], b, keys)
    return filt, expect


def _check(s: Setup, filt, expect, got):
    for i, exp in expect.items():
        a = int(s.start[i])
        assert np.array_equal(got[a: a + exp.size], exp), "request %d" % i
    for t in range(len(s.blocks)):
        assert np.array_equal(s.srv.filter_words(t), filt[t]), "filter %d" % t


@pytest.fixture(scope="module")
def reference():
    s = Setup(W.budget_bytes, 20_000, 2e5)
    filt, expect = _oracle_replay(s)
    s.close()
    return filt, expect


def test_batched_serving_equals_serial_replay(reference):
    s = Setup(W.budget_bytes, 20_000, 2e5, max_window_requests=512)
    lat = s.srv.replay(s.rec, s.arr)
    assert (lat > 0).all()
    _check(s, *reference, s.results())
    st = s.srv.stats()
    assert st["requests"] == 20_000 and st["windows"] < 20_000  # requests were batched
    assert st["phases"] >= st["windows"]
    s.close()


def test_serving_under_half_budget_evicts_and_stays_exact(reference):
    total = int(W.filter_blocks().sum()) * 32
    s = Setup(total // 2, 20_000, 2e5, max_window_requests=512)
    s.srv.replay(s.rec, s.arr)
    _check(s, *reference, s.results())
    st = s.srv.stats()
    assert st["evictions"] > 0 and st["admission_waits"] >= 0
    assert st["resident_bytes"] <= total // 2
    s.close()


def test_all_arrivals_at_once(reference):
    s = Setup(W.budget_bytes, 20_000, float("inf"), max_window_requests=4096)
    s.srv.replay(s.rec, s.arr)
    _check(s, *reference, s.results())
    s.close()


def test_serial_per_request_launches_equal_oracle(reference):
    s = Setup(W.budget_bytes, 20_000, 2e5)
    lat = s.srv.replay(s.rec, s.arr, serial=True)
    assert (lat > 0).all()
    _check(s, *reference, s.results())
    assert s.srv.stats()["windows"] == 0
    s.close()


def test_alone_equals_in_the_mix():
    n = 3000
    mix = Setup(W.budget_bytes, n, 3e5)
    mix.srv.replay(mix.rec, mix.arr)
    got_mix = mix.results()
    alone = Setup(W.budget_bytes, n, 3e5)
    for i in range(n):  # one request in the system at a time
        r = alone.rec[i]
        t = alone.srv.submit(int(r["op"]), int(r["filter"]),
                             _View(int(r["hashes"]), int(r["n"])),
                             _View(int(r["out"]), 0) if r["op"] == sb.OP_FIND else None)
        alone.srv.wait(t)
    got_alone = alone.results()
    for i in range(n):
        if mix.op[i] == sb.OP_FIND:
            a, w = int(mix.start[i]), (int(mix.size[i]) + 31) // 32
            assert np.array_equal(got_mix[a: a + w], got_alone[a: a + w]), i
    for t in range(len(mix.blocks)):
        assert np.array_equal(mix.srv.filter_words(t), alone.srv.filter_words(t))
    mix.close()
    alone.close()


def test_pinned_host_payloads():
    n = 4000
    s = Setup(W.budget_bytes, n, 2e5, pinned=True)
    s.srv.replay(s.rec, s.arr)
    filt, expect = _oracle_replay(s, n)
    _check(s, filt, expect, s.results())
    s.close()


def test_server_errors_are_statuses():
    srv = sb.Server(1 << 20, max_window_requests=16)
    small = srv.add_filter(100)
    huge = srv.add_filter(1 << 20)  # 32 MiB: larger than the whole budget
    h = torch.zeros(1 << 20, dtype=torch.int64, device=dev())
    out = torch.zeros(1 << 15, dtype=torch.int32, device=dev())
    with pytest.raises(sb.SbbfError) as e:
        srv.submit(sb.OP_FIND, huge, h[:10], out)
    assert e.value.status == sb.sbbf.SBBF_EBUSY
    with pytest.raises(sb.SbbfError) as e:
        srv.submit(sb.OP_FIND, 7, h[:10], out)
    assert e.value.status == sb.sbbf.SBBF_EINVAL
    with pytest.raises(sb.SbbfError) as e:
        srv.submit(5, small, h[:10], out)
    assert e.value.status == sb.sbbf.SBBF_EINVAL
    big = sb.Server(1 << 30)
    f = big.add_filter(1 << 20)
    t = big.submit(sb.OP_FIND, f, h, out)
    rc = big.wait_status(t, timeout_ns=1)
    assert rc in (sb.sbbf.SBBF_ETIMEOUT, sb.sbbf.SBBF_OK)
    big.wait(t)
    assert big.poll(t)
    t0 = srv.submit(sb.OP_INSERT, small, h[:0])  # empty request: done at once
    assert srv.poll(t0)
    srv.close()
    big.close()


class _View:
    """Minimal tensor-like view of raw memory for Server.submit."""

    def __init__(self, ptr, n):
        self._p, self._n = ptr, n

    def data_ptr(self):
        return self._p

    def numel(self):
        return self._n


def test_submits_take_amortised_constant_time():
    """400,000 requests through one server (empty ones, done at submission,
    no GPU work) replay in well under a second: the per-ticket tables grow
    geometrically.  Growing them by one element per request copies the whole
    table every time, which took minutes here and, in the full serving
    workload, made throughput fall with every request served."""
    import time
    srv = sb.Server(1 << 20)
    f = srv.add_filter(64)
    n = 400_000
    rec = np.zeros(n, dtype=sb.REQUEST_DTYPE)
    rec["op"], rec["filter"], rec["n"] = sb.OP_INSERT, f, 0
    t0 = time.perf_counter()
    lat = srv.replay(rec, np.zeros(n, np.uint64))
    elapsed = time.perf_counter() - t0
    srv.close()
    assert lat.size == n
    assert elapsed < 5.0, elapsed
