"""GPU parity of the batched multi-filter path: tagged, segment and per-filter
forms, every launch shape the autotuner may pick, and the CUDA-graph batch
launch, all bit-exact against the CPU oracle (or against each other where the
oracle already fixed one of them)."""
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

SIZES = [1, 2, 5, 64, 100, 4096, 10_007, 65_536]


def _segments(n_keys, cfg, role=0):
    off = np.concatenate([[0], np.cumsum(n_keys)]).astype(np.int64)
    keys = inp.stream(cfg, role, int(off[-1]))
    return keys, off


def _oracle_arena(sizes, keys, ids):
    base = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.uint64)
    arena = np.zeros(8 * int(np.sum(sizes)), np.uint32)
    bad = oracle.multi_insert(arena, base, sizes, keys, ids)
    return arena, base, bad


def _ids_from_offsets(off):
    return np.repeat(np.arange(off.size - 1, dtype=np.uint32), np.diff(off))


def test_tagged_parity_with_invalid_ids():
    sizes = np.array(SIZES, np.uint32)
    n = 300_001
    keys = inp.stream(40, 0, n)
    ids = (inp.stream(40, 4, n) % np.uint64(len(SIZES) + 1)).astype(np.uint32)
    ids[ids == len(SIZES)] = 0xFFFFFFFF
    ids[::1000] = len(SIZES)  # another invalid id
    m = sb.MultiFilter(sizes)
    m.insert(to_dev(keys), ids=torch.from_numpy(ids.view(np.int32)).to(dev()))
    arena, base, bad = _oracle_arena(sizes, keys, ids)
    assert m.invalid_count() == bad and bad > 0
    assert m.invalid_count() == 0  # reading resets
    assert np.array_equal(m.to_numpy(), arena)
    q = np.concatenate([inp.stream(40, 1, 200_003), keys[:50_000]])
    qid = (inp.stream(40, 5, q.size) % np.uint64(len(SIZES) + 1)).astype(np.uint32)
    qid[qid == len(SIZES)] = 0x80000000
    bits = m.find(to_dev(q), ids=torch.from_numpy(qid.view(np.int32)).to(dev()))
    ref_bits, badq = oracle.multi_find(arena, base, sizes, q, qid)
    assert np.array_equal(bits_np(bits), ref_bits)
    assert m.invalid_count() == badq


def test_segments_tagged_and_per_filter_agree():
    w = wl.C3_SMALL
    n_keys, blocks = w.sizes()
    ins, ins_off, q, q_off = wl.gen_multi(w, device=dev())
    h_ins_off, h_q_off = w.offsets()
    # inputs regenerate on the host by the same recipe
    assert np.array_equal(u64_np(ins), inp.stream(w.cfg, 0, int(h_ins_off[-1])))
    for t in (0, 7, w.n_filters - 1):
        assert np.array_equal(u64_np(q[h_q_off[t]:h_q_off[t + 1]]),
                              inp.segment_queries(w.cfg, h_ins_off, h_q_off, w.member_frac, t))
    m_seg, m_tag, m_each = (sb.MultiFilter(blocks) for _ in range(3))
    m_seg.insert(ins, offsets=ins_off)
    ids = sb.fill_segment_ids(torch.empty(ins.numel(), dtype=torch.int32, device=dev()), ins_off)
    m_tag.insert(ins, ids=ids)
    m_each.insert_each(ins, h_ins_off)
    a_seg = m_seg.to_numpy()
    assert np.array_equal(a_seg, m_tag.to_numpy())
    assert np.array_equal(a_seg, m_each.to_numpy())
    # the oracle, filter by filter
    keys = u64_np(ins)
    for t in range(w.n_filters):
        f = oracle.new_filter(int(blocks[t]))
        oracle.insert(f, int(blocks[t]), keys[h_ins_off[t]:h_ins_off[t + 1]])
        assert np.array_equal(m_seg.filter_words(a_seg, t), f), t
    b_seg = bits_np(m_seg.find(q, offsets=q_off))
    qids = sb.fill_segment_ids(torch.empty(q.numel(), dtype=torch.int32, device=dev()), q_off)
    b_tag = bits_np(m_seg.find(q, ids=qids))
    b_each = bits_np(m_seg.find_each(q, h_q_off))
    assert np.array_equal(b_seg, b_tag) and np.array_equal(b_seg, b_each)
    qh = u64_np(q)
    for t in range(0, w.n_filters, 5):
        f = m_seg.filter_words(a_seg, t)
        ref = oracle.find(np.ascontiguousarray(f), int(blocks[t]), qh[h_q_off[t]:h_q_off[t + 1]])
        got = b_seg[h_q_off[t] // 32: h_q_off[t + 1] // 32]
        assert np.array_equal(got, ref), t
    # members always hit
    hit = np.unpackbits(b_seg.view(np.uint8), bitorder="little").astype(bool)
    t_sample = 3
    member = inp.segment_queries(w.cfg, h_ins_off, h_q_off, w.member_frac, t_sample)
    inserted = set(keys[h_ins_off[t_sample]:h_ins_off[t_sample + 1]].tolist())
    is_mem = np.array([int(x) in inserted for x in member])
    assert hit[h_q_off[t_sample]:h_q_off[t_sample + 1]][is_mem].all()


def test_shuffled_tagged_insert_equals_grouped():
    w = wl.C3_SMALL
    _, blocks = w.sizes()
    ins, ins_off, _, _ = wl.gen_multi(w, device=dev())
    ids = sb.fill_segment_ids(torch.empty(ins.numel(), dtype=torch.int32, device=dev()), ins_off)
    g = torch.Generator(device=dev())
    g.manual_seed(1234)
    perm = torch.randperm(ins.numel(), device=dev(), generator=g)
    m1, m2 = sb.MultiFilter(blocks), sb.MultiFilter(blocks)
    m1.insert(ins, offsets=ins_off)
    m2.insert(ins[perm].contiguous(), ids=ids[perm].contiguous())
    assert np.array_equal(m1.to_numpy(), m2.to_numpy())


@pytest.mark.parametrize("form", [sb.FORM_SEGMENTS, sb.FORM_TAGGED])
def test_every_launch_shape_is_bit_exact(form):
    """All shapes the autotuner may choose give identical words and answers."""
    w = wl.C3_SMALL
    _, blocks = w.sizes()
    ins, ins_off, q, q_off = wl.gen_multi(w, device=dev())
    kw_i = {"offsets": ins_off}
    kw_q = {"offsets": q_off}
    if form == sb.FORM_TAGGED:
        kw_i = {"ids": sb.fill_segment_ids(torch.empty(ins.numel(), dtype=torch.int32,
                                                       device=dev()), ins_off)}
        kw_q = {"ids": sb.fill_segment_ids(torch.empty(q.numel(), dtype=torch.int32,
                                                       device=dev()), q_off)}
    m = sb.MultiFilter(blocks)
    m.insert(ins, **kw_i)
    ref_words = m.to_numpy()
    ref_bits = bits_np(m.find(q, **kw_q))
    for threads in (128, 256, 512):
        for lanes in (1, 8):
            m2 = sb.MultiFilter(blocks)
            m2.set_tuning(sb.OP_INSERT, form, threads, lanes, 1)
            m2.insert(ins, **kw_i)
            assert np.array_equal(m2.to_numpy(), ref_words), (threads, lanes)
            for unroll in (1, 2, 4):
                for l1 in (0, 1):
                    m.set_tuning(sb.OP_FIND, form, threads, lanes, unroll, l1)
                    got = bits_np(m.find(q, **kw_q))
                    assert np.array_equal(got, ref_bits), (threads, lanes, unroll, l1)
    with pytest.raises(sb.SbbfError):
        m.set_tuning(sb.OP_FIND, form, 96, 1, 1)


def test_autotuner_picks_a_verified_shape_and_leaves_filters_alone():
    w = wl.C3_SMALL
    _, blocks = w.sizes()
    ins, ins_off, q, q_off = wl.gen_multi(w, device=dev())
    m = sb.MultiFilter(blocks)
    m.insert(ins[: ins.numel() // 2].contiguous(),
             offsets=torch.clamp(ins_off, max=ins.numel() // 2))
    before = m.to_numpy()
    ms_i = m.tune(sb.OP_INSERT, ins, offsets=ins_off)
    ms_f = m.tune(sb.OP_FIND, q, offsets=q_off)
    assert np.array_equal(m.to_numpy(), before)  # tuning inserts into scratch only
    for op, ms in ((sb.OP_INSERT, ms_i), (sb.OP_FIND, ms_f)):
        t = m.get_tuning(op, sb.FORM_SEGMENTS)
        assert t["threads"] in (128, 256, 512) and t["lanes"] in (1, 8)
        assert t["l1_bypass"] in (0, 1)
        assert ms > 0 or ms == -1.0
    # a second tune of the same size class is answered from the cache
    assert m.tune(sb.OP_FIND, q, offsets=q_off) == -1.0
    m.insert(ins, offsets=ins_off)
    ref = sb.MultiFilter(blocks)
    ref.insert(ins, offsets=ins_off)
    assert np.array_equal(m.to_numpy(), ref.to_numpy())
    assert np.array_equal(bits_np(m.find(q, offsets=q_off)), bits_np(ref.find(q, offsets=q_off)))


def test_graph_launch_equals_separate_launches():
    w = wl.C3_SMALL
    _, blocks = w.sizes()
    ins, ins_off, q, q_off = wl.gen_multi(w, device=dev())
    m = sb.MultiFilter(blocks)
    out = torch.empty(sb.out_words(q.numel()), dtype=torch.int32, device=dev())
    m.graph_launch(ins, ins_off, q, q_off, out)
    ref = sb.MultiFilter(blocks)
    ref.insert(ins, offsets=ins_off)
    ref_bits = ref.find(q, offsets=q_off)
    assert np.array_equal(m.to_numpy(), ref.to_numpy())
    assert np.array_equal(bits_np(out), bits_np(ref_bits))
    # relaunch with other buffers (arguments updated in place), and with an
    # empty insert part
    half = q.numel() // 2 // 64 * 64
    q_off2 = torch.clamp(q_off, max=half)
    out2 = torch.zeros(sb.out_words(half), dtype=torch.int32, device=dev())
    m.graph_launch(None, None, q[:half].contiguous(), q_off2, out2)
    assert np.array_equal(bits_np(out2), bits_np(ref_bits)[: half // 32])
    m.clear()
    m.graph_launch(ins, ins_off, q, q_off, out)
    assert np.array_equal(bits_np(out), bits_np(ref_bits))


def test_config_c3_full_size_every_filter():
    """4096 filters (1k..4M keys), one graph launch of all inserts then all
    4x lookups; batched == per-filter launches on every word and answer; and
    every filter's words and every one of the 8.17e9 answers equal the
    oracle's, filter by filter, with the oracle's queries generated on the
    host and equal to the device-generated ones."""
    w = wl.C3
    n_keys, blocks = w.sizes()
    h_ins_off, h_q_off = w.offsets()
    ins, ins_off, q, q_off = wl.gen_multi(w, device=dev())
    m = sb.MultiFilter(blocks)
    m.tune(sb.OP_INSERT, ins, offsets=ins_off)
    m.tune(sb.OP_FIND, q, offsets=q_off)
    out = torch.empty(sb.out_words(q.numel()), dtype=torch.int32, device=dev())
    m.graph_launch(ins, ins_off, q, q_off, out)
    arena = m.to_numpy()
    each = sb.MultiFilter(blocks)
    each.insert_each(ins, h_ins_off)
    assert np.array_equal(each.to_numpy(), arena)
    out_each = each.find_each(q, h_q_off)
    assert torch.equal(out_each, out)
    del each, out_each, ins
    torch.cuda.empty_cache()
    bits = bits_np(out)
    del out

    def check(t, qs):
        keys = inp.fast_stream(w.cfg, 0, int(n_keys[t]), int(h_ins_off[t]), threads=1)
        f = oracle.new_filter(int(blocks[t]))
        oracle.insert(f, int(blocks[t]), keys)
        if not np.array_equal(m.filter_words(arena, t), f):
            return "words of filter %d" % t
        if not np.array_equal(bits[h_q_off[t] // 32: h_q_off[t + 1] // 32],
                              oracle.find(f, int(blocks[t]), qs)):
            return "lookups of filter %d" % t
        return None

    # groups of filters with about 2^26 lookups each; per group the host
    # generates the queries, checks them against the device's, and the
    # oracle checks each filter on its own thread
    errors, pending = [], []
    t0 = 0
    threads = oracle.num_cores()
    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        while t0 < w.n_filters:
            t1 = int(np.searchsorted(h_q_off, h_q_off[t0] + (1 << 26), side="right")) - 1
            t1 = min(max(t1, t0 + 1), w.n_filters)
            qh = inp.fast_segment_queries(w.cfg, h_ins_off, h_q_off, w.member_frac, t0, t1)
            a, b = int(h_q_off[t0]), int(h_q_off[t1])
            assert np.array_equal(u64_np(q[a:b]), qh), "queries of filters %d..%d" % (t0, t1)
            pending.append([ex.submit(check, t, qh[int(h_q_off[t]) - a: int(h_q_off[t + 1]) - a])
                            for t in range(t0, t1)])
            while len(pending) > 4:  # bounds the host memory held by queued groups
                errors += [e for e in (fu.result() for fu in pending.pop(0)) if e]
            t0 = t1
        for group in pending:
            errors += [e for e in (fu.result() for fu in group) if e]
    assert not errors, errors[:10]
    del q
    torch.cuda.empty_cache()
