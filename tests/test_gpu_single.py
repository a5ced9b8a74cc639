"""GPU parity: the CUDA single-filter path against the CPU oracle, bit for bit.

Inputs are seeded splitmix64 streams (tests/sbbf_inputs.py or the library's
device generator, itself checked against the host copy here).  Filter words
and packed lookup results must be identical to the oracle's: the method is
integer-only, so the tolerance is zero.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2101_01719_gb300 as sb
from paper_2101_01719_gb300 import sbbf as abi
from paper_2101_01719_gb300 import workloads as wl
import sbbf_inputs as inp
from gpu_util import (bit_at, bits_np, compare_all_lookups, compare_words, dev,
                      oracle_filter_of_stream, to_dev, u64_np)

pytestmark = pytest.mark.gpu


def _oracle_filter(B, keys):
    f = oracle.new_filter(B)
    oracle.insert(f, B, keys)
    return f


SIZES = [(1, 0), (1, 1), (3, 63), (7, 64), (4096, 65), (4096, 100_003), (32768, 1_000_001),
         (1_000_003, 777_777), (2**22 + 5, 2_000_000)]


@pytest.mark.parametrize("B,n", SIZES)
def test_insert_and_find_parity(B, n):
    keys = inp.stream(100 + B % 97, 0, n)
    q = np.concatenate([inp.stream(100 + B % 97, 1, 3 * n + 17), keys[: n // 2]])
    f = sb.Filter(B)
    f.insert(to_dev(keys))
    bits = f.find(to_dev(q))
    ref = _oracle_filter(B, keys)
    assert np.array_equal(f.to_numpy(), ref)
    ref_bits = oracle.find(ref, B, q)
    got = bits_np(bits)
    assert got.size == ref_bits.size
    assert np.array_equal(got, ref_bits)


@pytest.mark.parametrize("offset", [1, 3])
def test_unaligned_hash_pointers(offset):
    """8-byte but not 16-byte aligned hash arrays take the scalar-load path."""
    B, n = 5000, 100_001
    keys = inp.stream(120, 0, n + offset)
    q = inp.stream(120, 1, 50_001 + offset)
    dk, dq = to_dev(keys), to_dev(q)
    f = sb.Filter(B)
    f.insert(dk[offset:])
    bits = f.find(dq[offset:])
    ref = _oracle_filter(B, keys[offset:])
    assert np.array_equal(f.to_numpy(), ref)
    assert np.array_equal(bits_np(bits), oracle.find(ref, B, q[offset:]))


def test_ragged_tails_every_residue():
    B = 257
    keys = inp.stream(121, 0, 5000)
    ref = _oracle_filter(B, keys)
    f = sb.Filter(B)
    f.insert(to_dev(keys))
    assert np.array_equal(f.to_numpy(), ref)
    q_all = inp.stream(121, 1, 300)
    for n in list(range(0, 130)) + [191, 192, 193, 255, 256, 257]:
        q = np.concatenate([q_all[: n // 2], keys[: n - n // 2]])
        out = torch.full((sb.out_words(n) + 2,), -1, dtype=torch.int32, device=dev())
        f.find(to_dev(q), out=out)
        got = bits_np(out)
        assert np.array_equal(got[: sb.out_words(n)], oracle.find(ref, B, q))
        assert (got[sb.out_words(n):] == 0xFFFFFFFF).all()  # nothing written past the end


def test_order_and_duplicates_do_not_matter():
    B = 3001
    keys = inp.stream(122, 0, 400_000)
    perm = inp.permutation(122, keys.size)
    dup = np.concatenate([keys[perm], keys[:100_000], keys[::7]])
    f1, f2 = sb.Filter(B), sb.Filter(B)
    f1.insert(to_dev(keys))
    f2.insert(to_dev(dup))
    assert np.array_equal(f1.to_numpy(), f2.to_numpy())
    assert np.array_equal(f1.to_numpy(), _oracle_filter(B, keys))


def test_concurrent_streams_insert():
    B = 2048
    keys = inp.stream(123, 0, 2_000_000)
    dk = to_dev(keys)
    f = sb.Filter(B)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    f.insert(dk[:1_000_000], stream=s1)
    f.insert(dk[1_000_000:], stream=s2)
    torch.cuda.synchronize()
    assert np.array_equal(f.to_numpy(), _oracle_filter(B, keys))


def test_union_and_clear():
    B = 12345
    a, b = inp.stream(124, 0, 200_000), inp.stream(124, 1, 150_000)
    fa, fb = sb.Filter(B), sb.Filter(B)
    fa.insert(to_dev(a))
    fb.insert(to_dev(b))
    fa.union_(fb)
    ref = oracle.union(_oracle_filter(B, a), _oracle_filter(B, b))
    assert np.array_equal(fa.to_numpy(), ref)
    fa.union_(fa)  # self-union is a no-op
    assert np.array_equal(fa.to_numpy(), ref)
    with pytest.raises(sb.SbbfError):
        fa.union_(sb.Filter(B + 1))
    fa.clear()
    assert not fa.to_numpy().any()


def test_library_owned_filter_roundtrip():
    """sbbf_create / sbbf_create_from_host / sbbf_copy_to_host through the C ABI."""
    L = abi.lib()
    B = 777
    keys = inp.stream(125, 0, 30_000)
    ref = _oracle_filter(B, keys)
    h = ctypes.c_void_p()
    assert L.sbbf_create(B, ctypes.byref(h)) == 0
    try:
        dk = to_dev(keys)
        s = torch.cuda.current_stream().cuda_stream
        assert L.sbbf_insert_hashes(h, dk.data_ptr(), keys.size, s) == 0
        host = np.zeros(8 * B, np.uint32)
        assert L.sbbf_copy_to_host(h, host.ctypes.data, host.nbytes, s) == 0
        assert np.array_equal(host, ref)
        small = np.zeros(8 * B - 1, np.uint32)
        assert L.sbbf_copy_to_host(h, small.ctypes.data, small.nbytes, s) == abi.SBBF_EINVAL
        assert L.sbbf_num_blocks(h) == B
        ptr, nbytes = ctypes.c_void_p(), ctypes.c_size_t()
        assert L.sbbf_device_words(h, ctypes.byref(ptr), ctypes.byref(nbytes)) == 0
        assert nbytes.value == 32 * B and ptr.value % 256 == 0
    finally:
        assert L.sbbf_destroy(h) == 0
    g = ctypes.c_void_p()
    assert L.sbbf_create_from_host(ref.ctypes.data, B, ctypes.byref(g)) == 0
    try:
        q = np.concatenate([keys[:1000], inp.stream(125, 1, 5000)])
        dq = to_dev(q)
        out = torch.empty(sb.out_words(q.size), dtype=torch.int32, device=dev())
        s = torch.cuda.current_stream().cuda_stream
        assert L.sbbf_find_hashes(g, dq.data_ptr(), q.size, out.data_ptr(), s) == 0
        assert np.array_equal(bits_np(out), oracle.find(ref, B, q))
    finally:
        L.sbbf_destroy(g)


def test_argument_errors_on_device():
    L = abi.lib()
    f = sb.Filter(64)
    keys = to_dev(inp.stream(126, 0, 100))
    s = torch.cuda.current_stream().cuda_stream
    assert L.sbbf_insert_hashes(f.handle, keys.data_ptr() + 4, 10, s) == abi.SBBF_EINVAL
    out = torch.empty(4, dtype=torch.int32, device=dev())
    assert L.sbbf_find_hashes(f.handle, keys.data_ptr(), 10, out.data_ptr() + 2, s) == \
        abi.SBBF_EINVAL
    assert L.sbbf_find_hashes(f.handle, keys.data_ptr(), 10, None, s) == abi.SBBF_EINVAL
    assert L.sbbf_insert_hashes(f.handle, None, 0, s) == abi.SBBF_OK  # n == 0 no-op
    with pytest.raises(TypeError):
        f.insert(keys.to(torch.int32))


def test_device_generators_match_host_copy():
    n = 1_000_003
    d = torch.empty(n, dtype=torch.int64, device=dev())
    sb.fill_splitmix64(d, 1234567, 0)
    got = u64_np(d)
    assert int(got[0]) == 6457827717110365317  # published splitmix64 reference output
    assert np.array_equal(got, inp.splitmix64(1234567, 0, n))
    sb.fill_splitmix64(d[:1000], 99, 5_000_000_000)
    assert np.array_equal(u64_np(d[:1000]), inp.splitmix64(99, 5_000_000_000, 1000))
    for w in (wl.C0, wl.C1, wl.C2):
        start = 99_000 if w is wl.C0 else 123_456_789
        q = wl.gen_queries(w, start, 100_000)
        exp = inp.workload_queries(w.cfg, w.n_insert, w.member_frac, w.member_prefix, start,
                                   100_000)
        assert np.array_equal(u64_np(q), exp)
        ins = wl.gen_inserts(w, 77, 1000)
        assert np.array_equal(u64_np(ins), inp.stream(w.cfg, 0, 1000, 77))


def test_count_bits():
    bits = to_dev(inp.stream(127, 0, 1000)).view(torch.int32)
    words = bits_np(bits)
    for n in (0, 1, 31, 33, 2000 - 5, 2000 * 32):
        c = int(sb.count_bits(bits, n).item())
        exp = sum(int(bit_at(words, k)) for k in range(n)) if n < 5000 else \
            int(np.unpackbits(words.view(np.uint8)).sum())
        assert c == exp


def test_host_pipe_parity():
    B = 32768
    n = 3 * 4096 + 77
    keys = inp.stream(128, 0, n)
    q = np.concatenate([inp.stream(128, 1, n), keys])
    hk = torch.from_numpy(keys.view(np.int64)).pin_memory()
    hq = torch.from_numpy(q.view(np.int64)).pin_memory()
    out = torch.zeros(sb.out_words(q.size), dtype=torch.int32).pin_memory()
    pipe = sb.HostPipe(4096)
    f = sb.Filter(B)
    pipe.insert(f, hk)
    pipe.find(f, hq, out)
    ref = _oracle_filter(B, keys)
    assert np.array_equal(f.to_numpy(), ref)
    assert np.array_equal(out.numpy().view(np.uint32), oracle.find(ref, B, q))
    # pageable host memory works too
    out2 = torch.zeros_like(out, device="cpu")
    pipe.find(f, torch.from_numpy(q.view(np.int64)), out2)
    assert np.array_equal(out2.numpy(), out.numpy())


@pytest.mark.parametrize("mode", ["copy", "direct"])
def test_host_pipe_into_region_pass_filter(mode):
    """Host-buffer lookups into a 128 MiB filter, which takes region passes
    for device batches of 8Mi hashes or more: staged chunks of 16Mi hashes go
    through two region passes, direct access to host memory through one
    pass; both give the single-pass device lookup's answers."""
    B = 2**22
    keys = inp.stream(127, 0, 2_000_000)
    q = np.concatenate([inp.stream(127, 1, 18_000_003), keys])
    f = sb.Filter(B)
    f.insert(to_dev(keys))
    assert f.region_passes(2**24) == 2
    f.set_partitioning(sb.PARTITION_OFF)
    exp = bits_np(f.find(to_dev(q)))
    f.set_partitioning(sb.PARTITION_AUTO)
    hq = torch.from_numpy(q.view(np.int64)).pin_memory()
    out = torch.full((sb.out_words(q.size),), -1, dtype=torch.int32).pin_memory()
    pipe = sb.HostPipe(2**24, mode=sb.PIPE_COPY if mode == "copy" else sb.PIPE_DIRECT)
    pipe.find(f, hq, out)
    assert np.array_equal(out.numpy().view(np.uint32), exp)


@pytest.mark.parametrize("mode", ["copy", "direct"])
def test_host_pipe_modes(mode):
    """Staged copies and in-place kernel access to pinned host memory give the
    oracle's filter and bits; direct mode refuses unmapped (pageable) memory."""
    B = 20_011
    n = 5 * 4096 + 33
    keys = inp.stream(129, 0, n)
    q = np.concatenate([inp.stream(129, 1, 2 * n), keys[:1000]])
    hk = torch.from_numpy(keys.view(np.int64)).pin_memory()
    hq = torch.from_numpy(q.view(np.int64)).pin_memory()
    out = torch.zeros(sb.out_words(q.size), dtype=torch.int32).pin_memory()
    pipe = sb.HostPipe(4096, mode=sb.PIPE_COPY if mode == "copy" else sb.PIPE_DIRECT)
    f = sb.Filter(B)
    pipe.insert(f, hk)
    pipe.find(f, hq, out)
    ref = _oracle_filter(B, keys)
    assert np.array_equal(f.to_numpy(), ref)
    assert np.array_equal(out.numpy().view(np.uint32), oracle.find(ref, B, q))
    if mode == "direct":
        with pytest.raises(sb.SbbfError):
            pipe.find(f, torch.from_numpy(q.view(np.int64)), out)  # pageable input
        # an odd-length tail and a 16-lane filter through the same mapping
        g = sb.Filter(777, lanes=16)
        pipe.insert(g, hk[:101])
        assert np.array_equal(g.to_numpy(), oracle.insert_k(np.zeros(777 * 16, np.uint32), 777,
                                                            16, keys[:101]))


def test_config_c0_full():
    """100k hashes in 4096 blocks; look up the 100k (all hit) then 1M fresh;
    bit-exact, and the measured FPR within the binomial interval."""
    w = wl.C0
    f = sb.Filter(w.num_blocks)
    wl.build_filter(w, f)
    q = wl.gen_queries(w, 0, w.n_lookup)
    bits = bits_np(f.find(q))
    keys = inp.stream(w.cfg, 0, w.n_insert)
    ref = _oracle_filter(w.num_blocks, keys)
    assert np.array_equal(f.to_numpy(), ref)
    qh = u64_np(q)
    ref_bits = oracle.find(ref, w.num_blocks, qh)
    assert np.array_equal(bits, ref_bits)
    hit = np.unpackbits(bits.view(np.uint8), bitorder="little")[: w.n_lookup].astype(bool)
    assert hit[: w.n_insert].all()
    fresh = ~np.isin(qh[w.n_insert:], keys)
    fp = int(hit[w.n_insert:][fresh].sum())
    p = oracle.fpr_poisson(w.n_insert / w.num_blocks)
    nq = int(fresh.sum())
    assert abs(fp / nq - p) <= 5 * np.sqrt(p * (1 - p) / nq) + 0.02 * p


def test_config_c1_full_size():
    """1M hashes into 32768 blocks; 256M lookups in one launch (the benchmark's
    launch): filter words and every one of the 268,435,456 answers equal the
    oracle's; members always hit."""
    w = wl.C1
    f = sb.Filter(w.num_blocks)
    wl.build_filter(w, f)
    keys = inp.stream(w.cfg, 0, w.n_insert)
    ref = _oracle_filter(w.num_blocks, keys)
    assert np.array_equal(f.to_numpy(), ref)
    q = wl.gen_queries(w, 0, w.n_lookup)
    bits = f.find(q)
    compare_all_lookups(w, ref, q, bits)
    head = 8 * 2**20
    member = inp.query_is_member(w.cfg, head, w.member_frac)
    hit = np.unpackbits(bits_np(bits[: head // 32]).view(np.uint8), bitorder="little").astype(bool)
    assert hit[member].all()


def test_bench_step_as_cuda_graph():
    """The 1 MiB filter's step as a CUDA graph: clear, insert 1M, look up
    256M, captured once and replayed; after two replays the words and every
    answer are the oracle's."""
    w = wl.C1
    f = sb.Filter(w.num_blocks)
    ins = wl.gen_inserts(w, 0, w.n_insert, device=dev())
    q = wl.gen_queries(w, 0, w.n_lookup)
    out = torch.empty(sb.out_words(w.n_lookup), dtype=torch.int32, device=dev())

    def step():
        f.clear()
        f.insert(ins)
        f.find(q, out=out)

    step()  # eager warm-up
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    out.fill_(-1)
    f.words.fill_(-1)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    keys = inp.stream(w.cfg, 0, w.n_insert)
    ref = _oracle_filter(w.num_blocks, keys)
    assert np.array_equal(f.to_numpy(), ref)
    compare_all_lookups(w, ref, q, out)


def test_config_c2_full_size():
    """The default benchmark workload as the benchmark runs it: 100M hashes
    into 4,194,304 blocks in 16M batches, then 1e9 lookups, captured as one
    CUDA graph and replayed twice: words bit-exact and every one of the 1e9
    answers equal to the oracle's."""
    w = wl.C2
    f = sb.Filter(w.num_blocks)
    ins = wl.gen_inserts(w, 0, w.n_insert, device=dev())
    q = wl.gen_queries(w, 0, w.n_lookup)
    out = torch.empty(sb.out_words(w.n_lookup), dtype=torch.int32, device=dev())

    def step():
        f.clear()
        for s0 in range(0, w.n_insert, w.insert_batch):
            f.insert(ins[s0:s0 + w.insert_batch])
        f.find(q, out=out)

    step()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    out.fill_(-1)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    del ins
    ref = oracle_filter_of_stream(w)
    compare_words(f.words, ref)
    compare_all_lookups(w, ref, q, out)
    del q, out, g
    torch.cuda.empty_cache()


PARTITION_CASES = [(2**17, 300_001), (3 * 2**17 + 9, 700_001), (2**19, 1_000_003),
                   (2**20, 0), (2**20, 1), (2**20 + 5, 16385), (3 * 2**20 - 1, 1_000_003),
                   (5 * 2**20 + 77, 2_500_000), (4_194_304, 4_200_000)]


@pytest.mark.parametrize("B,n", PARTITION_CASES)
def test_partitioned_insert_equals_oracle(B, n):
    """Slice-partitioned inserts (forced on) give the oracle's filter,
    across slice counts 1..41 (4 MiB slices for inserts; up to 4 slices the
    scatter ranks by warp match, past 4 by per-key atomics), ragged tiles and
    tails."""
    keys = inp.stream(130 + B % 11, 0, n)
    f = sb.Filter(B).set_partitioning(sb.PARTITION_ON)
    f.insert(to_dev(keys))
    ref = _oracle_filter(B, keys)
    assert np.array_equal(f.to_numpy(), ref)
    g = sb.Filter(B).set_partitioning(sb.PARTITION_OFF)
    g.insert(to_dev(keys))
    assert np.array_equal(g.to_numpy(), ref)


def test_partitioned_insert_unaligned_and_repeated():
    B, n = 2 * 2**20 + 3, 3_000_001
    keys = inp.stream(131, 0, n + 1)
    dk = to_dev(keys)
    f = sb.Filter(B).set_partitioning(sb.PARTITION_ON)
    f.insert(dk[1:])             # 8-byte aligned only
    f.insert(dk[: n // 3])       # a smaller batch reuses the scratch
    f.insert(dk[1:])             # idempotent
    ref = _oracle_filter(B, np.concatenate([keys[1:], keys[: n // 3]]))
    assert np.array_equal(f.to_numpy(), ref)
    with pytest.raises(sb.SbbfError):
        f.set_partitioning(7)


def test_partitioned_many_slices():
    """41 slices (per-key atomic ranking): inserts and lookups,
    with an odd batch length and an 8-byte-aligned (not 16) hash array, which
    the scatter reads without bulk copies."""
    B, n = 41 * 2**20 + 123, 2_000_001
    keys = inp.stream(132, 0, n + 1)
    dk = to_dev(keys)
    ref = _oracle_filter(B, keys[:n])
    for view in (dk[:n], dk[1:]):
        f = sb.Filter(B).set_partitioning(sb.PARTITION_ON)
        f.insert(view)
        exp = ref if view.data_ptr() == dk.data_ptr() else _oracle_filter(B, keys[1:])
        assert np.array_equal(f.to_numpy(), exp)
    f = sb.Filter(B)
    f.words.copy_(torch.from_numpy(ref.view(np.int32)).to(dev()))
    q = np.concatenate([inp.stream(132, 1, n), keys[: n // 2]])
    dq = to_dev(q)
    f.set_partitioning(sb.PARTITION_ON)
    for view, qq in ((dq, q), (dq[1:], q[1:])):
        assert np.array_equal(bits_np(f.find(view)), oracle.find(ref, B, qq))


@pytest.mark.parametrize("B,n", [(2**20, 1), (2**20 + 5, 16_385), (3 * 2**20 - 1, 1_000_003),
                                 (5 * 2**20 + 77, 2_500_033)])
def test_partitioned_find_equals_oracle(B, n):
    """Slice-partitioned lookups (forced on) answer exactly as the oracle,
    every bit at its original position, tail bits zero; 1 and 3 slices (32
    MiB slices, warp-match ranking) and 6 (per-key atomics)."""
    keys = inp.stream(140 + B % 13, 0, max(1, n // 3))
    q = np.concatenate([inp.stream(140 + B % 13, 1, n - n // 4), keys[: n // 4]])[:n]
    f = sb.Filter(B)
    f.insert(to_dev(keys))
    ref = _oracle_filter(B, keys)
    f.set_partitioning(sb.PARTITION_ON)
    out = torch.full((sb.out_words(n) + 1,), -1, dtype=torch.int32, device=dev())
    f.find(to_dev(q), out=out)
    got = bits_np(out)
    assert np.array_equal(got[: sb.out_words(n)], oracle.find(ref, B, q))
    assert got[-1] == 0xFFFFFFFF  # nothing written past the answers
    f.set_partitioning(sb.PARTITION_OFF)
    assert np.array_equal(bits_np(f.find(to_dev(q))), oracle.find(ref, B, q))


@pytest.mark.parametrize("B,n,passes", [(2**21 + 1, 1, 2), (2**21 + 1, 100_003, 2),
                                         (3 * 2**20 - 1, 1_000_003, 2),
                                         (5 * 2**20 + 77, 2_500_033, 3)])
def test_region_pass_lookups_equal_oracle(B, n, passes):
    """Lookups by region passes (forced): the first pass writes every answer
    word, the later ones OR in the answers of the hashes whose block lies in
    their range.  Every answer equals the oracle's and the single-pass
    lookup's, tail bits are zero, and nothing is written outside the answer
    words, with the output at 0, 4, 8 and 12 bytes past a 16-byte boundary
    (over stale words, which the first pass must overwrite)."""
    keys = inp.stream(150 + B % 7, 0, max(1, n // 3))
    q = np.concatenate([inp.stream(150 + B % 7, 1, n - n // 4), keys[: n // 4]])[:n]
    f = sb.Filter(B)
    f.insert(to_dev(keys))
    ref = _oracle_filter(B, keys)
    exp = oracle.find(ref, B, q)
    dq = to_dev(q)
    f.set_partitioning(sb.PARTITION_REGIONS)
    assert f.region_passes(n) == passes
    nw = sb.out_words(n)
    for shift_words in (0, 1, 2, 3):
        out = torch.full((shift_words + nw + 1,), -1, dtype=torch.int32, device=dev())
        f.find(dq, out=out[shift_words: shift_words + nw])
        got = bits_np(out)
        assert (got[:shift_words] == 0xFFFFFFFF).all() and got[-1] == 0xFFFFFFFF
        assert np.array_equal(got[shift_words: shift_words + nw], exp)
    f.set_partitioning(sb.PARTITION_OFF)
    assert np.array_equal(bits_np(f.find(dq)), exp)


def test_region_passes_random_shapes():
    """Seeded random filter sizes (one to four 64 MiB regions, ragged) and
    batch lengths (ragged tails, empty): lookups by forced region passes
    equal the single-pass lookups, and inserts by forced region passes give
    the single-pass filter, word for word."""
    rng = np.random.default_rng(2101)
    for trial in range(12):
        B = int(rng.integers(2**20, 4 * 2**21 + 3))
        n = int(rng.choice([0, 1, 63, 65, int(rng.integers(1, 3_000_000))]))
        keys = inp.stream(190 + trial, 0, max(n, 1))[:n]
        dk = to_dev(keys) if n else torch.empty(0, dtype=torch.int64, device=dev())
        f = sb.Filter(B).set_partitioning(sb.PARTITION_REGIONS)
        g = sb.Filter(B).set_partitioning(sb.PARTITION_OFF)
        f.insert(dk)
        g.insert(dk)
        assert torch.equal(f.words, g.words), (B, n)
        q = np.concatenate([inp.stream(190 + trial, 1, n), keys[: n // 3]])
        dq = to_dev(q) if q.size else torch.empty(0, dtype=torch.int64, device=dev())
        assert torch.equal(f.find(dq), g.find(dq)), (B, n)
        del f, g


@pytest.mark.parametrize("B,n,passes", [(2**21 + 1, 1, 2), (2**21 + 1, 1_000_003, 2),
                                         (5 * 2**20 + 77, 2_500_001, 3)])
def test_region_pass_inserts_equal_oracle(B, n, passes):
    """Inserts by region passes (forced): one launch per block range, each
    inserting only the hashes whose block lies in its range, give the
    oracle's filter, from a 16-byte aligned and an 8-byte aligned hash
    array."""
    keys = inp.stream(160 + B % 5, 0, n + 1)
    dk = to_dev(keys)
    for view, kk in ((dk[:n], keys[:n]), (dk[1:], keys[1:])):
        f = sb.Filter(B).set_partitioning(sb.PARTITION_REGIONS)
        assert f.region_passes(n, lookup=False) == passes
        f.insert(view)
        assert np.array_equal(f.to_numpy(), _oracle_filter(B, kk))


@pytest.mark.parametrize("B,n", [(32768, 1_000_003), (3 * 2**20 - 1, 200_001), (7, 130)])
@pytest.mark.parametrize("shift_words", [1, 2, 3])
def test_find_into_offset_outputs(B, n, shift_words):
    """Answers written 4, 8 or 12 bytes past a 16-byte boundary (the lookup
    picks 16-, 8- or 4-byte stores by the output's alignment) equal the
    oracle's, and the words on either side stay untouched."""
    keys = inp.stream(170, 0, max(1, n // 4))
    q = np.concatenate([inp.stream(170, 1, n - n // 8), keys[: n // 8]])
    ref = _oracle_filter(B, keys)
    f = sb.Filter(B)
    f.insert(to_dev(keys))
    w = sb.out_words(n)
    buf = torch.full((w + shift_words + 4,), -1, dtype=torch.int32, device=dev())
    f.find(to_dev(q), out=buf[shift_words: shift_words + w])
    got = bits_np(buf)
    assert np.array_equal(got[shift_words: shift_words + w], oracle.find(ref, B, q))
    assert (got[:shift_words] == 0xFFFFFFFF).all() and (got[shift_words + w:] == 0xFFFFFFFF).all()


@pytest.mark.parametrize("bits_per_key", [5, 8, 10.5, 12.8])
def test_bits_per_key_sweep(bits_per_key):
    """The sweep of the L2-resident configuration: 1M hashes at 5, 8, 10.5
    and 12.8 bits per key (19,532 / 31,250 / 41,016 / 50,000 blocks).  The
    filter words and the answers for 2M fresh hashes equal the oracle's, and
    the false-positive count lies in the binomial interval of the paper's
    Poisson sum."""
    n, q = 1_000_000, 2_000_000
    B = int(np.ceil(n * bits_per_key / 256))
    keys = inp.stream(190, 0, n)
    fresh = inp.stream(190, 1, q)
    f = sb.Filter(B)
    f.insert(to_dev(keys))
    ref = oracle.new_filter(B)
    oracle.insert_mt(ref, B, keys, oracle.num_cores())
    assert np.array_equal(f.to_numpy(), ref)
    got = bits_np(f.find(to_dev(fresh)))
    exp, _ = oracle.find_mt(ref, B, fresh, oracle.num_cores())
    assert np.array_equal(got, exp)
    fp = int(np.unpackbits(got.view(np.uint8)).sum())
    p = oracle.fpr_poisson(n / B)
    assert abs(fp / q - p) <= 5 * np.sqrt(p * (1 - p) / q) + 0.02 * p, (fp / q, p)


def test_partition_applies_follows_the_rule():
    """sbbf_partition_applies and sbbf_region_passes report the automatic
    rule (region passes for lookups of at least 8Mi hashes into filters of
    84-192 MiB, 64 MiB per region; otherwise partitioned from 4Mi hashes for
    inserts and 8Mi for lookups, a filter of at least 96 MiB for inserts and
    more than 128 MiB for lookups, at least 0.25 hashes per block for
    inserts and 0.6 for lookups) and the forced modes."""
    f = sb.Filter(2**23)  # 256 MiB
    assert f.partition_applies(2**22) and not f.partition_applies(2**22 - 1)  # 4Mi minimum
    assert f.partition_applies(2**23, lookup=True)           # 8Mi minimum for lookups
    assert not f.partition_applies(2**23 - 1, lookup=True)
    assert f.region_passes(2**27) == 1
    g = sb.Filter(2**25)  # 1 GiB
    assert g.partition_applies(2**23) and not g.partition_applies(2**23 - 1)  # 0.25 per block
    assert g.partition_applies(20_132_660, lookup=True)      # ceil(0.6 * 2^25)
    assert not g.partition_applies(20_132_659, lookup=True)
    del g
    big = 2**27
    ins96 = sb.Filter(3 * 2**20)  # 96 MiB: inserts partition, lookups do not
    assert ins96.partition_applies(big) and not ins96.partition_applies(big, lookup=True)
    assert not sb.Filter(3 * 2**20 - 1).partition_applies(big)
    at128 = sb.Filter(2**22)  # 128 MiB: lookups by two region passes
    assert at128.partition_applies(big) and not at128.partition_applies(big, lookup=True)
    assert at128.region_passes(big) == 2 and at128.region_passes(2**23) == 2
    assert at128.region_passes(2**23 - 1) == 1 and at128.region_passes(0) == 1
    at192 = sb.Filter(6 * 2**20)  # 192 MiB: three region passes
    assert at192.region_passes(big) == 3 and not at192.partition_applies(big, lookup=True)
    assert at192.partition_applies(2**23 - 1, lookup=True) is False  # below 8Mi: random
    above = sb.Filter(6 * 2**20 + 1)  # past 192 MiB: partitioned lookups
    assert above.region_passes(big) == 1 and above.partition_applies(big, lookup=True)
    assert sb.Filter(84 * 2**15).region_passes(big) == 1       # 84 MiB: random
    assert sb.Filter(84 * 2**15 + 1).region_passes(big) == 2
    assert ins96.region_passes(big) == 2
    ins96.set_partitioning(sb.PARTITION_OFF)
    assert ins96.region_passes(big) == 1
    forced = sb.Filter(2**21 + 1).set_partitioning(sb.PARTITION_REGIONS)  # 64 MiB + 32 B
    assert forced.region_passes(1) == 2 and sb.Filter(2**21).set_partitioning(
        sb.PARTITION_REGIONS).region_passes(big) == 1
    assert not forced.partition_applies(big, lookup=True)
    assert forced.partition_applies(2**22) is False and forced.region_passes(5, lookup=False) == 2
    big_forced = sb.Filter(2**23).set_partitioning(sb.PARTITION_REGIONS)  # 256 MiB: 4 regions
    assert big_forced.region_passes(2**22, lookup=False) == 4
    assert not big_forced.partition_applies(2**22)
    del ins96, at128, at192, above, forced, big_forced
    f.set_partitioning(sb.PARTITION_OFF)
    assert not f.partition_applies(2**30) and not f.partition_applies(2**30, lookup=True)
    f.set_partitioning(sb.PARTITION_ON)
    assert f.partition_applies(1) and f.partition_applies(1, lookup=True)
    assert not sb.Filter(4096, lanes=4).set_partitioning(sb.PARTITION_ON).partition_applies(2**30)


def test_partitioned_find_many_sub_ranges():
    """A batch large enough that every scatter range spans several answer
    sub-ranges (2^18 positions each), members spread through it, a ragged
    last range and tail: each answer lands at its original position exactly
    as the oracle says, and nothing is written past the answers."""
    B, n = 9 * 2**20 + 7, 100_000_037
    keys = inp.stream(150, 0, 12_000_000)
    q = np.concatenate([inp.stream(150, 1, n - keys.size), keys])
    q = q[np.random.default_rng(150).permutation(n)]
    ref = oracle.new_filter(B)
    oracle.insert_mt(ref, B, keys, oracle.num_cores())
    f = sb.Filter(B)
    f.words.copy_(torch.from_numpy(ref.view(np.int32)).to(dev()))
    f.set_partitioning(sb.PARTITION_ON)
    out = torch.full((sb.out_words(n) + 1,), -1, dtype=torch.int32, device=dev())
    f.find(to_dev(q), out=out)
    got = bits_np(out)
    exp, _ = oracle.find_mt(ref, B, q, oracle.num_cores())
    assert np.array_equal(got[: sb.out_words(n)], exp)
    assert got[-1] == 0xFFFFFFFF


def test_device_status_of_partitioned_calls():
    """The bulk-copy waits of the partitioned passes report through the
    filter's device status word: after ordinary partitioned calls no wait
    ran out (SBBF_OK); a recorded timeout bit (set on the host side, as a
    timed-out wait would) comes back once as SBBF_ETIMEOUT, then the word is
    clear again.  No device wait is made to run out."""
    B, n = 2**23 + 5, 5_000_001
    keys = inp.stream(190, 0, n)
    f = sb.Filter(B).set_partitioning(sb.PARTITION_ON)
    assert f.device_status() == abi.SBBF_OK  # nothing ran yet
    dk = to_dev(keys)
    f.insert(dk)
    bits = f.find(dk)
    assert f.device_status() == abi.SBBF_OK
    assert np.unpackbits(bits_np(bits).view(np.uint8), bitorder="little")[:n].all()
    for b in (1, 2, 3):
        f.record_device_status(b)
        assert f.device_status() == abi.SBBF_ETIMEOUT
        assert f.device_status() == abi.SBBF_OK
    f.record_device_status(0)
    assert f.device_status() == abi.SBBF_OK


@pytest.mark.parametrize("crowd_frac", [1.0, 0.3])
def test_partitioned_crowded_slices_take_the_fixup_path(crowd_frac):
    """Hashes that crowd one slice far beyond its share overflow their
    scatter buckets; the ranges of the CTAs that spilled are redone by the
    unpartitioned path, so inserts and lookups still equal the oracle's, when
    every CTA spills (all hashes in the first 1/64 of the blocks) and when
    only the CTAs holding the first 30% of the batch do."""
    B, n = 2**23 + 5, 5_000_003
    keys = inp.stream(191, 0, n)
    k = int(n * crowd_frac)
    keys[:k] = keys[:k] >> np.uint64(6)  # top bits below 2^58: blocks below B/64
    ref = _oracle_filter(B, keys)
    f = sb.Filter(B).set_partitioning(sb.PARTITION_ON)
    dk = to_dev(keys)
    f.insert(dk)
    assert np.array_equal(f.to_numpy(), ref)
    q = np.concatenate([inp.stream(191, 1, n), keys[::3]])
    q[: n // 2] = q[: n // 2] >> np.uint64(6)
    got = bits_np(f.find(to_dev(q)))
    assert np.array_equal(got, oracle.find(ref, B, q))
    assert f.device_status() == abi.SBBF_OK
