"""Pins of the oracle's key hashing (XXH64), of Parquet's block layout and of
the four- and sixteen-lane variants.

The paper hashes each key once to 64 bits and fixes no hash function; the
oracle's key hash is XXH64, the hash Parquet's split block filters use.  Two
independent sources pin it: XXH64's published test vectors, and the Bloom
filters Apache Arrow's Parquet writer builds (pyarrow, where installed),
whose bitsets must equal the oracle's filters up to the lane permutation the
seed-order reading predicts.
"""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle
import sbbf_inputs as inp

# Published XXH64 digests (the xxHash reference documentation and the
# python-xxhash package documentation), covering the empty input, the 1-byte
# and 4-byte tails, a seed, and the 32-byte stripe loop with a 7-byte tail.
XXH64_VECTORS = [
    (b"", 0, 0xEF46DB3751D8E999),
    (b"a", 0, 0xD24EC4F1A98C6E5B),
    (b"abc", 0, 0x44BC2CF5AD770999),
    (b"xxhash", 0, 0x32DD38952C4BC720),
    (b"xxhash", 20141025, 0xB559B98D844E0635),
    (b"Nobody inspects the spammish repetition", 0, 0xFBCEA83C8A378BF1),
]


@pytest.mark.parametrize("data,seed,want", XXH64_VECTORS)
def test_xxh64_published_vectors(data, seed, want):
    assert oracle.xxh64(data, seed) == want


def test_xxh64_fixed_and_var_agree_with_one_shot():
    keys = inp.stream(7, 0, 257)
    h = oracle.xxh64_fixed(keys)
    assert [int(x) for x in h[:5]] == [oracle.xxh64(int(k).to_bytes(8, "little")) for k in keys[:5]]
    k32 = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    h32 = oracle.xxh64_fixed(k32, seed=5)
    assert int(h32[3]) == oracle.xxh64(int(k32[3]).to_bytes(4, "little"), 5)
    lens = np.arange(0, 70, dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    data = (inp.stream(7, 1, int(offsets[-1])) & np.uint64(0xFF)).astype(np.uint8)
    hv = oracle.xxh64_var(data, offsets, seed=9)
    for k in (0, 3, 4, 7, 8, 31, 32, 33, 63, 64, 69):
        seg = data[int(offsets[k]):int(offsets[k + 1])].tobytes()
        assert int(hv[k]) == oracle.xxh64(seg, 9), k


# ---- Apache Arrow's Parquet Bloom filters -------------------------------------

def parquet_bitset(column, ndv, fpp=0.01):
    """Writes one column with a Bloom filter through pyarrow and returns the
    filter's words (little-endian uint32).  The filter is stored as a Thrift
    header followed by a power-of-two bitset, so the bitset is the largest
    power of two that fits in the stored length."""
    pa = pytest.importorskip("pyarrow")
    pq = pytest.importorskip("pyarrow.parquet")
    table = pa.table({"c": column})
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "t.parquet")
        pq.write_table(table, path, bloom_filter_options={"c": {"ndv": ndv, "fpp": fpp}})
        cc = pq.ParquetFile(path).metadata.row_group(0).column(0)
        off, length = cc.bloom_filter_offset, cc.bloom_filter_length
        raw = open(path, "rb").read()[off:off + length]
    nbytes = 1 << (length.bit_length() - 1)
    assert raw[0] == 0x15  # field 1 (numBytes), i32
    return np.frombuffer(raw[length - nbytes:], dtype="<u4").astype(np.uint32)


def oracle_filter(hashes, num_blocks):
    f = oracle.new_filter(num_blocks)
    oracle.insert(f, num_blocks, hashes)
    return f


def test_parquet_int64_filter_is_the_oracle_filter_with_lane_pairs_swapped():
    pa = pytest.importorskip("pyarrow")
    vals = inp.stream(8, 0, 20_000).view(np.int64)
    bits = parquet_bitset(pa.array(vals, type=pa.int64()), ndv=20_000)
    nb = bits.size // 8
    f = oracle_filter(oracle.xxh64_fixed(vals.astype("<i8")), nb)
    assert not np.array_equal(f, bits)  # the two lane orders differ ...
    assert np.array_equal(oracle.swap_lane_pairs(f), bits)  # ... by the pair swap


def test_parquet_int32_filter():
    pa = pytest.importorskip("pyarrow")
    vals = (inp.stream(8, 1, 5_000) >> np.uint64(32)).astype(np.uint32).view(np.int32)
    bits = parquet_bitset(pa.array(vals, type=pa.int32()), ndv=5_000, fpp=0.05)
    f = oracle_filter(oracle.xxh64_fixed(vals.astype("<i4")), bits.size // 8)
    assert np.array_equal(oracle.swap_lane_pairs(f), bits)


def test_parquet_binary_filter_all_tail_paths():
    pa = pytest.importorskip("pyarrow")
    n = 3_000
    lens = (inp.stream(8, 2, n) % np.uint64(100)).astype(np.uint64)
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    data = (inp.stream(8, 3, int(offsets[-1])) & np.uint64(0xFF)).astype(np.uint8)
    vals = [data[int(offsets[k]):int(offsets[k + 1])].tobytes() for k in range(n)]
    bits = parquet_bitset(pa.array(vals, type=pa.binary()), ndv=n)
    f = oracle_filter(oracle.xxh64_var(data, offsets), bits.size // 8)
    assert np.array_equal(oracle.swap_lane_pairs(f), bits)


def test_swap_lane_pairs_is_an_involution():
    w = inp.stream(8, 4, 64).astype(np.uint32)
    s = oracle.swap_lane_pairs(w)
    assert np.array_equal(oracle.swap_lane_pairs(s), w)
    assert s[0] == w[1] and s[1] == w[0] and s[7] == w[6]


# ---- four- and sixteen-lane variants ----------------------------------------

def test_k8_is_the_appendix_filter():
    hs = inp.stream(9, 0, 5000)
    a = oracle_filter(hs, 97)
    b = oracle.insert_k(np.zeros(8 * 97, np.uint32), 97, 8, hs)
    assert np.array_equal(a, b)
    q = inp.stream(9, 1, 3000)
    assert np.array_equal(oracle.find(a, 97, q), oracle.find_k(b, 97, 8, q))


@pytest.mark.parametrize("k", [4, 16])
def test_k_lanes_extend_the_appendix_mask(k):
    """Lanes shared with the eight-lane scheme set the same bits as the
    appendix mask; every lane holds exactly one bit."""
    for h in list(inp.stream(9, 2, 200)) + [0, 1, 1 << 31, 0xFFFFFFFF]:
        h = int(h)
        w = oracle.insert_k(np.zeros(k, np.uint32), 1, k, [h])
        m = oracle.make_mask(h & 0xFFFFFFFF)
        assert np.array_equal(w[:min(k, 8)], m[:min(k, 8)])
        assert all(bin(int(x)).count("1") == 1 for x in w)


def test_sixteen_lane_seeds_reading():
    """Lanes 8..15 use (splitmix64 output j of seed 0 >> 32) | 1: checked
    against the test inputs' own splitmix64, which is pinned to the
    published reference outputs."""
    for j in range(8):
        want = (int(inp._splitmix64_at(0, j)) >> 32) | 1
        assert oracle.seed_k(8 + j) == want
        assert want & 1
    assert [oracle.seed_k(i) for i in range(8)] == [int(s) for s in oracle.seeds()]


@pytest.mark.parametrize("k", [4, 16])
def test_k_lane_closed_forms(k):
    # x = 0: bit 0 in every lane; x = 2^31: odd seed * 2^31 = 2^31 -> bit 16;
    # x = 1: lane i holds bit s_i >> 27.
    for x, bit_of in ((0, lambda i: 0), (1 << 31, lambda i: 16),
                      (1, lambda i: oracle.seed_k(i) >> 27)):
        w = oracle.insert_k(np.zeros(k, np.uint32), 1, k, [x])
        assert [int(v) for v in w] == [1 << bit_of(i) for i in range(k)]


@pytest.mark.parametrize("k", [4, 16])
def test_k_lane_block_selection_and_no_false_negatives(k):
    hs = inp.stream(9, 3, 4000)
    nb = 61
    w = oracle.insert_k(np.zeros(k * nb, np.uint32), nb, k, hs)
    # each key touched only its block (appendix block_index)
    one = oracle.insert_k(np.zeros(k * nb, np.uint32), nb, k, hs[:1])
    b = oracle.block_index(int(hs[0]), nb)
    assert np.count_nonzero(one) == k and np.count_nonzero(one[k * b:k * b + k]) == k
    bits = oracle.find_k(w, nb, k, hs[:3999])
    got = np.unpackbits(bits.view(np.uint8), bitorder="little")
    assert got[:3999].all() and not got[3999:].any()


@pytest.mark.parametrize("k", [4, 16])
def test_fpr_k_closed_form(k):
    q = 31 / 32
    for a in (3.0, 12.19, 48.76):
        closed = math.fsum(math.comb(k, j) * (-1) ** j * math.exp(-a * (1 - q ** j))
                           for j in range(k + 1))
        assert abs(oracle.fpr_poisson_k(a, k) - closed) < 1e-9 * closed + 1e-12


@pytest.mark.parametrize("k,bits_per_key", [(4, 10.5), (16, 10.5)])
def test_k_lane_measured_fpr(k, bits_per_key):
    n = 60_000
    nb = int(math.ceil(n * bits_per_key / (32 * k)))
    w = oracle.insert_k(np.zeros(k * nb, np.uint32), nb, k, inp.stream(9, 4, n))
    qn = 400_000
    fp = oracle.find_k(w, nb, k, inp.stream(9, 5, qn))
    rate = int(np.unpackbits(fp.view(np.uint8)).sum()) / qn
    p = oracle.fpr_poisson_k(n / nb, k)
    assert abs(rate - p) <= 5 * math.sqrt(p * (1 - p) / qn) + 0.02 * p


def test_bad_lane_count_rejected():
    with pytest.raises(ValueError):
        oracle.insert_k(np.zeros(6, np.uint32), 1, 6, [1])


# ---- planted mistakes in a copy of the oracle must fail a pin above ------------

MUTANTS = {
    "xxh_round_rotation": ("acc = xrotl(acc, 31);", "acc = xrotl(acc, 30);"),
    "xxh_tail4_rotation": ("acc = xrotl(acc, 23) * XP2 + XP3;", "acc = xrotl(acc, 22) * XP2 + XP3;"),
    "xxh_length_dropped": ("acc += (uint64_t)len;", "acc += 0;"),
    "xxh_merge_repeats_v3": ("acc = xmerge(acc, v4);", "acc = xmerge(acc, v3);"),
    "xxh_big_endian_read": ("for (int i = bytes - 1; i >= 0; --i) v = (v << 8) | p[i];",
                            "for (int i = 0; i < bytes; ++i) v = (v << 8) | p[i];"),
    "xxh_avalanche_shift": ("acc ^= acc >> 29;", "acc ^= acc >> 28;"),
    "seed16_wrong_half": ("oracle_splitmix64_at(0, (uint64_t)(i - 8)) >> 32)",
                          "oracle_splitmix64_at(0, (uint64_t)(i - 8)) >> 31)"),
    "k_lane_block_halved": ("words[(uint64_t)k * b + (uint64_t)i] |=",
                            "words[(uint64_t)k * (b / 2) + (uint64_t)i] |="),
    "k_lane_shift_28": ("uint32_t bit = (uint32_t)(oracle_seed_k(i) * x) >> 27;\n      words",
                        "uint32_t bit = (uint32_t)(oracle_seed_k(i) * x) >> 28;\n      words"),
    "fpr_k_power": ("pow(1.0 - pow(q, (double)i), (double)k)",
                    "pow(1.0 - pow(q, (double)i), (double)(k - 1))"),
}
NEEDS_PYARROW = {"swap_identity": ("out[w] = in[w ^ 1];", "out[w] = in[w];")}


def _mutant_fails_a_pin(L):
    import ctypes
    P32, P64 = ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)
    u64, sz, i32 = ctypes.c_uint64, ctypes.c_size_t, ctypes.c_int
    L.oracle_xxh64.restype = u64
    L.oracle_xxh64.argtypes = [ctypes.c_void_p, sz, u64]
    L.oracle_seed_k.restype = ctypes.c_uint32
    L.oracle_seed_k.argtypes = [i32]
    L.oracle_insert_k.restype = i32
    L.oracle_insert_k.argtypes = [P32, ctypes.c_uint32, i32, P64, sz]
    L.oracle_fpr_poisson_k.restype = ctypes.c_double
    L.oracle_fpr_poisson_k.argtypes = [ctypes.c_double, i32]
    L.oracle_swap_lane_pairs.argtypes = [P32, sz, P32]
    L.oracle_xxh64_fixed.argtypes = [ctypes.c_void_p, sz, sz, u64, P64]
    for data, seed, want in XXH64_VECTORS:
        buf = ctypes.create_string_buffer(data, max(len(data), 1))
        if L.oracle_xxh64(buf, len(data), seed) != want:
            return True
    for j in range(8):
        if L.oracle_seed_k(8 + j) != ((int(inp._splitmix64_at(0, j)) >> 32) | 1):
            return True
    for k in (4, 16):
        for x, bit_of in ((1 << 31, lambda i: 16), (1, lambda i: L.oracle_seed_k(i) >> 27)):
            w = np.zeros(k, np.uint32)
            h = np.array([x], np.uint64)
            L.oracle_insert_k(w.ctypes.data_as(P32), 1, k, h.ctypes.data_as(P64), 1)
            if [int(v) for v in w] != [1 << bit_of(i) for i in range(k)]:
                return True
        # one key touches only its own block
        hs = inp.stream(9, 3, 1)
        w = np.zeros(k * 61, np.uint32)
        L.oracle_insert_k(w.ctypes.data_as(P32), 61, k, hs.ctypes.data_as(P64), 1)
        b = oracle.block_index(int(hs[0]), 61)
        if np.count_nonzero(w[k * b:k * b + k]) != k:
            return True
        q = 31 / 32
        a = 12.19
        closed = math.fsum(math.comb(k, j) * (-1) ** j * math.exp(-a * (1 - q ** j))
                           for j in range(k + 1))
        if abs(L.oracle_fpr_poisson_k(a, k) - closed) > 1e-9 * closed + 1e-12:
            return True
    try:
        import pyarrow as pa
    except ImportError:
        return False
    vals = inp.stream(8, 0, 2_000).view(np.int64)
    bits = parquet_bitset(pa.array(vals, type=pa.int64()), ndv=2_000)
    keys = np.ascontiguousarray(vals.astype("<i8"))
    hs = np.empty(vals.size, np.uint64)
    L.oracle_xxh64_fixed(keys.ctypes.data_as(ctypes.c_void_p), 8, keys.size, 0, hs.ctypes.data_as(P64))
    f = oracle_filter(hs, bits.size // 8)
    out = np.empty_like(f)
    L.oracle_swap_lane_pairs(f.ctypes.data_as(P32), f.size, out.ctypes.data_as(P32))
    return not np.array_equal(out, bits)


@pytest.mark.parametrize("name", sorted(MUTANTS) + sorted(NEEDS_PYARROW))
def test_key_and_lane_mutant_is_caught(name):
    import test_oracle_mutants as tm
    if name in NEEDS_PYARROW:
        pytest.importorskip("pyarrow")
    old, new = {**MUTANTS, **NEEDS_PYARROW}[name]
    with tempfile.TemporaryDirectory() as tmp:
        L = tm._build(tmp, name, old, new)
        assert _mutant_fails_a_pin(L), "mutant %s passed every pin" % name


def test_unmutated_copy_passes_key_and_lane_pins():
    import test_oracle_mutants as tm
    with tempfile.TemporaryDirectory() as tmp:
        L = tm._build(tmp, "identity", "#include <math.h>", "#include <math.h>")
        assert not _mutant_fails_a_pin(L)
