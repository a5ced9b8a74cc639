"""Pins for the scalar CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with a retyped copy of itself: each check is
a value the paper (or its appendix code) produces, a closed form, an
invariant, or brute force on tiny inputs.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import sbbf_inputs as inp

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


# ---- input generator -------------------------------------------------------

def test_splitmix64_reference_vector():
    """Both host splitmix64 copies reproduce the published reference outputs."""
    seed, expect = None, {}
    for row in _read_rows("splitmix64_reference.txt"):
        if row[0] == "seed":
            seed = int(row[1])
            expect[seed] = []
        else:
            expect[seed].append(int(row[0]))
    for seed, vals in expect.items():
        got_c = [oracle.splitmix64_at(seed, i) for i in range(len(vals))]
        got_np = [int(v) for v in inp.splitmix64(seed, 0, len(vals))]
        assert got_c == vals
        assert got_np == vals
    # counter form == sequential form: any window equals the full prefix slice
    full = oracle.splitmix64_fill(99, 0, 1000)
    assert np.array_equal(oracle.splitmix64_fill(99, 123, 500), full[123:623])
    assert np.array_equal(inp.splitmix64(99, 0, 1000), full)


# ---- block_index (appendix figure) -----------------------------------------

def test_appendix_golden_masks():
    """Masks and block indexes equal those the paper's appendix code printed."""
    rows = _read_rows("appendix_masks.txt")
    assert len(rows) >= 7
    for row in rows:
        h = int(row[0], 16)
        assert oracle.block_index(h, 4096) == int(row[1])
        assert oracle.block_index(h, 1000) == int(row[2])
        assert [int(x, 16) for x in row[3:11]] == [int(v) for v in oracle.make_mask(h)]


@pytest.mark.parametrize("B", [1, 2, 3, 1000, 4096, 4194304, 2**30, 2**32 - 1])
def test_block_index_closed_forms(B):
    # all-ones hash lands in the last block; hashes below 2^32 in block 0
    assert oracle.block_index(2**64 - 1, B) == B - 1
    assert oracle.block_index(2**32 - 1, B) == 0
    assert oracle.block_index(0, B) == 0
    # block b receives exactly the high halves in [ceil(b 2^32/B), ceil((b+1) 2^32/B))
    rng = np.random.default_rng(B)
    for b in rng.integers(0, B, size=20):
        b = int(b)
        first = -(-(b << 32) // B)
        nxt = -(-((b + 1) << 32) // B)
        assert oracle.block_index(first << 32, B) == b
        assert oracle.block_index(((nxt - 1) << 32) | 0xFFFFFFFF, B) == b
        if first > 0:
            assert oracle.block_index((first - 1) << 32, B) == b - 1


def test_block_index_ignores_low_half_and_is_monotone():
    hs = inp.stream(7, 0, 2000)
    for h in hs[:200]:
        h = int(h)
        assert oracle.block_index(h, 12345) == oracle.block_index(h & ~0xFFFFFFFF, 12345)
    srt = np.sort(hs)
    blocks = [oracle.block_index(int(h), 777) for h in srt]
    assert blocks == sorted(blocks)
    assert max(blocks) < 777


# ---- make_mask (intro + appendix figure) -----------------------------------

def test_mask_closed_forms():
    # x = 0: every product is 0 -> bit 0 in every lane
    assert list(oracle.make_mask(0)) == [1] * 8
    # x = 2^31: odd s times 2^31 is 2^31 mod 2^32 -> top five bits 10000b = 16
    assert list(oracle.make_mask(2**31)) == [1 << 16] * 8
    # x = 2^k: bit index = bits (27-k)..(31-k) of the seed
    s = oracle.seeds()
    assert all(int(v) & 1 for v in s), "seeds must be odd"
    for k in range(0, 28):
        m = oracle.make_mask(1 << k)
        for i in range(8):
            assert int(m[i]) == 1 << ((int(s[i]) >> (27 - k)) & 31)


def test_mask_one_bit_per_lane_eight_bits_total():
    xs = inp.stream(11, 0, 20000)
    for x in xs:
        m = oracle.make_mask(int(x) & 0xFFFFFFFF)
        assert all(bin(int(w)).count("1") == 1 for w in m)


def test_mask_uses_low_half_only():
    for h in inp.stream(12, 0, 300):
        h = int(h)
        assert np.array_equal(oracle.make_mask(h), oracle.make_mask(h & 0xFFFFFFFF))


def test_mask_lane_bits_roughly_uniform():
    """Each lane's bit index is close to uniform over [0,32) (multiply-shift)."""
    xs = inp.stream(13, 0, 64000) & np.uint64(0xFFFFFFFF)
    counts = np.zeros((8, 32), np.int64)
    for x in xs[:32000]:
        m = oracle.make_mask(int(x))
        for i in range(8):
            counts[i, int(m[i]).bit_length() - 1] += 1
    expect = 32000 / 32
    chi2 = ((counts - expect) ** 2 / expect).sum(axis=1)
    assert (chi2 < 100).all(), chi2  # 31 dof; 100 is far in the tail


# ---- insert / find (appendix add_hash, find_hash) --------------------------

def test_single_insert_sets_eight_bits_in_one_block():
    for h in inp.stream(14, 0, 50):
        h = int(h)
        B = 97
        f = oracle.new_filter(B)
        oracle.insert(f, B, [h])
        b = oracle.block_index(h, B)
        nz = np.nonzero(f)[0]
        assert set(nz // 8) == {b} and len(nz) == 8
        assert np.array_equal(f[8 * b: 8 * b + 8], oracle.make_mask(h))
        assert oracle.find_one(f, B, h)


def test_no_false_negatives_c0():
    B = 4096
    keys = inp.stream(0, inp.ROLE_INSERT, 100_000)
    f = oracle.new_filter(B)
    oracle.insert(f, B, keys)
    bits = oracle.find(f, B, keys)
    assert bits.size == (100_000 + 31) // 32
    assert np.all(bits == 0xFFFFFFFF)  # 100000 is a multiple of 32
    bits = oracle.find(f, B, keys[:99_990])
    assert np.all(bits[:-1] == 0xFFFFFFFF)
    assert bits[-1] == (1 << (99_990 % 32)) - 1


def test_order_independence_and_idempotence():
    B = 1000
    keys = inp.stream(15, 0, 30000)
    f1 = oracle.new_filter(B)
    oracle.insert(f1, B, keys)
    perm = inp.permutation(15, keys.size)
    dup = np.concatenate([keys[perm], keys[:5000]])
    f2 = oracle.new_filter(B)
    oracle.insert(f2, B, dup)
    assert np.array_equal(f1, f2)
    oracle.insert(f2, B, keys)  # inserting again changes nothing
    assert np.array_equal(f1, f2)


def test_union_equals_insert_of_union():
    B = 513
    a = inp.stream(16, 0, 9000)
    b = inp.stream(16, 1, 7000)
    fa, fb, fab = oracle.new_filter(B), oracle.new_filter(B), oracle.new_filter(B)
    oracle.insert(fa, B, a)
    oracle.insert(fb, B, b)
    oracle.insert(fab, B, np.concatenate([a, b]))
    assert np.array_equal(oracle.union(fa.copy(), fb), fab)
    assert np.array_equal(oracle.union(fb.copy(), fa), fab)


def test_find_monotone_under_inserts():
    B = 64
    q = inp.stream(17, 1, 5000)
    f = oracle.new_filter(B)
    prev = oracle.find(f, B, q)
    assert not prev.any()  # empty filter answers no
    for chunk in np.array_split(inp.stream(17, 0, 3000), 6):
        oracle.insert(f, B, chunk)
        cur = oracle.find(f, B, q)
        assert np.array_equal(cur & prev, prev)
        prev = cur


@pytest.mark.parametrize("B", [1, 2, 3])
def test_brute_force_tiny(B):
    """All 2^10 subsets of 10 hashes: the filter is the OR of one-key filters,
    and find(h) holds iff every lane bit of h was set by some inserted key in
    h's block."""
    hs = [int(x) for x in inp.stream(18, B, 10)]
    single = []
    for h in hs:
        f = oracle.new_filter(B)
        oracle.insert(f, B, [h])
        single.append(f)
    probes = [int(x) for x in inp.stream(18, 10 + B, 40)] + hs
    for mask in range(1 << len(hs)):
        chosen = [hs[i] for i in range(len(hs)) if mask >> i & 1]
        f = oracle.new_filter(B)
        oracle.insert(f, B, chosen)
        expect = np.zeros(8 * B, np.uint32)
        for i in range(len(hs)):
            if mask >> i & 1:
                expect |= single[i]
        assert np.array_equal(f, expect)
        if mask % 37 == 0:
            bits = oracle.find(f, B, probes)
            for k, p in enumerate(probes):
                pb, pm = oracle.block_index(p, B), oracle.make_mask(p)
                lanes_ok = all(
                    any(oracle.block_index(c, B) == pb
                        and oracle.make_mask(c)[i] == pm[i] for c in chosen)
                    for i in range(8))
                assert bool(bits[k // 32] >> (k % 32) & 1) == lanes_ok


def test_find_output_tail_bits_zero():
    B = 8
    keys = inp.stream(19, 0, 200)
    f = oracle.new_filter(B)
    oracle.insert(f, B, keys)
    for n in (0, 1, 31, 32, 33, 63, 65):
        bits = oracle.find(f, B, keys[:n])
        assert bits.size == (n + 31) // 32
        if n % 32:
            assert bits[-1] >> (n % 32) == 0


def test_block_range_insert_tiles_the_filter():
    B = 1001
    keys = inp.stream(20, 0, 40000)
    full = oracle.new_filter(B)
    oracle.insert(full, B, keys)
    cuts = [0, 1, 250, 251, 700, B]
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        sub = np.zeros(8 * (hi - lo), np.uint32)
        oracle.insert_block_range(sub, B, keys, lo, hi)
        assert np.array_equal(sub, full[8 * lo: 8 * hi])


def test_block_ranges_insert_equals_full_insert():
    B = 5003
    keys = inp.stream(23, 0, 60000)
    full = oracle.new_filter(B)
    oracle.insert(full, B, keys)
    lo = np.array([0, 7, 100, 2500, 4990], np.uint64)
    hi = np.array([3, 8, 160, 3000, 5003], np.uint64)
    out = np.zeros(8 * int((hi - lo).sum()), np.uint32)
    oracle.insert_block_ranges(out, B, keys, lo, hi)
    expect = np.concatenate([full[8 * int(a): 8 * int(b)] for a, b in zip(lo, hi)])
    assert np.array_equal(out, expect)


# ---- several filters in one arena -------------------------------------------

def test_multi_filter_equals_separate_filters():
    sizes = [1, 5, 64, 300]
    base = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.uint64)
    arena = np.zeros(8 * sum(sizes), np.uint32)
    keys = inp.stream(21, 0, 20000)
    ids = (inp.stream(21, 4, 20000) % np.uint64(len(sizes) + 1)).astype(np.uint32)
    ids[ids == len(sizes)] = 0xFFFFFFFF  # invalid id
    bad = oracle.multi_insert(arena, base, sizes, keys, ids)
    assert bad == int((ids == 0xFFFFFFFF).sum()) and bad > 0
    for t, B in enumerate(sizes):
        f = oracle.new_filter(B)
        oracle.insert(f, B, keys[ids == t])
        assert np.array_equal(arena[8 * int(base[t]): 8 * (int(base[t]) + B)], f)
    q = inp.stream(21, 1, 5000)
    qid = (inp.stream(21, 5, 5000) % np.uint64(len(sizes) + 1)).astype(np.uint32)
    qid[qid == len(sizes)] = 77
    bits, badq = oracle.multi_find(arena, base, sizes, q, qid)
    assert badq == int((qid == 77).sum())
    for k in range(q.size):
        t = int(qid[k])
        if t >= len(sizes):
            exp = False
        else:
            B = sizes[t]
            exp = oracle.find_one(arena[8 * int(base[t]): 8 * (int(base[t]) + B)], B, int(q[k]))
        assert bool(bits[k // 32] >> (k % 32) & 1) == exp


# ---- FPR analysis -----------------------------------------------------------

def _fpr_closed_form(a):
    """Binomial expansion of (1-q^i)^8 summed against Poisson(a):
    sum_k C(8,k) (-1)^k exp(-a (1 - q^k)), q = 31/32."""
    q = 31.0 / 32.0
    return math.fsum(math.comb(8, k) * (-1) ** k * math.exp(-a * (1 - q ** k))
                     for k in range(9))


@pytest.mark.parametrize("a", [0.3, 2.79, 20.0, 24.4140625, 30.517578125,
                               23.84185791015625, 51.2, 52.0, 100.0])
def test_fpr_series_equals_closed_form(a):
    assert oracle.fpr_poisson(a) == pytest.approx(_fpr_closed_form(a), rel=1e-9, abs=1e-13)  # abs: cancellation in the alternating sum


def test_fpr_limits():
    assert oracle.fpr_poisson(0.0) == 0.0
    # small a: one key in the block dominates, fpr ~ a * (1/32)^8
    assert oracle.fpr_poisson(1e-6) == pytest.approx(1e-6 * 32.0 ** -8, rel=1e-5)
    assert oracle.fpr_poisson(5000.0) == pytest.approx(1.0, abs=1e-9)
    xs = [oracle.fpr_poisson(a) for a in np.linspace(1, 80, 50)]
    assert all(x < y for x, y in zip(xs, xs[1:]))


def test_fpr_matches_paper_table():
    """The paper's measured epsilon (benchmark table) lies within 3% of the
    formula at its three sizes."""
    for n, B, eps in _read_rows("paper_fpr.txt"):
        a = int(n) / int(B)
        assert oracle.fpr_poisson(a) * 100 == pytest.approx(float(eps), rel=0.03)


def test_paper_claims():
    rows = {r[0]: r for r in _read_rows("paper_claims.txt")}
    a_lo, eps_lo = float(rows["a_lo"][1]), float(rows["a_lo"][3])
    a_hi, eps_hi = float(rows["a_hi"][1]), float(rows["a_hi"][3])
    assert round(oracle.fpr_poisson(a_lo) * 100, 2) == eps_lo
    assert round(oracle.fpr_poisson(a_hi) * 100) == eps_hi
    ratio = float(rows["max_ratio"][1])
    for a in np.linspace(a_lo, a_hi, 65):
        bpk = 256.0 / a
        std = min(oracle.fpr_standard(bpk, k) for k in range(1, 40))
        assert oracle.fpr_poisson(a) <= ratio * std
    # space at which the SBBF reaches 1.0%: bisect the monotone formula
    target = float(rows["sbbf_eps_percent"][1]) / 100
    lo, hi = 1.0, 60.0
    for _ in range(200):
        mid = (lo + hi) / 2
        lo, hi = (mid, hi) if oracle.fpr_poisson(mid) < target else (lo, mid)
    bpk = 256.0 / lo
    std = min(oracle.fpr_standard(bpk, k) for k in range(1, 40))
    assert std * 100 == pytest.approx(float(rows["sbbf_eps_percent"][3]), abs=0.01)


def _binomial_ok(fp, q, p):
    return abs(fp / q - p) <= 5 * math.sqrt(p * (1 - p) / q) + 0.02 * p


def _measured_fpr(B, n_ins, n_q, cfg):
    keys = inp.stream(cfg, inp.ROLE_INSERT, n_ins)
    fresh = inp.stream(cfg, inp.ROLE_FRESH, n_q)
    fresh = fresh[~np.isin(fresh, keys)]
    f = oracle.new_filter(B)
    oracle.insert(f, B, keys)
    bits = oracle.find(f, B, fresh)
    hits = int(np.unpackbits(bits.view(np.uint8)).sum())
    return hits, fresh.size


def test_fpr_statistical_c0():
    """100k keys in 4096 blocks, 1M fresh lookups: measured FPR within the
    binomial interval of the Poisson sum."""
    fp, q = _measured_fpr(4096, 100_000, 1_000_000, 0)
    p = oracle.fpr_poisson(100_000 / 4096)
    assert _binomial_ok(fp, q, p), (fp / q, p)


@pytest.mark.parametrize("bits_per_key", [5, 8, 10.5, 12.8])
def test_fpr_statistical_sweep(bits_per_key):
    n = 1_000_000
    B = math.ceil(n * bits_per_key / 256)
    fp, q = _measured_fpr(B, n, 400_000, 1)
    p = oracle.fpr_poisson(n / B)
    assert _binomial_ok(fp, q, p), (bits_per_key, fp / q, p)


# ---- timing drivers -----------------------------------------------------------

def test_multithreaded_drivers_equal_scalar():
    B = 4099
    keys = inp.stream(22, 0, 123_457)
    q = inp.stream(22, 1, 200_003)
    f = oracle.new_filter(B)
    oracle.insert(f, B, keys)
    for t in (1, 3, 8):
        g = oracle.new_filter(B)
        used = oracle.insert_mt(g, B, keys, t)
        assert used == t
        assert np.array_equal(f, g)
        bits, used = oracle.find_mt(f, B, q, t)
        assert np.array_equal(bits, oracle.find(f, B, q))


def test_query_recipe_members_hit():
    B = 4096
    keys = inp.stream(0, 0, 100_000)
    f = oracle.new_filter(B)
    oracle.insert(f, B, keys)
    q = inp.queries(0, keys, 50_000, 0.5)
    member = inp.query_is_member(0, 50_000, 0.5)
    assert 0.48 < member.mean() < 0.52
    bits = oracle.find(f, B, q)
    hit = np.unpackbits(bits.view(np.uint8), bitorder="little")[: q.size].astype(bool)
    assert hit[member].all()
    m10 = inp.query_is_member(2, 200_000, 0.1)
    assert 0.095 < m10.mean() < 0.105


# ---- the paper's appendix code, compiled here (x86-64 + AVX2 only) ----------

def test_appendix_crosscheck():
    from golden import make_appendix_masks as ax
    why = ax.available()
    if why:
        pytest.skip(why)
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        exe = ax.build(d)
        for B, n_ins, n_q, cfg in ((1, 40, 200, 30), (3, 100, 300, 31),
                                    (1000, 20000, 20000, 32), (4096, 30000, 30000, 33),
                                    (65537, 50000, 10000, 34)):
            ins = inp.stream(cfg, 0, n_ins)
            q = np.concatenate([inp.stream(cfg, 1, n_q), ins[: n_q // 4]])
            blocks, masks, words, finds = ax.run(exe, B, ins, q)
            assert blocks == [oracle.block_index(int(h), B) for h in ins]
            assert masks == [[int(v) for v in oracle.make_mask(int(h))] for h in ins]
            f = oracle.new_filter(B)
            oracle.insert(f, B, ins)
            assert words == [int(v) for v in f]
            bits = oracle.find(f, B, q)
            got = [int(bits[k // 32] >> (k % 32) & 1) for k in range(q.size)]
            assert got == finds
