"""Pins for the oracle's block-range verification digest (a checking aid, not
part of the method): per range of blocks, the sum mod 2^64 of splitmix64
output u seeded with 64-bit unit u's value, the set-bit count, and the count
of blocks holding both an all-zero lane and a non-zero lane.

The pins come from outside the digest code: the seeded-input module's own
splitmix64 (itself pinned to the published reference sequence), numpy's
unpackbits, the insert step's one-bit-per-lane property, additivity over
ranges, and brute-force single-bit sensitivity.  Each pin runs on the real
oracle and on copies with a planted mistake, every one of which must fail a
pin."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import sbbf_inputs as inp

SRC = os.path.join(os.path.dirname(oracle.__file__), "sbbf_oracle.c")
M64 = (1 << 64) - 1

MUTANTS = {
    "high_half_dropped": ("(uint64_t)blk[i] | ((uint64_t)blk[i + 1] << 32)", "(uint64_t)blk[i]"),
    "index_off_by_one": ("digest[r] += oracle_splitmix64_at(v, u);",
                         "digest[r] += oracle_splitmix64_at(v, u + 1);"),
    "index_per_block": ("const uint64_t u = ((first_block + b) * (uint64_t)lanes + (uint64_t)i) / 2;",
                        "const uint64_t u = (uint64_t)i / 2;"),
    "slice_index_local": ("const uint64_t u = ((first_block + b) * (uint64_t)lanes + (uint64_t)i) / 2;",
                          "const uint64_t u = (b * (uint64_t)lanes + (uint64_t)i) / 2;"),
    "popcount_once_per_word": ("bits[r] += 1;\n        w &= w - 1u;", "bits[r] += 1;\n        w = 0;"),
    "xor_fold": ("digest[r] += oracle_splitmix64_at(v, u);",
                 "digest[r] ^= oracle_splitmix64_at(v, u);"),
    "bits_skip_last_lane": ("for (int i = 0; i < lanes; ++i) {\n      uint32_t w = blk[i];",
                            "for (int i = 0; i < lanes - 1; ++i) {\n      uint32_t w = blk[i];"),
    "partial_counts_empty_blocks": ("if (zero_lanes > 0 && zero_lanes < lanes)",
                                    "if (zero_lanes > 0)"),
    "range_too_wide": ("const uint64_t r = b / range_blocks;",
                       "const uint64_t r = b / (range_blocks + 1);"),
}


class _Lib:
    """range_digest over a compiled copy of the oracle (real or mutated)."""

    def __init__(self, so):
        self.L = ctypes.CDLL(so)
        P64, P32 = ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)
        self.L.oracle_range_digest.argtypes = [P32, ctypes.c_uint64, ctypes.c_uint64,
                                               ctypes.c_int, ctypes.c_uint64, P64, P64, P64]

    def __call__(self, words, lanes, range_blocks, threads=1):
        """As oracle.range_digest; `threads` runs of whole ranges, one after
        another, each from its own first block."""
        w = np.ascontiguousarray(words, np.uint32)
        nb = w.size // lanes
        n = -(-nb // range_blocks)
        out = [np.zeros(n, np.uint64) for _ in range(3)]
        runs = max(1, min(threads, n))
        for k in range(runs):
            r0, r1 = n * k // runs, n * (k + 1) // runs
            b0, b1 = r0 * range_blocks, min(nb, r1 * range_blocks)
            p64 = [o[r0:].ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) for o in out]
            self.L.oracle_range_digest(w[b0 * lanes:].ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                       b0, b1 - b0, lanes, range_blocks, *p64)
        return out


def _compile(tmp, name, old=None, new=None):
    src = open(SRC).read()
    if old is not None:
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    c, so = os.path.join(tmp, name + ".c"), os.path.join(tmp, name + ".so")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-std=c99", "-O1", "-fPIC", "-shared", "-I", os.path.dirname(SRC),
                    "-o", so, c, "-lm", "-lpthread"], check=True)
    return _Lib(so)


def _sm_sum(seeds, first_unit):
    """sum mod 2^64 of splitmix64 output (first_unit + k) seeded with seeds[k],
    by the seeded-input module's generator."""
    tot = 0
    for k, s in enumerate(seeds):
        tot += int(inp.splitmix64(int(s), first_unit + k, 1)[0])
    return tot & M64


def _built_filter(lanes, nb, n_keys, cfg):
    """A filter of `lanes` lanes built by the oracle's inserts."""
    words = np.zeros(nb * lanes, np.uint32)
    oracle.insert_k(words, nb, lanes, inp.stream(cfg, 0, n_keys))
    return words


def _pins(D):
    """Yields (name, passed)."""
    # 1. all-zero words: every unit's seed is 0, so range r's digest is the sum
    #    of generator outputs over its units.
    ok = True
    for lanes in (4, 8, 16):
        nb, R = 37, 5
        d, b, p = D(np.zeros(nb * lanes, np.uint32), lanes, R)
        upb = lanes // 2
        for r in range(d.size):
            lo, hi = r * R, min(nb, (r + 1) * R)
            ok &= int(d[r]) == _sm_sum([0] * ((hi - lo) * upb), lo * upb)
        ok &= not b.any() and not p.any()
    yield "zero words: sum of generator outputs", ok
    # 2. one non-zero word: unit u's seed becomes the word (low half) or the
    #    word << 32 (high half); every other term stays as in the zero case.
    ok = True
    for lanes, w_idx, val in ((8, 0, 1), (8, 13, 0xDEADBEEF), (4, 7, 5), (16, 33, 0x80000000)):
        nb, R = 9, 4
        words = np.zeros(nb * lanes, np.uint32)
        words[w_idx] = val
        d, _, _ = D(words, lanes, R)
        dz, _, _ = D(np.zeros_like(words), lanes, R)
        u, r = w_idx // 2, (w_idx // lanes) // R
        seed = val << 32 if w_idx % 2 else val
        delta = (int(inp.splitmix64(seed, u, 1)[0]) - int(inp.splitmix64(0, u, 1)[0])) & M64
        ok &= (int(d[r]) - int(dz[r])) & M64 == delta
        ok &= all(int(d[k]) == int(dz[k]) for k in range(d.size) if k != r)
    yield "one word: its unit's generator output", ok
    # 3. set bits against numpy's bit unpacking, ragged last range.
    ok = True
    for lanes in (4, 8, 16):
        nb, R = 101, 16
        words = inp.stream(7, lanes, nb * lanes // 2).view(np.uint32).copy()
        words[::3] = 0
        words[1::5] &= np.uint32(0x0F0F0F0F)
        _, b, _ = D(words, lanes, R)
        exp = [int(np.unpackbits(words[r * R * lanes: min(nb, (r + 1) * R) * lanes]
                                 .view(np.uint8)).sum()) for r in range(b.size)]
        ok &= [int(x) for x in b] == exp
    yield "bits == unpackbits", ok
    # 4. additivity: a range's figures are the sums of its halves' figures, and
    #    one range over everything is the sum of all.
    ok = True
    for lanes in (4, 8, 16):
        nb = 64
        words = _built_filter(lanes, nb, 150, 8)
        first = int(np.flatnonzero(words.reshape(nb, lanes).any(axis=1))[0])
        words[lanes * first] = 0  # one planted partial block
        d6, b6, p6 = D(words, lanes, 6)
        d3, b3, p3 = D(words, lanes, 3)
        dall, ball, pall = D(words, lanes, 1000)
        for r in range(d6.size):
            parts = range(2 * r, min(d3.size, 2 * r + 2))
            ok &= int(d6[r]) == sum(int(d3[k]) for k in parts) & M64
            ok &= int(b6[r]) == sum(int(b3[k]) for k in parts)
            ok &= int(p6[r]) == sum(int(p3[k]) for k in parts)
        ok &= dall.size == 1 and int(dall[0]) == sum(int(x) for x in d3) & M64
        ok &= int(ball[0]) == int(b3.sum()) and int(pall[0]) == int(p3.sum()) == 1
    yield "additive over ranges", ok
    # 5. inserts set one bit in every lane of a block: no partial block after
    #    inserts; a planted zero lane in a non-empty block counts once, in its
    #    range; a block zeroed whole does not count.
    ok = True
    for lanes in (4, 8, 16):
        nb, R = 200, 32
        words = _built_filter(lanes, nb, 120, 9)
        _, _, p = D(words, lanes, R)
        ok &= not p.any()
        blocks = words.reshape(nb, lanes)
        nonempty = np.flatnonzero(blocks.any(axis=1))
        planted = nonempty[::7]
        for k, blk in enumerate(planted):
            blocks[blk, k % lanes] = 0
        emptied = nonempty[3::7]
        blocks[emptied] = 0
        planted = np.setdiff1d(planted, emptied)
        _, _, p = D(words, lanes, R)
        exp = np.bincount(planted // R, minlength=p.size)
        ok &= [int(x) for x in p] == [int(x) for x in exp]
    yield "partial blocks", ok
    # 6. every single-bit flip changes the digest of its own range and no other.
    ok = True
    lanes, nb, R = 8, 6, 2
    base = _built_filter(lanes, nb, 10, 10)
    d0, _, _ = D(base, lanes, R)
    for w in range(base.size):
        for bit in range(32):
            words = base.copy()
            words[w] ^= np.uint32(1 << bit)
            d, _, _ = D(words, lanes, R)
            r = (w // lanes) // R
            ok &= d[r] != d0[r] and all(d[k] == d0[k] for k in range(d.size) if k != r)
    yield "single-bit flips", ok
    # 7. order: swapping two unequal units, or the two halves of a unit,
    #    changes the digest.
    ok = True
    words = _built_filter(8, 4, 40, 11)
    d0, _, _ = D(words, 8, 4)
    u = words.view(np.uint64).copy()
    i, j = 1, 9
    assert u[i] != u[j]
    u[[i, j]] = u[[j, i]]
    ok &= D(u.view(np.uint32), 8, 4)[0][0] != d0[0]
    sw = words.copy()
    k = next(k for k in range(0, sw.size, 2) if sw[k] != sw[k + 1])
    sw[[k, k + 1]] = sw[[k + 1, k]]
    ok &= D(sw, 8, 4)[0][0] != d0[0]
    yield "unit order and halves", ok
    # 8. split into runs of whole ranges (each run from its own first block),
    #    the figures are those of one pass over everything.
    ok = True
    for lanes in (4, 16):
        words = _built_filter(lanes, 301, 900, 12)
        one = D(words, lanes, 10)
        for runs in (2, 7, 31):
            ok &= all(np.array_equal(a, c) for a, c in zip(D(words, lanes, 10, threads=runs), one))
    yield "runs of ranges", ok


def test_oracle_digest_passes_every_pin():
    for name, passed in _pins(oracle.range_digest):
        assert passed, name


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_digest_mutant_is_caught(name):
    with tempfile.TemporaryDirectory() as tmp:
        D = _compile(tmp, name, *MUTANTS[name])
        assert any(not passed for _, passed in _pins(D)), "mutant %s passed every pin" % name


def test_unmutated_copy_passes_every_pin():
    with tempfile.TemporaryDirectory() as tmp:
        D = _compile(tmp, "identity")
        for name, passed in _pins(D):
            assert passed, name
