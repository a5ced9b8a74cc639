"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one.  Each mutant is a textual edit of oracle/sbbf_oracle.c,
compiled into a temporary library on the CPU; the real oracle is untouched.
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import sbbf_inputs as inp

SRC = os.path.join(os.path.dirname(oracle.__file__), "sbbf_oracle.c")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

MUTANTS = {
    "shift_28": ("uint32_t bit = product >> 27;", "uint32_t bit = product >> 28;"),
    "lanes_swapped": ("0x44974d91u, 0x47b6137bu,", "0x47b6137bu, 0x44974d91u,"),
    "block_from_low_half": ("uint64_t high = hash >> 32;",
                            "uint64_t high = hash & 0xffffffffu;"),
    "block_no_shift": ("return product >> 32;", "return product >> 31;"),
    "find_any_lane": ("if ((~words[8 * b + i] & mask[i]) != 0) return 0;\n  }\n  return 1;",
                      "if ((words[8 * b + i] & mask[i]) != 0) return 1;\n  }\n  return 0;"),
    "insert_wrong_lane": ("for (int i = 0; i < 8; ++i) words[8 * b + i] |= mask[i];",
                          "for (int i = 0; i < 8; ++i) words[8 * b + (i ^ 1)] |= mask[i];"),
    "insert_wrong_block": ("for (int i = 0; i < 8; ++i) words[8 * b + i] |= mask[i];",
                           "for (int i = 0; i < 8; ++i) words[8 * (b / 2) + i] |= mask[i];"),
    "multi_base_not_scaled": ("insert_one(arena + 8 * base_block[t]",
                              "insert_one(arena + base_block[t]"),
    "fpr_power_7": ("sum += exp(log_p) * pow(lane_hit, 8.0);",
                    "sum += exp(log_p) * pow(lane_hit, 7.0);"),
    "fpr_lane_prob": ("const double q = 1.0 - 1.0 / 32.0;",
                      "const double q = 1.0 - 1.0 / 31.0;"),
    "fpr_poisson_off_by_one": ("lgamma((double)i + 1.0)", "lgamma((double)i + 2.0)"),
    "splitmix_shift": ("z = (z ^ (z >> 30))", "z = (z ^ (z >> 31))"),
}


def _build(tmp, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mut = src.replace(old, new, 1)
    c = os.path.join(tmp, name + ".c")
    so = os.path.join(tmp, name + ".so")
    open(c, "w").write(mut)
    hdr = os.path.join(os.path.dirname(SRC))
    subprocess.run(["gcc", "-std=c99", "-O1", "-fPIC", "-shared", "-I", hdr,
                    "-o", so, c, "-lm", "-lpthread"], check=True)
    L = ctypes.CDLL(so)
    P64, P32 = ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)
    L.oracle_block_index.restype = ctypes.c_uint64
    L.oracle_block_index.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
    L.oracle_make_mask.argtypes = [ctypes.c_uint32, P32]
    L.oracle_insert.argtypes = [P32, ctypes.c_uint32, P64, ctypes.c_size_t]
    L.oracle_find.argtypes = [P32, ctypes.c_uint32, P64, ctypes.c_size_t, P32]
    L.oracle_multi_insert.restype = ctypes.c_uint64
    L.oracle_multi_insert.argtypes = [P32, P64, P32, ctypes.c_uint32, P64, P32,
                                      ctypes.c_size_t]
    L.oracle_fpr_poisson.restype = ctypes.c_double
    L.oracle_fpr_poisson.argtypes = [ctypes.c_double]
    L.oracle_splitmix64_at.restype = ctypes.c_uint64
    L.oracle_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    return L


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _rows(name):
    return [l.split() for l in open(os.path.join(GOLDEN, name))
            if l.strip() and not l.startswith("#")]


def _first_failure(L):
    """Name of the first pin the library fails, else None.  Stops at the first
    failure so that a mutant that already mis-indexes blocks never writes."""
    for name, passed in _pins(L):
        if not passed:
            return name
    return None


def _pins(L):
    """Yields (name, passed) for a compact set of the oracle's pins."""
    ok = True
    for r in _rows("appendix_masks.txt"):
        h = int(r[0], 16)
        m = np.zeros(8, np.uint32)
        L.oracle_make_mask(h & 0xFFFFFFFF, _p32(m))
        ok &= L.oracle_block_index(h, 4096) == int(r[1])
        ok &= L.oracle_block_index(h, 1000) == int(r[2])
        ok &= [int(x, 16) for x in r[3:11]] == [int(v) for v in m]
    yield "appendix masks", ok
    yield "splitmix reference", L.oracle_splitmix64_at(1234567, 0) == 6457827717110365317
    # no false negatives + measured FPR within the binomial interval
    B, keys, q = 4096, inp.stream(0, 0, 100_000), inp.stream(0, 1, 200_000)
    f = np.zeros(8 * B, np.uint32)
    L.oracle_insert(_p32(f), B, _p64(keys), keys.size)
    bits = np.zeros((keys.size + 31) // 32, np.uint32)
    L.oracle_find(_p32(f), B, _p64(keys), keys.size, _p32(bits))
    yield "no false negatives", bool(np.all(bits == 0xFFFFFFFF))
    qb = np.zeros((q.size + 31) // 32, np.uint32)
    L.oracle_find(_p32(f), B, _p64(q), q.size, _p32(qb))
    fp = int(np.unpackbits(qb.view(np.uint8)).sum()) / q.size
    p = oracle.fpr_poisson(100_000 / 4096)  # the real oracle's formula
    yield "fpr statistical", abs(fp - p) <= 5 * math.sqrt(p * (1 - p) / q.size) + 0.02 * p
    # the formula against its binomial-expansion closed form and the paper
    def closed(a):
        qq = 31 / 32
        return math.fsum(math.comb(8, k) * (-1) ** k * math.exp(-a * (1 - qq ** k))
                         for k in range(9))
    yield "fpr closed form", all(abs(L.oracle_fpr_poisson(a) - closed(a)) < 1e-9 * closed(a) + 1e-13
                                 for a in (2.79, 24.4, 52.0))
    # multi-filter arena == separate filters
    sizes = np.array([3, 17, 40], np.uint32)
    base = np.array([0, 3, 20], np.uint64)
    arena = np.zeros(8 * 60, np.uint32)
    mk = inp.stream(3, 0, 3000)
    ids = (inp.stream(3, 4, 3000) % np.uint64(3)).astype(np.uint32)
    L.oracle_multi_insert(_p32(arena), _p64(base), _p32(sizes), 3, _p64(mk), _p32(ids), mk.size)
    good = True
    for t in range(3):
        g = oracle.new_filter(int(sizes[t]))
        oracle.insert(g, int(sizes[t]), mk[ids == t])
        good &= np.array_equal(arena[8 * int(base[t]): 8 * (int(base[t]) + int(sizes[t]))], g)
    yield "multi == single", bool(good)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    with tempfile.TemporaryDirectory() as tmp:
        L = _build(tmp, name, old, new)
        failed = _first_failure(L)
    assert failed is not None, "mutant %s passed every pin" % name


def test_unmutated_copy_passes_every_pin():
    with tempfile.TemporaryDirectory() as tmp:
        L = _build(tmp, "identity", "#include <math.h>", "#include <math.h>")
        assert _first_failure(L) is None
