"""Scalar CPU oracle for split block Bloom filters (arXiv 2101.01719).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The product path (the
CUDA library and its Python binding) never imports, links or calls it.

The arithmetic lives in ``sbbf_oracle.c`` (plain C99, no intrinsics); this
module compiles it with gcc and exposes it through ctypes on numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbbf_oracle.c")
_HDR = os.path.join(_HERE, "sbbf_oracle.h")
_LIB_PATH = os.path.join(_HERE, "libsbbf_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libsbbf_oracle.so`` (gcc, -O2, C99)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                                  os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
               "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            u64, u32, sz, i32 = (ctypes.c_uint64, ctypes.c_uint32,
                                 ctypes.c_size_t, ctypes.c_int)
            P64, P32 = ctypes.POINTER(u64), ctypes.POINTER(u32)
            sigs = {
                "oracle_block_index": (u64, [u64, u32]),
                "oracle_make_mask": (None, [u32, P32]),
                "oracle_seeds": (None, [P32]),
                "oracle_insert": (None, [P32, u32, P64, sz]),
                "oracle_insert_block_range": (None, [P32, u32, P64, sz, u64, u64]),
                "oracle_insert_block_ranges": (None, [P32, u32, P64, sz, P64, P64, sz]),
                "oracle_find_one": (i32, [P32, u32, u64]),
                "oracle_find": (None, [P32, u32, P64, sz, P32]),
                "oracle_union": (None, [P32, P32, sz]),
                "oracle_multi_insert": (u64, [P32, P64, P32, u32, P64, P32, sz]),
                "oracle_multi_find": (u64, [P32, P64, P32, u32, P64, P32, sz, P32]),
                "oracle_fpr_poisson": (ctypes.c_double, [ctypes.c_double]),
                "oracle_fpr_standard": (ctypes.c_double,
                                        [ctypes.c_double, ctypes.c_double]),
                "oracle_splitmix64_at": (u64, [u64, u64]),
                "oracle_splitmix64_fill": (None, [u64, u64, sz, P64]),
                "oracle_find_mt": (i32, [P32, u32, P64, sz, P32, i32]),
                "oracle_insert_mt": (i32, [P32, u32, P64, sz, i32]),
                "oracle_num_cores": (i32, []),
                "oracle_seed_k": (u32, [i32]),
                "oracle_insert_k": (i32, [P32, u32, i32, P64, sz]),
                "oracle_find_k": (i32, [P32, u32, i32, P64, sz, P32]),
                "oracle_fpr_poisson_k": (ctypes.c_double, [ctypes.c_double, i32]),
                "oracle_xxh64": (u64, [ctypes.c_void_p, sz, u64]),
                "oracle_xxh64_fixed": (None, [ctypes.c_void_p, sz, sz, u64, P64]),
                "oracle_xxh64_var": (None, [ctypes.c_void_p, P64, sz, u64, P64]),
                "oracle_swap_lane_pairs": (None, [P32, sz, P32]),
                "oracle_range_digest": (None, [P32, u64, u64, i32, u64, P64, P64, P64]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _c_u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a


def _c_u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


# ---- thin numpy wrappers -------------------------------------------------

def seeds() -> np.ndarray:
    out = np.zeros(8, np.uint32)
    lib().oracle_seeds(_u32p(out))
    return out


def block_index(h: int, num_blocks: int) -> int:
    return int(lib().oracle_block_index(h, num_blocks))


def make_mask(x: int) -> np.ndarray:
    out = np.zeros(8, np.uint32)
    lib().oracle_make_mask(x & 0xFFFFFFFF, _u32p(out))
    return out


def new_filter(num_blocks: int) -> np.ndarray:
    """An empty filter: num_blocks * 8 zero words."""
    return np.zeros(int(num_blocks) * 8, np.uint32)


def insert(words: np.ndarray, num_blocks: int, hashes) -> np.ndarray:
    h = _c_u64(hashes)
    assert words.dtype == np.uint32 and words.flags.c_contiguous
    assert words.size == 8 * num_blocks
    lib().oracle_insert(_u32p(words), num_blocks, _u64p(h), h.size)
    return words


def insert_block_range(sub_words, num_blocks, hashes, lo, hi):
    h = _c_u64(hashes)
    assert sub_words.dtype == np.uint32 and sub_words.size == 8 * (hi - lo)
    lib().oracle_insert_block_range(_u32p(sub_words), num_blocks, _u64p(h),
                                    h.size, lo, hi)
    return sub_words


def insert_block_ranges(out_words, num_blocks, hashes, lo, hi):
    """Blocks of sorted disjoint ranges [lo[r], hi[r]) after inserting hashes,
    ORed into out_words (the ranges' blocks one after another)."""
    h = _c_u64(hashes)
    lo_, hi_ = _c_u64(lo), _c_u64(hi)
    assert out_words.dtype == np.uint32 and out_words.size == 8 * int((hi_ - lo_).sum())
    lib().oracle_insert_block_ranges(_u32p(out_words), num_blocks, _u64p(h), h.size,
                                     _u64p(lo_), _u64p(hi_), lo_.size)
    return out_words


def find_one(words, num_blocks, h) -> bool:
    return bool(lib().oracle_find_one(_u32p(words), num_blocks, h))


def find(words: np.ndarray, num_blocks: int, hashes) -> np.ndarray:
    h = _c_u64(hashes)
    out = np.zeros((h.size + 31) // 32, np.uint32)
    lib().oracle_find(_u32p(words), num_blocks, _u64p(h), h.size, _u32p(out))
    return out


def union(dst: np.ndarray, src: np.ndarray) -> np.ndarray:
    assert dst.size == src.size
    s = _c_u32(src)
    lib().oracle_union(_u32p(dst), _u32p(s), dst.size)
    return dst


def multi_insert(arena, base_block, num_blocks, hashes, ids) -> int:
    h, t = _c_u64(hashes), _c_u32(ids)
    bb, nb = _c_u64(base_block), _c_u32(num_blocks)
    return int(lib().oracle_multi_insert(_u32p(arena), _u64p(bb), _u32p(nb),
                                         nb.size, _u64p(h), _u32p(t), h.size))


def multi_find(arena, base_block, num_blocks, hashes, ids):
    h, t = _c_u64(hashes), _c_u32(ids)
    bb, nb = _c_u64(base_block), _c_u32(num_blocks)
    out = np.zeros((h.size + 31) // 32, np.uint32)
    bad = lib().oracle_multi_find(_u32p(arena), _u64p(bb), _u32p(nb), nb.size,
                                  _u64p(h), _u32p(t), h.size, _u32p(out))
    return out, int(bad)


def fpr_poisson(a: float) -> float:
    return float(lib().oracle_fpr_poisson(a))


def fpr_standard(bits_per_key: float, k: float) -> float:
    return float(lib().oracle_fpr_standard(bits_per_key, k))


def splitmix64_at(seed: int, i: int) -> int:
    return int(lib().oracle_splitmix64_at(seed, i))


def splitmix64_fill(seed: int, start: int, n: int) -> np.ndarray:
    out = np.empty(n, np.uint64)
    lib().oracle_splitmix64_fill(seed, start, n, _u64p(out))
    return out


def find_mt(words, num_blocks, hashes, n_threads):
    h = _c_u64(hashes)
    out = np.zeros((h.size + 31) // 32, np.uint32)
    used = lib().oracle_find_mt(_u32p(words), num_blocks, _u64p(h), h.size,
                                _u32p(out), n_threads)
    return out, int(used)


def insert_mt(words, num_blocks, hashes, n_threads) -> int:
    h = _c_u64(hashes)
    return int(lib().oracle_insert_mt(_u32p(words), num_blocks, _u64p(h),
                                      h.size, n_threads))


def num_cores() -> int:
    return int(lib().oracle_num_cores())


# ---- lane-count variants, key hashing, Parquet layout ----------------------

def seed_k(i: int) -> int:
    return int(lib().oracle_seed_k(i))


def insert_k(words: np.ndarray, num_blocks: int, k: int, hashes) -> np.ndarray:
    h = _c_u64(hashes)
    assert words.dtype == np.uint32 and words.flags.c_contiguous
    assert words.size == k * num_blocks
    if lib().oracle_insert_k(_u32p(words), num_blocks, k, _u64p(h), h.size) != 0:
        raise ValueError("lanes must be 4, 8 or 16")
    return words


def find_k(words: np.ndarray, num_blocks: int, k: int, hashes) -> np.ndarray:
    h = _c_u64(hashes)
    assert words.size == k * num_blocks
    out = np.zeros((h.size + 31) // 32, np.uint32)
    if lib().oracle_find_k(_u32p(words), num_blocks, k, _u64p(h), h.size, _u32p(out)) != 0:
        raise ValueError("lanes must be 4, 8 or 16")
    return out


def fpr_poisson_k(a: float, k: int) -> float:
    return float(lib().oracle_fpr_poisson_k(a, k))


def xxh64(data: bytes, seed: int = 0) -> int:
    buf = ctypes.create_string_buffer(bytes(data), max(len(data), 1))
    return int(lib().oracle_xxh64(buf, len(data), seed))


def xxh64_fixed(keys: np.ndarray, seed: int = 0) -> np.ndarray:
    """XXH64 of each element's little-endian bytes (keys: a 1-D integer array)."""
    a = np.ascontiguousarray(keys)
    a = a.astype(a.dtype.newbyteorder("<"), copy=False)
    out = np.empty(a.size, np.uint64)
    lib().oracle_xxh64_fixed(a.ctypes.data_as(ctypes.c_void_p), a.dtype.itemsize, a.size,
                             seed, _u64p(out))
    return out


def xxh64_var(data: np.ndarray, offsets: np.ndarray, seed: int = 0) -> np.ndarray:
    """XXH64 of data[offsets[k]:offsets[k+1]] for each k."""
    d = np.ascontiguousarray(data, dtype=np.uint8)
    o = _c_u64(offsets)
    n = o.size - 1
    out = np.empty(max(n, 0), np.uint64)
    if d.size == 0:
        d = np.zeros(1, np.uint8)
    lib().oracle_xxh64_var(d.ctypes.data_as(ctypes.c_void_p), _u64p(o), n, seed, _u64p(out))
    return out


def swap_lane_pairs(words: np.ndarray) -> np.ndarray:
    """Appendix lane order <-> Parquet's salt order (word w <-> word w ^ 1)."""
    w = _c_u32(words)
    assert w.size % 2 == 0
    out = np.empty_like(w)
    lib().oracle_swap_lane_pairs(_u32p(w), w.size, _u32p(out))
    return out


def range_digest(words: np.ndarray, lanes: int, range_blocks: int, threads: int = 1):
    """Per block range: (digest, set bits, blocks with both a zero and a
    non-zero lane), each a uint64 array of ceil(num_blocks / range_blocks).
    With threads > 1 the ranges are split into that many runs of whole ranges,
    each computed by the same scalar C code on its own thread."""
    w = _c_u32(words)
    assert lanes in (4, 8, 16) and w.size % lanes == 0 and range_blocks >= 1
    nb = w.size // lanes
    n_ranges = -(-nb // range_blocks)
    d = np.zeros(n_ranges, np.uint64)
    b = np.zeros(n_ranges, np.uint64)
    p = np.zeros(n_ranges, np.uint64)
    runs = max(1, min(threads, n_ranges))
    cuts = [n_ranges * k // runs for k in range(runs + 1)]

    def run(k):
        r0, r1 = cuts[k], cuts[k + 1]
        b0, b1 = r0 * range_blocks, min(nb, r1 * range_blocks)
        if r1 > r0:
            lib().oracle_range_digest(_u32p(w[b0 * lanes:]), b0, b1 - b0, lanes, range_blocks,
                                      _u64p(d[r0:]), _u64p(b[r0:]), _u64p(p[r0:]))

    if runs == 1:
        run(0)
    else:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(runs) as ex:
            list(ex.map(run, range(runs)))
    return d, b, p
