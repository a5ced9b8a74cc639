"""Seeded synthetic inputs shared by the oracle-side and GPU-side tests.

This module holds no arithmetic of the filter itself.  It only produces
64-bit hash values (splitmix64, Steele/Lea/Flood 2014, in counter form) and
mixes them into query streams by the recipe below, so that the same bytes can
be handed to the CPU oracle and to the CUDA library.  The CUDA library and the
oracle each carry their own splitmix64 for sizes that cannot be materialised
on the host; tests pin all three against the published reference sequence.

Stream seeds: ``0x5BBF000000000000 | (cfg << 8) | role`` with roles
0 = inserted hashes, 1 = fresh lookup hashes, 2 = member selector,
3 = filter sizes, 4 = order / shuffles, 5 = arrivals, 6 = request sizes.

Query recipe (member fraction f): query j is a member when
``(r_j >> 32) < round(f * 2^32)`` with r_j the role-2 stream; a member is
``inserted[((r_j & 0xffffffff) * n_inserted) >> 32]``, otherwise the fresh
role-1 value j.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

ROLE_INSERT, ROLE_FRESH, ROLE_MEMBER, ROLE_SIZES, ROLE_ORDER = 0, 1, 2, 3, 4
ROLE_ARRIVAL, ROLE_REQSIZE = 5, 6


def stream_seed(cfg: int, role: int) -> int:
    return 0x5BBF000000000000 | (cfg << 8) | role


def splitmix64(seed: int, start: int, n: int) -> np.ndarray:
    """Outputs start..start+n-1 of the splitmix64 stream seeded with `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream(cfg: int, role: int, n: int, start: int = 0) -> np.ndarray:
    return splitmix64(stream_seed(cfg, role), start, n)


def member_threshold(frac: float) -> int:
    return int(round(frac * 2.0**32))


def queries(cfg: int, inserted: np.ndarray, n_queries: int, frac: float,
            start: int = 0) -> np.ndarray:
    """Query hashes start..start+n_queries-1 by the recipe in the docstring."""
    r = stream(cfg, ROLE_MEMBER, n_queries, start)
    fresh = stream(cfg, ROLE_FRESH, n_queries, start)
    thr = np.uint64(member_threshold(frac))
    member = (r >> np.uint64(32)) < thr
    with np.errstate(over="ignore"):
        idx = ((r & np.uint64(0xFFFFFFFF)) * np.uint64(len(inserted))) >> np.uint64(32)
    out = fresh.copy()
    out[member] = inserted[idx[member].astype(np.int64)]
    return out


def query_is_member(cfg: int, n_queries: int, frac: float, start: int = 0):
    r = stream(cfg, ROLE_MEMBER, n_queries, start)
    return (r >> np.uint64(32)) < np.uint64(member_threshold(frac))


def uniform01(cfg: int, role: int, n: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0,1) from the top 53 bits of a stream."""
    return (stream(cfg, role, n, start) >> np.uint64(11)).astype(np.float64) * 2.0**-53


def multi_filter_sizes(cfg: int, n_filters: int, lo: float, hi: float,
                       bits_per_key: float):
    """Key counts log-uniform in [lo, hi] (rounded) and blocks sized at
    bits_per_key, rounded up to whole 256-bit blocks."""
    u = uniform01(cfg, ROLE_SIZES, n_filters)
    n_keys = np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    blocks = np.ceil(n_keys * bits_per_key / 256.0).astype(np.int64)
    blocks = np.maximum(blocks, 1)
    return n_keys, blocks


def permutation(cfg: int, n: int, start: int = 0) -> np.ndarray:
    """A seeded permutation of 0..n-1 (argsort of a role-4 stream)."""
    return np.argsort(stream(cfg, ROLE_ORDER, n, start), kind="stable")


def workload_queries(cfg: int, n_inserted: int, frac: float, prefix: int, start: int,
                     n: int) -> np.ndarray:
    """Lookup hashes start..start+n-1 of a single-filter workload: indices
    below `prefix` are inserted hashes in order; the rest follow the query
    recipe indexed from `prefix`, members being inserted hash
    ((r & 0xffffffff) * n_inserted) >> 32 regenerated from the role-0 stream."""
    j = np.arange(start, start + n, dtype=np.int64)
    out = np.empty(n, np.uint64)
    pre = j < prefix
    if pre.any():
        out[pre] = stream(cfg, ROLE_INSERT, int(pre.sum()), int(j[pre][0]))
    rest = ~pre
    if rest.any():
        k0 = int(j[rest][0]) - prefix
        m = int(rest.sum())
        r = stream(cfg, ROLE_MEMBER, m, k0)
        fresh = stream(cfg, ROLE_FRESH, m, k0)
        member = (r >> np.uint64(32)) < np.uint64(member_threshold(frac))
        with np.errstate(over="ignore"):
            idx = ((r & np.uint64(0xFFFFFFFF)) * np.uint64(n_inserted)) >> np.uint64(32)
        vals = fresh.copy()
        if member.any():
            seed = np.uint64(stream_seed(cfg, ROLE_INSERT))
            vals[member] = _splitmix64_at(seed, idx[member])
        out[rest] = vals
    return out


def sampled_queries(cfg: int, n_inserted: int, frac: float, prefix: int,
                    idx: np.ndarray) -> np.ndarray:
    """Lookup hashes at arbitrary indices idx (same recipe as workload_queries)."""
    idx = np.asarray(idx, dtype=np.uint64)
    out = np.empty(idx.size, np.uint64)
    pre = idx < np.uint64(prefix)
    out[pre] = _splitmix64_at(np.uint64(stream_seed(cfg, ROLE_INSERT)), idx[pre])
    k = idx[~pre] - np.uint64(prefix)
    r = _splitmix64_at(np.uint64(stream_seed(cfg, ROLE_MEMBER)), k)
    fresh = _splitmix64_at(np.uint64(stream_seed(cfg, ROLE_FRESH)), k)
    member = (r >> np.uint64(32)) < np.uint64(member_threshold(frac))
    with np.errstate(over="ignore"):
        midx = ((r & np.uint64(0xFFFFFFFF)) * np.uint64(n_inserted)) >> np.uint64(32)
    vals = fresh
    vals[member] = _splitmix64_at(np.uint64(stream_seed(cfg, ROLE_INSERT)), midx[member])
    out[~pre] = vals
    return out


def _splitmix64_at(seed, i):
    """splitmix64 outputs at arbitrary indices i (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(i, np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def multi_offsets(n_keys: np.ndarray, lookup_factor: int):
    q = ((lookup_factor * n_keys + 63) // 64) * 64
    ins = np.concatenate([[0], np.cumsum(n_keys)]).astype(np.int64)
    qo = np.concatenate([[0], np.cumsum(q)]).astype(np.int64)
    return ins, qo


def segment_queries(cfg: int, ins_off: np.ndarray, q_off: np.ndarray, frac: float,
                    t: int) -> np.ndarray:
    """Lookups of filter t in the segment layout: query k (global index) is a
    member when (r_k >> 32) < threshold, namely inserted key
    ins_off[t] + (((r_k & 0xffffffff) * n_t) >> 32), else fresh output k."""
    k = np.arange(q_off[t], q_off[t + 1], dtype=np.uint64)
    r = _splitmix64_at(np.uint64(stream_seed(cfg, ROLE_MEMBER)), k)
    fresh = _splitmix64_at(np.uint64(stream_seed(cfg, ROLE_FRESH)), k)
    n_t = int(ins_off[t + 1] - ins_off[t])
    member = ((r >> np.uint64(32)) < np.uint64(member_threshold(frac))) & (n_t > 0)
    with np.errstate(over="ignore"):
        idx = np.uint64(ins_off[t]) + (((r & np.uint64(0xFFFFFFFF)) * np.uint64(n_t))
                                       >> np.uint64(32))
    out = fresh.copy()
    out[member] = _splitmix64_at(np.uint64(stream_seed(cfg, ROLE_INSERT)), idx[member])
    return out


# ---- native, threaded generation for billions of hashes ------------------------
#
# sbbf_inputs_native.c produces the same streams (pinned against the numpy
# functions above by tests/test_inputs_native.py); it is compiled with gcc on
# first use into tests/libsbbf_inputs.so.

import ctypes as _c
import os as _os
import subprocess as _sp
import threading as _th

_HERE = _os.path.dirname(_os.path.abspath(__file__))
_NSRC = _os.path.join(_HERE, "sbbf_inputs_native.c")
_NLIB = _os.path.join(_HERE, "libsbbf_inputs.so")
_nlib = None
_nlock = _th.Lock()


def _native():
    global _nlib
    with _nlock:
        if _nlib is None:
            if (not _os.path.exists(_NLIB)
                    or _os.path.getmtime(_NLIB) < _os.path.getmtime(_NSRC)):
                tmp = _NLIB + ".tmp.%d" % _os.getpid()
                _sp.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall", "-o", tmp,
                         _NSRC, "-lpthread"], check=True)
                _os.replace(tmp, _NLIB)
            L = _c.CDLL(_NLIB)
            u64, sz, i32, u32 = _c.c_uint64, _c.c_size_t, _c.c_int, _c.c_uint32
            P64 = _c.POINTER(_c.c_uint64)
            PI64 = _c.POINTER(_c.c_int64)
            L.sin_fill.argtypes = [u64, u64, sz, P64, i32]
            L.sin_fill.restype = i32
            L.sin_workload_queries.argtypes = [u64, u64, u64, u64, u64, u64, u64, sz, P64, i32]
            L.sin_workload_queries.restype = i32
            L.sin_segment_queries.argtypes = [u64, u64, u64, u64, PI64, PI64, u32, u32, P64, i32]
            L.sin_segment_queries.restype = i32
            _nlib = L
    return _nlib


def _threads(threads):
    return threads or (_os.cpu_count() or 1)


def _p64(a):
    return a.ctypes.data_as(_c.POINTER(_c.c_uint64))


def fast_splitmix64(seed: int, start: int, n: int, threads: int = 0) -> np.ndarray:
    """splitmix64(seed, start, n), generated natively on several threads."""
    out = np.empty(n, np.uint64)
    if n:
        _native().sin_fill(seed, start, n, _p64(out), _threads(threads))
    return out


def fast_stream(cfg: int, role: int, n: int, start: int = 0, threads: int = 0) -> np.ndarray:
    return fast_splitmix64(stream_seed(cfg, role), start, n, threads)


def fast_workload_queries(cfg: int, n_inserted: int, frac: float, prefix: int, start: int,
                          n: int, threads: int = 0) -> np.ndarray:
    """workload_queries(...), generated natively on several threads."""
    out = np.empty(n, np.uint64)
    if n:
        _native().sin_workload_queries(
            stream_seed(cfg, ROLE_INSERT), stream_seed(cfg, ROLE_FRESH),
            stream_seed(cfg, ROLE_MEMBER), member_threshold(frac), n_inserted, prefix, start, n,
            _p64(out), _threads(threads))
    return out


def fast_segment_queries(cfg: int, ins_off: np.ndarray, q_off: np.ndarray, frac: float,
                         t0: int, t1: int, threads: int = 0) -> np.ndarray:
    """Lookups of filters t0..t1-1 (segment_queries of each, concatenated)."""
    ins_off = np.ascontiguousarray(ins_off, np.int64)
    q_off = np.ascontiguousarray(q_off, np.int64)
    out = np.empty(int(q_off[t1] - q_off[t0]), np.uint64)
    if out.size:
        P = _c.POINTER(_c.c_int64)
        _native().sin_segment_queries(
            stream_seed(cfg, ROLE_INSERT), stream_seed(cfg, ROLE_FRESH),
            stream_seed(cfg, ROLE_MEMBER), member_threshold(frac),
            ins_off.ctypes.data_as(P), q_off.ctypes.data_as(P), t0, t1, _p64(out),
            _threads(threads))
    return out
