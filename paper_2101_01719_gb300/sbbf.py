"""Thin Python binding of ``libsbbf.so`` (ctypes).

Argument marshalling only: every step of insert, lookup and union runs in the
library's CUDA kernels.  PyTorch supplies device memory (filters created here
are backed by a torch tensor and wrapped with ``sbbf_wrap``) and streams
(``torch.cuda.current_stream()`` unless a stream is passed).  There is no CPU
fallback: if the library is missing or fails to load, every call raises.

Tensors passed in must be CUDA tensors on the filter's device; a tensor used on
a stream other than the one it was allocated on must be kept alive by the
caller (``Tensor.record_stream``) until the work completes.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsbbf.so")

SBBF_OK, SBBF_EINVAL, SBBF_ENOMEM, SBBF_ECUDA, SBBF_EBUSY, SBBF_ETIMEOUT, SBBF_ERANGE = range(7)

_lib = None
_lock = threading.Lock()

_c = ctypes
_P = _c.c_void_p
_u32, _u64, _sz, _int = _c.c_uint32, _c.c_uint64, _c.c_size_t, _c.c_int

# name -> (restype, argtypes); every symbol declared in include/sbbf.h.
SIGNATURES = {
    "sbbf_status_string": (_c.c_char_p, [_int]),
    "sbbf_last_cuda_error": (_int, []),
    "sbbf_version": (_u32, []),
    "sbbf_create": (_int, [_u32, _c.POINTER(_P)]),
    "sbbf_wrap": (_int, [_P, _u32, _c.POINTER(_P)]),
    "sbbf_create_lanes": (_int, [_u32, _u32, _c.POINTER(_P)]),
    "sbbf_wrap_lanes": (_int, [_P, _u32, _u32, _c.POINTER(_P)]),
    "sbbf_lanes": (_u32, [_P]),
    "sbbf_serialized_size": (_sz, [_P]),
    "sbbf_serialize": (_int, [_P, _P, _sz, _P]),
    "sbbf_deserialize": (_int, [_P, _sz, _c.POINTER(_P)]),
    "sbbf_parquet_header": (_int, [_u64, _P, _sz, _c.POINTER(_sz)]),
    "sbbf_parquet_parse_header": (_int, [_P, _sz, _c.POINTER(_u64), _c.POINTER(_sz)]),
    "sbbf_parquet_size": (_sz, [_P]),
    "sbbf_export_parquet": (_int, [_P, _P, _sz, _c.POINTER(_sz), _P]),
    "sbbf_import_parquet": (_int, [_P, _sz, _c.POINTER(_P), _c.POINTER(_sz)]),
    "sbbf_create_from_host": (_int, [_P, _u32, _c.POINTER(_P)]),
    "sbbf_destroy": (_int, [_P]),
    "sbbf_num_blocks": (_u32, [_P]),
    "sbbf_device_words": (_int, [_P, _c.POINTER(_P), _c.POINTER(_sz)]),
    "sbbf_clear": (_int, [_P, _P]),
    "sbbf_insert_hashes": (_int, [_P, _P, _sz, _P]),
    "sbbf_set_partitioning": (_int, [_P, _int]),
    "sbbf_partition_applies": (_int, [_P, _sz, _int, _P]),
    "sbbf_device_status": (_int, [_P, _P]),
    "sbbf_record_device_status": (_int, [_P, _u32, _P]),
    "sbbf_find_hashes": (_int, [_P, _P, _sz, _P, _P]),
    "sbbf_union": (_int, [_P, _P, _P]),
    "sbbf_copy_to_host": (_int, [_P, _P, _sz, _P]),
    "sbbf_host_pipe_create": (_int, [_sz, _c.POINTER(_P)]),
    "sbbf_host_pipe_destroy": (_int, [_P]),
    "sbbf_host_pipe_set_mode": (_int, [_P, _int]),
    "sbbf_insert_hashes_host": (_int, [_P, _P, _P, _sz, _P]),
    "sbbf_find_hashes_host": (_int, [_P, _P, _P, _sz, _P, _P]),
    "sbbf_hash_keys": (_int, [_P, _u32, _sz, _u64, _P, _P]),
    "sbbf_hash_bytes": (_int, [_P, _P, _sz, _u64, _P, _P]),
    "sbbf_insert_keys": (_int, [_P, _P, _u32, _sz, _u64, _P]),
    "sbbf_find_keys": (_int, [_P, _P, _u32, _sz, _u64, _P, _P]),
    "sbbf_insert_bytes": (_int, [_P, _P, _P, _sz, _u64, _P]),
    "sbbf_find_bytes": (_int, [_P, _P, _P, _sz, _u64, _P, _P]),
    "sbbf_fill_splitmix64": (_int, [_P, _sz, _u64, _u64, _P]),
    "sbbf_fill_queries": (_int, [_P, _sz, _u64, _u64, _u64, _u64, _u64, _u64, _u64, _P]),
    "sbbf_count_bits": (_int, [_P, _sz, _P, _P]),
    "sbbf_region_passes": (_int, [_P, _sz, _int, _c.POINTER(_u32)]),
    "sbbf_range_digest": (_int, [_P, _u64, _u32, _u64, _P, _P, _P, _P]),
    "sbbf_fill_segment_queries": (_int, [_P, _sz, _P, _P, _u32, _u64, _u64, _u64, _u64, _P]),
    "sbbf_fill_segment_ids": (_int, [_P, _sz, _P, _u32, _P]),
    "sbbf_multi_create": (_int, [_P, _u32, _c.POINTER(_P)]),
    "sbbf_multi_destroy": (_int, [_P]),
    "sbbf_multi_num_filters": (_u32, [_P]),
    "sbbf_multi_filter_info": (_int, [_P, _u32, _c.POINTER(_u64), _c.POINTER(_u32)]),
    "sbbf_multi_device_words": (_int, [_P, _c.POINTER(_P), _c.POINTER(_sz)]),
    "sbbf_multi_clear": (_int, [_P, _P]),
    "sbbf_multi_copy_to_host": (_int, [_P, _P, _sz, _P]),
    "sbbf_multi_insert": (_int, [_P, _P, _P, _sz, _P]),
    "sbbf_multi_find": (_int, [_P, _P, _P, _sz, _P, _P]),
    "sbbf_multi_insert_segments": (_int, [_P, _P, _P, _sz, _P]),
    "sbbf_multi_find_segments": (_int, [_P, _P, _P, _sz, _P, _P]),
    "sbbf_multi_insert_each": (_int, [_P, _P, _P, _P]),
    "sbbf_multi_find_each": (_int, [_P, _P, _P, _P, _P]),
    "sbbf_multi_invalid_count": (_int, [_P, _c.POINTER(_u64), _P]),
    "sbbf_multi_get_tuning": (_int, [_P, _int, _int, _c.POINTER(_int), _c.POINTER(_int),
                                     _c.POINTER(_int), _c.POINTER(_int)]),
    "sbbf_multi_set_tuning": (_int, [_P, _int, _int, _int, _int, _int, _int]),
    "sbbf_multi_tune": (_int, [_P, _int, _int, _P, _P, _sz, _P, _c.POINTER(_c.c_float)]),
    "sbbf_multi_graph_create": (_int, [_P, _c.POINTER(_P)]),
    "sbbf_multi_graph_destroy": (_int, [_P]),
    "sbbf_multi_graph_launch": (_int, [_P, _P, _P, _sz, _P, _P, _sz, _P, _P]),
    "sbbf_multi_find_noalloc": (_int, [_P, _P, _u32, _P, _P, _sz, _P, _P, _P]),
    "sbbf_server_create": (_int, [_P, _c.POINTER(_P)]),
    "sbbf_server_destroy": (_int, [_P]),
    "sbbf_server_add_filter": (_int, [_P, _u32, _c.POINTER(_u32)]),
    "sbbf_server_submit": (_int, [_P, _P, _c.POINTER(_u64)]),
    "sbbf_server_poll": (_int, [_P, _u64, _c.POINTER(_int)]),
    "sbbf_server_wait": (_int, [_P, _u64, _u64]),
    "sbbf_server_drain": (_int, [_P, _u64]),
    "sbbf_server_prefill": (_int, [_P, _u32, _P, _sz]),
    "sbbf_server_copy_filter": (_int, [_P, _u32, _P, _sz]),
    "sbbf_server_stats": (_int, [_P, _P]),
    "sbbf_server_replay": (_int, [_P, _P, _P, _sz, _P]),
    "sbbf_server_replay_serial": (_int, [_P, _P, _P, _sz, _P]),
    "sbbf_shard_range": (_int, [_u32, _u32, _u32, _c.POINTER(_u32), _c.POINTER(_u32)]),
    "sbbf_shard_routed_capacity": (_sz, [_sz, _u32, _int]),
    "sbbf_shard_route_scratch_bytes": (_sz, [_sz, _u32]),
    "sbbf_shard_route": (_int, [_P, _sz, _u32, _u32, _int, _P, _P, _P, _P, _sz, _P]),
    "sbbf_shard_insert": (_int, [_P, _u32, _u32, _P, _sz, _P]),
    "sbbf_shard_find": (_int, [_P, _u32, _u32, _P, _sz, _P, _P]),
    "sbbf_shard_unpermute": (_int, [_P, _P, _sz, _sz, _P, _P]),
}

OP_INSERT, OP_FIND = 0, 1
FORM_SEGMENTS, FORM_TAGGED = 0, 1
PARTITION_AUTO, PARTITION_OFF, PARTITION_ON, PARTITION_REGIONS = 0, 1, 2, 3
PIPE_AUTO, PIPE_COPY, PIPE_DIRECT = 0, 1, 2


class SbbfError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = "%s failed: %s" % (what, lib().sbbf_status_string(status).decode())
        if status == SBBF_ECUDA:
            msg += " (cudaError %d)" % lib().sbbf_last_cuda_error()
        super().__init__(msg)


def lib():
    """The loaded ``libsbbf.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    "libsbbf.so is not built (%s); run paper_2101_01719_gb300.build.build()"
                    % LIB_PATH)
            L = _c.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str) -> None:
    if status != SBBF_OK:
        raise SbbfError(status, what)


def stream_handle(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _hashes_ptr(t: torch.Tensor, device) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("hashes must be a CUDA tensor")
    if t.dtype not in (torch.int64, torch.uint64):
        raise TypeError("hashes must be int64 or uint64 (64-bit hash values)")
    if not t.is_contiguous():
        raise ValueError("hashes must be contiguous")
    if device is not None and t.device != device:
        raise ValueError("hashes are on %s, filter on %s" % (t.device, device))
    return t.data_ptr()


_KEY_DTYPES = (torch.int32, torch.int64) + tuple(
    getattr(torch, n) for n in ("uint32", "uint64") if hasattr(torch, n))


def _keys_arg(t: torch.Tensor, device):
    """(pointer, key_bytes) of a fixed-width key tensor (4- or 8-byte ints)."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("keys must be a CUDA tensor")
    if t.dtype not in _KEY_DTYPES:
        raise TypeError("keys must be 32- or 64-bit integers")
    if not t.is_contiguous():
        raise ValueError("keys must be contiguous")
    if device is not None and t.device != device:
        raise ValueError("keys are on %s, filter on %s" % (t.device, device))
    return t.data_ptr(), t.element_size()


def _bytes_args(data: torch.Tensor, offsets: torch.Tensor, device):
    """(data pointer, offsets pointer, n) of byte-string keys: key k is
    data[offsets[k]:offsets[k+1]] (data uint8, offsets int64 of n + 1)."""
    for name, t in (("data", data), ("offsets", offsets)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise TypeError("%s must be a contiguous CUDA tensor" % name)
        if device is not None and t.device != device:
            raise ValueError("%s is on %s, filter on %s" % (name, t.device, device))
    if data.dtype != torch.uint8:
        raise TypeError("data must be uint8")
    if offsets.dtype != torch.int64 or offsets.dim() != 1 or offsets.numel() < 1:
        raise TypeError("offsets must be a 1-D int64 tensor of n + 1 entries")
    if data.numel() == 0:  # all keys empty: any readable address will do
        data = torch.zeros(8, dtype=torch.uint8, device=offsets.device)
    return data.data_ptr(), offsets.data_ptr(), offsets.numel() - 1, data


def hash_keys(keys: torch.Tensor, seed: int = 0, out: torch.Tensor | None = None, stream=None):
    """XXH64 of each fixed-width key (its little-endian bytes) on the device."""
    ptr, kb = _keys_arg(keys, None)
    n = keys.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=keys.device)
    with torch.cuda.device(keys.device):
        check(lib().sbbf_hash_keys(ptr, kb, n, seed, out.data_ptr(), stream_handle(stream)),
              "sbbf_hash_keys")
    return out


def hash_bytes(data: torch.Tensor, offsets: torch.Tensor, seed: int = 0,
               out: torch.Tensor | None = None, stream=None):
    """XXH64 of each byte string data[offsets[k]:offsets[k+1]] on the device."""
    dp, op, n, _keep = _bytes_args(data, offsets, None)
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=offsets.device)
    with torch.cuda.device(offsets.device):
        check(lib().sbbf_hash_bytes(dp, op, n, seed, out.data_ptr(), stream_handle(stream)),
              "sbbf_hash_bytes")
    return out


def out_words(n: int) -> int:
    """Words of packed lookup output for n hashes."""
    return (n + 31) // 32


def _host_bytes(buf):
    import numpy as np
    a = np.frombuffer(buf, dtype=np.uint8) if isinstance(buf, (bytes, bytearray, memoryview)) \
        else np.ascontiguousarray(buf, dtype=np.uint8)
    return a


def parquet_header(num_bytes: int) -> bytes:
    """Thrift BloomFilterHeader of a Parquet bitset of num_bytes bytes (host)."""
    n = _sz()
    check(lib().sbbf_parquet_header(num_bytes, None, 0, _c.byref(n)), "sbbf_parquet_header")
    out = (_c.c_uint8 * n.value)()
    check(lib().sbbf_parquet_header(num_bytes, out, n.value, _c.byref(n)), "sbbf_parquet_header")
    return bytes(out)


def parse_parquet_header(buf):
    """(bitset bytes, header length) of a Parquet Bloom filter (host)."""
    a = _host_bytes(buf)
    nb, hl = _u64(), _sz()
    check(lib().sbbf_parquet_parse_header(a.ctypes.data, a.size, _c.byref(nb), _c.byref(hl)),
          "sbbf_parquet_parse_header")
    return int(nb.value), int(hl.value)


class _DeviceWords:
    """__cuda_array_interface__ over a library-owned filter's words."""

    def __init__(self, ptr, n_words):
        self.__cuda_array_interface__ = {"shape": (n_words,), "typestr": "<i4",
                                         "data": (ptr, False), "version": 3}


class Filter:
    """A split block Bloom filter of ``num_blocks`` blocks of ``lanes`` 32-bit
    words (8, the paper's; 4 or 16) whose words live in a torch tensor
    (``self.words``, int32, ``num_blocks * lanes``)."""

    def __init__(self, num_blocks: int, device=None, words: torch.Tensor | None = None,
                 lanes: int = 8):
        if num_blocks <= 0 or num_blocks >= 2**32:
            raise ValueError("num_blocks must be in [1, 2^32)")
        if lanes not in (4, 8, 16):
            raise ValueError("lanes must be 4, 8 or 16")
        if words is None:
            dev = (torch.device("cuda", torch.cuda.current_device()) if device is None
                   else torch.device(device))
            words = torch.zeros(num_blocks * lanes, dtype=torch.int32, device=dev)
        if words.numel() != num_blocks * lanes or not words.is_cuda or not words.is_contiguous():
            raise ValueError("words must be a contiguous CUDA tensor of num_blocks*lanes int32")
        self.words = words
        self.num_blocks = int(num_blocks)
        self.lanes = int(lanes)
        self.device = words.device
        h = _P()
        with torch.cuda.device(self.device):
            check(lib().sbbf_wrap_lanes(words.data_ptr(), num_blocks, lanes, _c.byref(h)),
                  "sbbf_wrap_lanes")
        self._h = h

    @classmethod
    def _adopt(cls, h):
        """A torch-backed copy of a library-owned filter handle (destroyed)."""
        try:
            lanes, nb = lib().sbbf_lanes(h), lib().sbbf_num_blocks(h)
            ptr, nbytes = _P(), _sz()
            check(lib().sbbf_device_words(h, _c.byref(ptr), _c.byref(nbytes)), "sbbf_device_words")
            dev = torch.device("cuda", torch.cuda.current_device())
            words = torch.as_tensor(_DeviceWords(ptr.value, nbytes.value // 4), device=dev).clone()
            torch.cuda.synchronize(dev)
        finally:
            lib().sbbf_destroy(h)
        return cls(nb, words=words, lanes=lanes)

    def serialize(self, stream=None):
        """The filter in the native checkpoint format (numpy uint8)."""
        import numpy as np
        n = lib().sbbf_serialized_size(self._h)
        out = np.empty(n, np.uint8)
        with torch.cuda.device(self.device):
            check(lib().sbbf_serialize(self._h, out.ctypes.data, n, stream_handle(stream)),
                  "sbbf_serialize")
        return out

    @classmethod
    def deserialize(cls, buf) -> "Filter":
        a = _host_bytes(buf)
        h = _P()
        check(lib().sbbf_deserialize(a.ctypes.data, a.size, _c.byref(h)), "sbbf_deserialize")
        return cls._adopt(h)

    def export_parquet(self, stream=None):
        """Header and bitset in Parquet's Bloom-filter format (numpy uint8)."""
        import numpy as np
        n = lib().sbbf_parquet_size(self._h)
        if n == 0:
            raise ValueError("Parquet filters have 8 lanes and fewer than 2^31 bytes")
        out = np.empty(n, np.uint8)
        w = _sz()
        with torch.cuda.device(self.device):
            check(lib().sbbf_export_parquet(self._h, out.ctypes.data, n, _c.byref(w),
                                            stream_handle(stream)), "sbbf_export_parquet")
        return out[:w.value]

    @classmethod
    def import_parquet(cls, buf):
        """(Filter, bytes consumed) from a Parquet Bloom filter."""
        a = _host_bytes(buf)
        h, used = _P(), _sz()
        check(lib().sbbf_import_parquet(a.ctypes.data, a.size, _c.byref(h), _c.byref(used)),
              "sbbf_import_parquet")
        return cls._adopt(h), int(used.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.sbbf_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def clear(self, stream=None):
        with torch.cuda.device(self.device):
            check(lib().sbbf_clear(self._h, stream_handle(stream)), "sbbf_clear")
        return self

    def set_partitioning(self, mode: int):
        """PARTITION_AUTO / PARTITION_OFF / PARTITION_ON / PARTITION_REGIONS (see sbbf.h)."""
        check(lib().sbbf_set_partitioning(self._h, mode), "sbbf_set_partitioning")
        return self

    def partition_applies(self, n: int, lookup: bool = False) -> bool:
        """Whether a batch of n hashes (inserts, or lookups) takes the
        partitioned path under the current mode."""
        v = _c.c_int(0)
        check(lib().sbbf_partition_applies(self._h, n, 1 if lookup else 0, _c.byref(v)),
              "sbbf_partition_applies")
        return bool(v.value)

    def region_passes(self, n: int, lookup: bool = True) -> int:
        """Region passes a lookup (or an insert) of n hashes takes (1: a
        single pass)."""
        p = _u32()
        check(lib().sbbf_region_passes(self._h, n, 1 if lookup else 0, _c.byref(p)),
              "sbbf_region_passes")
        return int(p.value)

    def device_status(self, stream=None) -> int:
        """sbbf_device_status: OK, or ETIMEOUT when a device-side wait of a
        partitioned call ran out since the last query (synchronises the
        stream; reading clears the status)."""
        with torch.cuda.device(self.device):
            st = int(lib().sbbf_device_status(self._h, stream_handle(stream)))
        if st not in (SBBF_OK, SBBF_ETIMEOUT):
            check(st, "sbbf_device_status")
        return st

    def record_device_status(self, bits: int, stream=None):
        """sbbf_record_device_status (testing the reporting path)."""
        with torch.cuda.device(self.device):
            check(lib().sbbf_record_device_status(self._h, bits, stream_handle(stream)),
                  "sbbf_record_device_status")
        return self

    def insert(self, hashes: torch.Tensor, stream=None):
        ptr = _hashes_ptr(hashes, self.device)
        with torch.cuda.device(self.device):
            check(lib().sbbf_insert_hashes(self._h, ptr, hashes.numel(), stream_handle(stream)),
                  "sbbf_insert_hashes")
        return self

    def find(self, hashes: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        n = hashes.numel()
        ptr = _hashes_ptr(hashes, self.device)
        if out is None:
            out = torch.empty(out_words(n), dtype=torch.int32, device=self.device)
        elif out.numel() < out_words(n) or not out.is_cuda or out.element_size() != 4:
            raise ValueError("out must be a CUDA int32 tensor of (n+31)//32 words")
        with torch.cuda.device(self.device):
            check(lib().sbbf_find_hashes(self._h, ptr, n, out.data_ptr(), stream_handle(stream)),
                  "sbbf_find_hashes")
        return out

    def _out(self, n, out):
        if out is None:
            return torch.empty(out_words(n), dtype=torch.int32, device=self.device)
        if out.numel() < out_words(n) or not out.is_cuda or out.element_size() != 4:
            raise ValueError("out must be a CUDA int32 tensor of (n+31)//32 words")
        return out

    def insert_keys(self, keys: torch.Tensor, seed: int = 0, stream=None):
        """Insert fixed-width keys, hashed with XXH64 inside the insert kernel."""
        ptr, kb = _keys_arg(keys, self.device)
        with torch.cuda.device(self.device):
            check(lib().sbbf_insert_keys(self._h, ptr, kb, keys.numel(), seed,
                                         stream_handle(stream)), "sbbf_insert_keys")
        return self

    def find_keys(self, keys: torch.Tensor, seed: int = 0, out: torch.Tensor | None = None,
                  stream=None):
        ptr, kb = _keys_arg(keys, self.device)
        n = keys.numel()
        out = self._out(n, out)
        with torch.cuda.device(self.device):
            check(lib().sbbf_find_keys(self._h, ptr, kb, n, seed, out.data_ptr(),
                                       stream_handle(stream)), "sbbf_find_keys")
        return out

    def insert_bytes(self, data: torch.Tensor, offsets: torch.Tensor, seed: int = 0,
                     stream=None):
        """Insert byte-string keys data[offsets[k]:offsets[k+1]] (XXH64 in-kernel)."""
        dp, op, n, _keep = _bytes_args(data, offsets, self.device)
        with torch.cuda.device(self.device):
            check(lib().sbbf_insert_bytes(self._h, dp, op, n, seed, stream_handle(stream)),
                  "sbbf_insert_bytes")
        return self

    def find_bytes(self, data: torch.Tensor, offsets: torch.Tensor, seed: int = 0,
                   out: torch.Tensor | None = None, stream=None):
        dp, op, n, _keep = _bytes_args(data, offsets, self.device)
        out = self._out(n, out)
        with torch.cuda.device(self.device):
            check(lib().sbbf_find_bytes(self._h, dp, op, n, seed, out.data_ptr(),
                                        stream_handle(stream)), "sbbf_find_bytes")
        return out

    def union_(self, other: "Filter", stream=None):
        with torch.cuda.device(self.device):
            check(lib().sbbf_union(self._h, other._h, stream_handle(stream)), "sbbf_union")
        return self

    def to_numpy(self):
        import numpy as np
        return self.words.cpu().numpy().view(np.uint32)

    def range_digest(self, range_blocks: int, stream=None):
        """Verification digest of this filter's words per range of
        ``range_blocks`` blocks (see :func:`range_digest`)."""
        return range_digest(self.words, self.lanes, range_blocks, stream)


class HostPipe:
    """Staging buffers and streams for host-memory insert/lookup calls."""

    def __init__(self, chunk_hashes: int = 1 << 24, mode: int = PIPE_AUTO):
        h = _P()
        check(lib().sbbf_host_pipe_create(chunk_hashes, _c.byref(h)), "sbbf_host_pipe_create")
        self._h = h
        self.chunk = chunk_hashes
        self.set_mode(mode)

    def set_mode(self, mode: int):
        """PIPE_AUTO / PIPE_COPY / PIPE_DIRECT (see sbbf.h)."""
        check(lib().sbbf_host_pipe_set_mode(self._h, mode), "sbbf_host_pipe_set_mode")
        self.mode = mode
        return self

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.sbbf_host_pipe_destroy(h)
            self._h = None

    def insert(self, f: Filter, h_hashes: torch.Tensor, stream=None):
        assert not h_hashes.is_cuda and h_hashes.is_contiguous() and h_hashes.element_size() == 8
        with torch.cuda.device(f.device):
            check(lib().sbbf_insert_hashes_host(f.handle, self._h, h_hashes.data_ptr(),
                                                h_hashes.numel(), stream_handle(stream)),
                  "sbbf_insert_hashes_host")

    def find(self, f: Filter, h_hashes: torch.Tensor, h_out: torch.Tensor, stream=None):
        assert not h_hashes.is_cuda and h_hashes.is_contiguous() and h_hashes.element_size() == 8
        assert not h_out.is_cuda and h_out.numel() >= out_words(h_hashes.numel())
        with torch.cuda.device(f.device):
            check(lib().sbbf_find_hashes_host(f.handle, self._h, h_hashes.data_ptr(),
                                              h_hashes.numel(), h_out.data_ptr(),
                                              stream_handle(stream)),
                  "sbbf_find_hashes_host")
        return h_out


# ---- synthetic inputs ------------------------------------------------------

def fill_splitmix64(out: torch.Tensor, seed: int, start: int = 0, stream=None):
    """out[k] = splitmix64 output (start + k) of `seed` (int64 view of the bits)."""
    assert out.is_cuda and out.element_size() == 8 and out.is_contiguous()
    check(lib().sbbf_fill_splitmix64(out.data_ptr(), out.numel(), seed & (2**64 - 1),
                                     start, stream_handle(stream)), "sbbf_fill_splitmix64")
    return out


def fill_queries(out: torch.Tensor, start: int, ins_seed: int, ins_start: int, n_inserted: int,
                 fresh_seed: int, member_seed: int, member_threshold: int, stream=None):
    assert out.is_cuda and out.element_size() == 8 and out.is_contiguous()
    check(lib().sbbf_fill_queries(out.data_ptr(), out.numel(), start, ins_seed, ins_start,
                                  n_inserted, fresh_seed, member_seed, member_threshold,
                                  stream_handle(stream)), "sbbf_fill_queries")
    return out


def count_bits(bits: torch.Tensor, n: int, stream=None) -> torch.Tensor:
    """Device count of set bits among the first n bits of a packed result."""
    cnt = torch.empty(1, dtype=torch.int64, device=bits.device)
    check(lib().sbbf_count_bits(bits.data_ptr(), n, cnt.data_ptr(), stream_handle(stream)),
          "sbbf_count_bits")
    return cnt


def range_digest(words: torch.Tensor, lanes: int, range_blocks: int, stream=None):
    """Per block range of a device word array (``lanes`` words per block):
    (digest, set bits, blocks with both a zero and a non-zero lane), three
    int64 tensors on the device holding the uint64 values bit for bit."""
    if not words.is_cuda or not words.is_contiguous() or words.element_size() != 4:
        raise ValueError("words must be a contiguous CUDA tensor of 32-bit words")
    if lanes not in (4, 8, 16) or words.numel() % lanes or range_blocks < 1:
        raise ValueError("lanes must be 4, 8 or 16 and divide the words; range_blocks >= 1")
    nb = words.numel() // lanes
    n_ranges = -(-nb // range_blocks)
    out = torch.empty(3, n_ranges, dtype=torch.int64, device=words.device)
    with torch.cuda.device(words.device):
        check(lib().sbbf_range_digest(words.data_ptr(), nb, lanes, range_blocks, out[0].data_ptr(),
                                      out[1].data_ptr(), out[2].data_ptr(), stream_handle(stream)),
              "sbbf_range_digest")
    return out[0], out[1], out[2]


def fill_segment_queries(out: torch.Tensor, q_offsets: torch.Tensor, ins_offsets: torch.Tensor,
                         ins_seed: int, fresh_seed: int, member_seed: int,
                         member_threshold: int, stream=None):
    """Query streams of several filters in the segment layout (see sbbf.h)."""
    assert out.is_cuda and out.element_size() == 8 and q_offsets.dtype == torch.int64
    n_filters = q_offsets.numel() - 1
    check(lib().sbbf_fill_segment_queries(out.data_ptr(), out.numel(), q_offsets.data_ptr(),
                                          ins_offsets.data_ptr(), n_filters, ins_seed, fresh_seed,
                                          member_seed, member_threshold, stream_handle(stream)),
          "sbbf_fill_segment_queries")
    return out


def fill_segment_ids(out: torch.Tensor, offsets: torch.Tensor, stream=None):
    """out[k] = filter of key k under the segment offsets (uint32 as int32)."""
    assert out.is_cuda and out.element_size() == 4 and offsets.dtype == torch.int64
    check(lib().sbbf_fill_segment_ids(out.data_ptr(), out.numel(), offsets.data_ptr(),
                                      offsets.numel() - 1, stream_handle(stream)),
          "sbbf_fill_segment_ids")
    return out


class MultiFilter:
    """Many filters of uneven size in one library-owned device arena.

    Keys reach filters by per-key ids (``ids=``, int32 tensor) or grouped per
    filter by offsets (``offsets=``, int64 CUDA tensor of n_filters + 1)."""

    def __init__(self, num_blocks, device=None):
        import numpy as np
        nb = np.ascontiguousarray(num_blocks, dtype=np.uint32)
        if nb.ndim != 1 or nb.size == 0 or (nb == 0).any():
            raise ValueError("num_blocks must be a non-empty list of sizes >= 1")
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.num_blocks = nb
        self.base = np.concatenate([[0], np.cumsum(nb.astype(np.uint64))[:-1]]).astype(np.uint64)
        h = _P()
        with torch.cuda.device(self.device):
            check(lib().sbbf_multi_create(nb.ctypes.data, nb.size, _c.byref(h)),
                  "sbbf_multi_create")
        self._h = h
        self._graph = None

    def __del__(self):
        g = getattr(self, "_graph", None)
        if g and _lib is not None:
            _lib.sbbf_multi_graph_destroy(g)
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.sbbf_multi_destroy(h)
            self._h = None

    @property
    def n_filters(self) -> int:
        return int(self.num_blocks.size)

    @property
    def total_blocks(self) -> int:
        return int(self.num_blocks.astype("uint64").sum())

    def _ctx(self):
        return torch.cuda.device(self.device)

    def clear(self, stream=None):
        with self._ctx():
            check(lib().sbbf_multi_clear(self._h, stream_handle(stream)), "sbbf_multi_clear")
        return self

    def to_numpy(self, stream=None):
        import numpy as np
        out = np.empty(self.total_blocks * 8, np.uint32)
        with self._ctx():
            check(lib().sbbf_multi_copy_to_host(self._h, out.ctypes.data, out.nbytes,
                                                stream_handle(stream)), "sbbf_multi_copy_to_host")
        return out

    def filter_words(self, arena, t: int):
        b = int(self.base[t])
        return arena[8 * b: 8 * (b + int(self.num_blocks[t]))]

    def insert(self, hashes, ids=None, offsets=None, stream=None):
        ptr = _hashes_ptr(hashes, self.device)
        n = hashes.numel()
        with self._ctx():
            if offsets is not None:
                check(lib().sbbf_multi_insert_segments(self._h, ptr, offsets.data_ptr(), n,
                                                       stream_handle(stream)),
                      "sbbf_multi_insert_segments")
            else:
                check(lib().sbbf_multi_insert(self._h, ptr, ids.data_ptr(), n,
                                              stream_handle(stream)), "sbbf_multi_insert")
        return self

    def find(self, hashes, ids=None, offsets=None, out=None, stream=None):
        ptr = _hashes_ptr(hashes, self.device)
        n = hashes.numel()
        if out is None:
            out = torch.empty(out_words(n), dtype=torch.int32, device=self.device)
        with self._ctx():
            if offsets is not None:
                check(lib().sbbf_multi_find_segments(self._h, ptr, offsets.data_ptr(), n,
                                                     out.data_ptr(), stream_handle(stream)),
                      "sbbf_multi_find_segments")
            else:
                check(lib().sbbf_multi_find(self._h, ptr, ids.data_ptr(), n, out.data_ptr(),
                                            stream_handle(stream)), "sbbf_multi_find")
        return out

    def insert_each(self, hashes, h_offsets, stream=None):
        import numpy as np
        ho = np.ascontiguousarray(h_offsets, dtype=np.uint64)
        with self._ctx():
            check(lib().sbbf_multi_insert_each(self._h, _hashes_ptr(hashes, self.device),
                                               ho.ctypes.data, stream_handle(stream)),
                  "sbbf_multi_insert_each")
        return self

    def find_each(self, hashes, h_offsets, out=None, stream=None):
        import numpy as np
        ho = np.ascontiguousarray(h_offsets, dtype=np.uint64)
        n = hashes.numel()
        if out is None:
            out = torch.empty(out_words(n), dtype=torch.int32, device=self.device)
        with self._ctx():
            check(lib().sbbf_multi_find_each(self._h, _hashes_ptr(hashes, self.device),
                                             ho.ctypes.data, out.data_ptr(),
                                             stream_handle(stream)), "sbbf_multi_find_each")
        return out

    def invalid_count(self, stream=None) -> int:
        v = _u64()
        with self._ctx():
            check(lib().sbbf_multi_invalid_count(self._h, _c.byref(v), stream_handle(stream)),
                  "sbbf_multi_invalid_count")
        return int(v.value)

    def get_tuning(self, op: int, form: int):
        t, l, u, b = _int(), _int(), _int(), _int()
        check(lib().sbbf_multi_get_tuning(self._h, op, form, _c.byref(t), _c.byref(l),
                                          _c.byref(u), _c.byref(b)), "sbbf_multi_get_tuning")
        return {"threads": t.value, "lanes": l.value, "unroll": u.value, "l1_bypass": b.value}

    def set_tuning(self, op: int, form: int, threads: int, lanes: int, unroll: int,
                   l1_bypass: int = 0):
        check(lib().sbbf_multi_set_tuning(self._h, op, form, threads, lanes, unroll, l1_bypass),
              "sbbf_multi_set_tuning")

    def tune(self, op: int, hashes, ids=None, offsets=None, stream=None) -> float:
        """Autotune the launch shape for (op, form) on a prefix of this batch."""
        form = FORM_SEGMENTS if offsets is not None else FORM_TAGGED
        aux = offsets if offsets is not None else ids
        ms = _c.c_float()
        with self._ctx():
            check(lib().sbbf_multi_tune(self._h, op, form, _hashes_ptr(hashes, self.device),
                                        aux.data_ptr(), hashes.numel(), stream_handle(stream),
                                        _c.byref(ms)), "sbbf_multi_tune")
        return float(ms.value)

    def graph_launch(self, ins, ins_offsets, q, q_offsets, out, stream=None):
        """Inserts then lookups of one batch as one CUDA graph launch."""
        if self._graph is None:
            g = _P()
            with self._ctx():
                check(lib().sbbf_multi_graph_create(self._h, _c.byref(g)),
                      "sbbf_multi_graph_create")
            self._graph = g
        n_i = 0 if ins is None else ins.numel()
        n_q = 0 if q is None else q.numel()
        with self._ctx():
            check(lib().sbbf_multi_graph_launch(
                self._graph, ins.data_ptr() if n_i else None,
                ins_offsets.data_ptr() if n_i else None, n_i,
                q.data_ptr() if n_q else None, q_offsets.data_ptr() if n_q else None, n_q,
                out.data_ptr() if n_q else None, stream_handle(stream)),
                "sbbf_multi_graph_launch")
        return out


# ---- serving -------------------------------------------------------------------

class _ServerConfig(_c.Structure):
    _fields_ = [("budget_bytes", _u64), ("max_window_requests", _u32),
                ("max_inflight_windows", _u32), ("max_window_keys", _u64),
                ("max_pending_requests", _u64)]


class _Request(_c.Structure):
    _fields_ = [("op", _u32), ("filter", _u32), ("n", _u64), ("d_hashes", _P),
                ("d_out_bits", _P)]


class _Stats(_c.Structure):
    _fields_ = [(k, _u64) for k in ("windows", "launches", "phases", "requests", "keys",
                                    "admissions", "evictions", "writebacks",
                                    "admission_waits",
                                    "resident_bytes")]


# numpy layout of sbbf_request_t (32 bytes)
REQUEST_DTYPE = [("op", "<u4"), ("filter", "<u4"), ("n", "<u8"), ("hashes", "<u8"),
                 ("out", "<u8")]


class Server:
    """Continuous-batching server over resident filters (see sbbf.h)."""

    def __init__(self, budget_bytes: int, max_window_requests: int = 4096,
                 max_inflight_windows: int = 2, max_window_keys: int = 1 << 26,
                 max_pending_requests: int = 1 << 24, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        cfg = _ServerConfig(budget_bytes, max_window_requests, max_inflight_windows,
                            max_window_keys, max_pending_requests)
        h = _P()
        with torch.cuda.device(self.device):
            check(lib().sbbf_server_create(_c.byref(cfg), _c.byref(h)), "sbbf_server_create")
        self._h = h
        self.num_blocks = []

    def close(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            self._h = None
            check(_lib.sbbf_server_destroy(h), "sbbf_server_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_filter(self, num_blocks: int) -> int:
        fid = _u32()
        check(lib().sbbf_server_add_filter(self._h, num_blocks, _c.byref(fid)),
              "sbbf_server_add_filter")
        self.num_blocks.append(int(num_blocks))
        return int(fid.value)

    def prefill(self, fid: int, hashes: torch.Tensor):
        with torch.cuda.device(self.device):
            check(lib().sbbf_server_prefill(self._h, fid, _hashes_ptr(hashes, None),
                                            hashes.numel()), "sbbf_server_prefill")

    def submit(self, op: int, fid: int, hashes, out=None) -> int:
        r = _Request(op, fid, hashes.numel(), hashes.data_ptr(),
                     out.data_ptr() if out is not None else None)
        t = _u64()
        check(lib().sbbf_server_submit(self._h, _c.byref(r), _c.byref(t)), "sbbf_server_submit")
        return int(t.value)

    def poll(self, ticket: int) -> bool:
        d = _int()
        check(lib().sbbf_server_poll(self._h, ticket, _c.byref(d)), "sbbf_server_poll")
        return bool(d.value)

    def wait(self, ticket: int, timeout_ns: int = 0):
        check(lib().sbbf_server_wait(self._h, ticket, timeout_ns), "sbbf_server_wait")

    def wait_status(self, ticket: int, timeout_ns: int = 0) -> int:
        return int(lib().sbbf_server_wait(self._h, ticket, timeout_ns))

    def drain(self, timeout_ns: int = 0):
        check(lib().sbbf_server_drain(self._h, timeout_ns), "sbbf_server_drain")

    def filter_words(self, fid: int):
        import numpy as np
        out = np.empty(self.num_blocks[fid] * 8, np.uint32)
        check(lib().sbbf_server_copy_filter(self._h, fid, out.ctypes.data, out.nbytes),
              "sbbf_server_copy_filter")
        return out

    def stats(self) -> dict:
        st = _Stats()
        check(lib().sbbf_server_stats(self._h, _c.byref(st)), "sbbf_server_stats")
        return {k: int(getattr(st, k)) for k, _ in _Stats._fields_}

    def replay(self, reqs, arrival_ns, serial: bool = False):
        """Submit a numpy array of REQUEST_DTYPE records at arrival_ns (uint64,
        from the call's start) and return per-request latencies in ns."""
        import numpy as np
        reqs = np.ascontiguousarray(reqs)
        arr = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
        lat = np.zeros(len(reqs), np.uint64)
        fn = lib().sbbf_server_replay_serial if serial else lib().sbbf_server_replay
        with torch.cuda.device(self.device):
            check(fn(self._h, reqs.ctypes.data, arr.ctypes.data, len(reqs), lat.ctypes.data),
                  "sbbf_server_replay_serial" if serial else "sbbf_server_replay")
        return lat


# ---- one filter sharded by block range (see sbbf.h) ------------------------------

def shard_range(num_blocks: int, n_shards: int, shard: int):
    """(lo, hi): the global blocks shard `shard` of n_shards owns."""
    lo, hi = _u32(), _u32()
    check(lib().sbbf_shard_range(num_blocks, n_shards, shard, _c.byref(lo), _c.byref(hi)),
          "sbbf_shard_range")
    return int(lo.value), int(hi.value)


def shard_route(hashes: torch.Tensor, num_blocks: int, n_shards: int, pad: bool, stream=None):
    """sbbf_shard_route: (routed hashes, their query indexes, per-shard counts),
    device tensors (int64, int32, int64); the counts stay on the device."""
    n = hashes.numel()
    dev = hashes.device
    cap = int(lib().sbbf_shard_routed_capacity(n, n_shards, 1 if pad else 0))
    routed = torch.empty(cap, dtype=torch.int64, device=dev)
    perm = torch.empty(cap, dtype=torch.int32, device=dev)
    counts = torch.empty(n_shards, dtype=torch.int64, device=dev)
    sb = int(lib().sbbf_shard_route_scratch_bytes(n, n_shards))
    scratch = torch.empty((sb + 7) // 8, dtype=torch.int64, device=dev)
    with torch.cuda.device(dev):
        check(lib().sbbf_shard_route(_hashes_ptr(hashes, dev) if n else None, n, num_blocks,
                                     n_shards, 1 if pad else 0, routed.data_ptr(),
                                     perm.data_ptr(), counts.data_ptr(), scratch.data_ptr(),
                                     scratch.numel() * 8, stream_handle(stream)),
              "sbbf_shard_route")
    return routed, perm, counts


def shard_insert(f: "Filter", num_blocks: int, lo: int, hashes: torch.Tensor, stream=None):
    with torch.cuda.device(f.device):
        check(lib().sbbf_shard_insert(f.handle, num_blocks, lo,
                                      _hashes_ptr(hashes, f.device) if hashes.numel() else None,
                                      hashes.numel(), stream_handle(stream)), "sbbf_shard_insert")


def shard_find(f: "Filter", num_blocks: int, lo: int, hashes: torch.Tensor, out=None,
               stream=None) -> torch.Tensor:
    n = hashes.numel()
    if out is None:
        out = torch.empty(out_words(n), dtype=torch.int32, device=f.device)
    with torch.cuda.device(f.device):
        check(lib().sbbf_shard_find(f.handle, num_blocks, lo,
                                    _hashes_ptr(hashes, f.device) if n else None, n,
                                    out.data_ptr() if n else None, stream_handle(stream)),
              "sbbf_shard_find")
    return out


def shard_unpermute(routed_bits: torch.Tensor, perm: torch.Tensor, n_routed: int, n: int,
                    out=None, stream=None) -> torch.Tensor:
    dev = perm.device
    if out is None:
        out = torch.empty(out_words(n), dtype=torch.int32, device=dev)
    with torch.cuda.device(dev):
        check(lib().sbbf_shard_unpermute(routed_bits.data_ptr() if n_routed else None,
                                         perm.data_ptr() if n_routed else None, n_routed, n,
                                         out.data_ptr() if n else None, stream_handle(stream)),
              "sbbf_shard_unpermute")
    return out
