"""GPU parity of keys hashed on the device (XXH64, the step before the
method): the hash arrays, and the filters and lookup bits of the fused
insert/lookup kernels, against the oracle's XXH64 and filter, bit for bit.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2101_01719_gb300 as sb
from paper_2101_01719_gb300 import sbbf as abi
import sbbf_inputs as inp
from gpu_util import bits_np, dev, to_dev, u64_np

pytestmark = pytest.mark.gpu


def _keys32(n, role):
    return (inp.stream(140, role, n) >> np.uint64(32)).astype(np.uint32)


def _dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).to(dev())


def _strings(n, role, max_len=200):
    lens = (inp.stream(141, role, n) % np.uint64(max_len + 1)).astype(np.uint64)
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    data = (inp.stream(141, role + 10, int(offsets[-1])) & np.uint64(0xFF)).astype(np.uint8)
    return data, offsets


def _oracle_filter(B, hashes):
    f = oracle.new_filter(B)
    oracle.insert(f, B, hashes)
    return f


@pytest.mark.parametrize("n,seed", [(1, 0), (63, 0), (100_003, 0), (100_003, 0xDEADBEEF12345)])
def test_hash_keys_u64(n, seed):
    keys = inp.stream(140, 0, n)
    got = u64_np(sb.hash_keys(to_dev(keys), seed=seed))
    assert np.array_equal(got, oracle.xxh64_fixed(keys, seed))


@pytest.mark.parametrize("offset", [0, 1])
def test_hash_keys_u32(offset):
    """offset 1: a 4-byte but not 8-byte aligned array takes the scalar path."""
    n = 70_001
    keys = _keys32(n + offset, 1)
    got = u64_np(sb.hash_keys(_dev32(keys)[offset:], seed=7))
    assert np.array_equal(got, oracle.xxh64_fixed(keys[offset:], 7))


@pytest.mark.parametrize("start", [0, 3, 5])
def test_hash_bytes_unaligned(start):
    """Byte strings of 0..200 bytes (every stripe and tail path) at data
    addresses with every alignment."""
    data, offsets = _strings(20_001, 2)
    buf = np.concatenate([np.zeros(start, np.uint8), data])
    d = torch.from_numpy(buf).to(dev())[start:]
    o = torch.from_numpy(offsets.view(np.int64)).to(dev())
    got = u64_np(sb.hash_bytes(d, o, seed=11))
    assert np.array_equal(got, oracle.xxh64_var(data, offsets, 11))


@pytest.mark.parametrize("B,n", [(1, 5), (4096, 100_000), (32768, 1_000_001), (1_000_003, 333_333)])
def test_fused_u64_insert_find(B, n):
    keys = inp.stream(142, B % 1000, n)
    q = np.concatenate([inp.stream(142, 999, 2 * n + 31), keys[: n // 3]])
    f = sb.Filter(B)
    f.insert_keys(to_dev(keys))
    bits = f.find_keys(to_dev(q))
    ref = _oracle_filter(B, oracle.xxh64_fixed(keys))
    assert np.array_equal(f.to_numpy(), ref)
    assert np.array_equal(bits_np(bits), oracle.find(ref, B, oracle.xxh64_fixed(q)))


def test_fused_u32_insert_find_with_seed():
    B, n, seed = 20_011, 500_001, 123456789
    keys = _keys32(n, 3)
    q = np.concatenate([_keys32(n, 4), keys[:1000]])
    f = sb.Filter(B)
    f.insert_keys(_dev32(keys), seed=seed)
    bits = f.find_keys(_dev32(q), seed=seed)
    ref = _oracle_filter(B, oracle.xxh64_fixed(keys, seed))
    assert np.array_equal(f.to_numpy(), ref)
    assert np.array_equal(bits_np(bits), oracle.find(ref, B, oracle.xxh64_fixed(q, seed)))


def test_fused_equals_hash_then_insert():
    B, n = 9_999, 200_000
    keys = to_dev(inp.stream(143, 0, n))
    a, b = sb.Filter(B), sb.Filter(B)
    a.insert_keys(keys, seed=5)
    b.insert(sb.hash_keys(keys, seed=5))
    assert torch.equal(a.words, b.words)


def test_fused_bytes_insert_find():
    B = 4096
    data, offsets = _strings(30_000, 5)
    qdata, qoff = _strings(40_000, 6, max_len=40)
    f = sb.Filter(B)
    f.insert_bytes(torch.from_numpy(data).to(dev()), torch.from_numpy(offsets.view(np.int64)).to(dev()))
    bits = f.find_bytes(torch.from_numpy(qdata).to(dev()), torch.from_numpy(qoff.view(np.int64)).to(dev()))
    ref = _oracle_filter(B, oracle.xxh64_var(data, offsets))
    assert np.array_equal(f.to_numpy(), ref)
    assert np.array_equal(bits_np(bits), oracle.find(ref, B, oracle.xxh64_var(qdata, qoff)))


def test_all_empty_strings():
    offsets = np.zeros(101, np.uint64)
    o = torch.from_numpy(offsets.view(np.int64)).to(dev())
    got = u64_np(sb.hash_bytes(torch.zeros(0, dtype=torch.uint8, device=dev()), o))
    assert np.all(got == oracle.xxh64(b""))


@pytest.mark.parametrize("op", ["insert", "find"])
def test_fused_partitioned_path(op):
    """A filter forced onto the partitioned path hashes into its scratch
    first; results are the oracle's."""
    B, n = 1 << 21, 3_000_000
    keys = inp.stream(144, 0, n)
    f = sb.Filter(B).set_partitioning(abi.PARTITION_ON)
    ref = _oracle_filter(B, oracle.xxh64_fixed(keys))
    if op == "insert":
        f.insert_keys(to_dev(keys))
        assert np.array_equal(f.to_numpy(), ref)
    else:
        g = sb.Filter(B).set_partitioning(abi.PARTITION_OFF)
        g.insert_keys(to_dev(keys))
        f.words.copy_(g.words)
        q = np.concatenate([inp.stream(144, 1, n), keys[:n // 2]])
        bits = f.find_keys(to_dev(q))
        assert np.array_equal(bits_np(bits), oracle.find(ref, B, oracle.xxh64_fixed(q)))


def test_key_arguments_rejected():
    L = abi.lib()
    f = sb.Filter(64)
    buf = torch.zeros(16, dtype=torch.int64, device=dev())
    s = abi.stream_handle()
    # key_bytes must be 4 or 8; 8-byte keys must be 8-byte aligned
    assert L.sbbf_insert_keys(f.handle, buf.data_ptr(), 2, 4, 0, s) == abi.SBBF_EINVAL
    assert L.sbbf_insert_keys(f.handle, buf.data_ptr() + 4, 8, 4, 0, s) == abi.SBBF_EINVAL
    assert L.sbbf_find_keys(f.handle, buf.data_ptr(), 8, 4, 0, None, s) == abi.SBBF_EINVAL
    assert L.sbbf_hash_bytes(buf.data_ptr(), buf.data_ptr() + 4, 1, 0, buf.data_ptr(), s) == abi.SBBF_EINVAL
    assert L.sbbf_insert_keys(f.handle, None, 8, 0, 0, s) == abi.SBBF_OK  # n == 0
    torch.cuda.synchronize()


@pytest.mark.parametrize("width", [8, 4])
def test_fused_keys_by_region_passes(width):
    """Raw 8- and 4-byte keys looked up by region passes (forced, and in
    automatic mode on a 128 MiB filter with 8Mi keys or more): each pass
    hashes its keys again; the answers equal the oracle's on the XXH64
    hashes and the single-pass lookup's; byte strings take no region pass."""
    B = 2**22
    n = 1_000_003
    if width == 8:
        keys, q = inp.stream(145, 0, n), inp.stream(145, 1, 3 * n)
        dk, dq = to_dev(keys), to_dev(np.concatenate([q, keys[: n // 2]]))
        hq = oracle.xxh64_fixed(np.concatenate([q, keys[: n // 2]]), 9)
        hk = oracle.xxh64_fixed(keys, 9)
    else:
        keys, q = _keys32(n, 7), _keys32(3 * n, 8)
        qq = np.concatenate([q, keys[: n // 2]])
        dk, dq = _dev32(keys), _dev32(qq)
        hq, hk = oracle.xxh64_fixed(qq, 9), oracle.xxh64_fixed(keys, 9)
    f = sb.Filter(B)
    f.insert_keys(dk, seed=9)
    ref = _oracle_filter(B, hk)
    assert np.array_equal(f.to_numpy(), ref)
    f.set_partitioning(abi.PARTITION_REGIONS)
    got = bits_np(f.find_keys(dq, seed=9))
    assert np.array_equal(got, oracle.find(ref, B, hq))
    f.set_partitioning(abi.PARTITION_OFF)
    assert np.array_equal(bits_np(f.find_keys(dq, seed=9)), got)
    f.set_partitioning(abi.PARTITION_AUTO)
    assert f.region_passes(2**23) == 2
    big = torch.cat([dq] * (2**23 // dq.numel() + 1))[: 2**23]
    auto = bits_np(f.find_keys(big, seed=9))
    f.set_partitioning(abi.PARTITION_OFF)
    assert np.array_equal(auto, bits_np(f.find_keys(big, seed=9)))
