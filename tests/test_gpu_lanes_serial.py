"""GPU parity of the four- and sixteen-lane filters against the oracle's
k-lane functions, and of serialization: the native checkpoint format and
Parquet's Bloom-filter format (bitset in Parquet's lane order)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2101_01719_gb300 as sb
import sbbf_inputs as inp
from gpu_util import bits_np, dev, to_dev

pytestmark = pytest.mark.gpu


def _oracle_k(B, k, hashes):
    return oracle.insert_k(np.zeros(B * k, np.uint32), B, k, hashes)


@pytest.mark.parametrize("k", [4, 16])
@pytest.mark.parametrize("B,n", [(1, 3), (97, 10_001), (4096, 300_000), (1_000_003, 1_000_001)])
def test_lanes_insert_find_parity(k, B, n):
    keys = inp.stream(150 + k, B % 1000, n)
    q = np.concatenate([inp.stream(150 + k, 999, 2 * n + 5), keys[: n // 2]])
    f = sb.Filter(B, lanes=k)
    f.insert(to_dev(keys))
    bits = f.find(to_dev(q))
    ref = _oracle_k(B, k, keys)
    assert np.array_equal(f.to_numpy(), ref)
    assert np.array_equal(bits_np(bits), oracle.find_k(ref, B, k, q))


@pytest.mark.parametrize("k", [4, 16])
def test_lanes_fused_keys(k):
    B, n = 7_919, 200_003
    keys = inp.stream(152, k, n)
    f = sb.Filter(B, lanes=k)
    f.insert_keys(to_dev(keys), seed=3)
    q = np.concatenate([inp.stream(152, 50 + k, n), keys[:999]])
    bits = f.find_keys(to_dev(q), seed=3)
    ref = _oracle_k(B, k, oracle.xxh64_fixed(keys, 3))
    assert np.array_equal(f.to_numpy(), ref)
    assert np.array_equal(bits_np(bits), oracle.find_k(ref, B, k, oracle.xxh64_fixed(q, 3)))


def test_lanes_union_clear_and_host_pipe():
    B = 1_234
    a, b = inp.stream(153, 0, 50_000), inp.stream(153, 1, 60_000)
    fa, fb = sb.Filter(B, lanes=4), sb.Filter(B, lanes=4)
    fa.insert(to_dev(a))
    fb.insert(to_dev(b))
    fa.union_(fb)
    assert np.array_equal(fa.to_numpy(), _oracle_k(B, 4, np.concatenate([a, b])))
    with pytest.raises(sb.SbbfError):
        fa.union_(sb.Filter(B, lanes=16))  # lane counts differ
    fb.clear()
    torch.cuda.synchronize()
    assert not fb.words.any()
    f16 = sb.Filter(B, lanes=16)
    pipe = sb.HostPipe(1 << 14)
    ha = torch.from_numpy(a.view(np.int64)).pin_memory()
    pipe.insert(f16, ha)
    hq = torch.from_numpy(b.view(np.int64)).pin_memory()
    out = torch.zeros(sb.out_words(b.size), dtype=torch.int32).pin_memory()
    pipe.find(f16, hq, out)
    ref = _oracle_k(B, 16, a)
    assert np.array_equal(f16.to_numpy(), ref)
    assert np.array_equal(out.numpy().view(np.uint32), oracle.find_k(ref, B, 16, b))


def _le32(words):
    return np.asarray(words, np.uint32).astype("<u4").tobytes()


@pytest.mark.parametrize("k,B", [(8, 4096), (4, 999), (16, 33)])
def test_native_round_trip_and_header(k, B):
    keys = inp.stream(154, k, 5 * B)
    f = sb.Filter(B, lanes=k)
    f.insert(to_dev(keys))
    buf = f.serialize()
    payload = buf[64:].tobytes()
    assert buf.size == 64 + 4 * k * B
    assert bytes(buf[:4]) == b"SBBF"
    hdr = buf[:40].view("<u4")
    assert list(hdr[1:4]) == [1, k, B]
    seeds = _le32([oracle.seed_k(i) for i in range(k)])
    assert int(buf[16:24].view("<u8")[0]) == oracle.xxh64(seeds)  # layout digest
    assert int(buf[24:32].view("<u8")[0]) == 4 * k * B
    assert int(buf[32:40].view("<u8")[0]) == oracle.xxh64(payload)  # checksum
    assert not buf[40:64].any()
    assert np.array_equal(np.frombuffer(payload, "<u4"), _oracle_k(B, k, keys))
    g = sb.Filter.deserialize(buf)
    assert g.lanes == k and g.num_blocks == B
    assert torch.equal(g.words, f.words)


def test_native_rejects_corruption():
    f = sb.Filter(256)
    f.insert(to_dev(inp.stream(155, 0, 1000)))
    buf = f.serialize()
    for mutate in (lambda b: b.__setitem__(64 + 100, b[64 + 100] ^ 1),  # payload bit
                   lambda b: b.__setitem__(4, 2),                        # version
                   lambda b: b.__setitem__(16, b[16] ^ 1),               # layout digest
                   lambda b: b.__setitem__(50, 1)):                      # reserved byte
        bad = buf.copy()
        mutate(bad)
        with pytest.raises(sb.SbbfError):
            sb.Filter.deserialize(bad)
    with pytest.raises(sb.SbbfError):
        sb.Filter.deserialize(buf[:-1])


@pytest.mark.parametrize("B", [1, 64, 32768])
def test_parquet_export_is_oracle_filter_in_parquet_order(B):
    keys = inp.stream(156, 0, 20 * B)
    f = sb.Filter(B)
    f.insert_keys(to_dev(keys))  # XXH64 seed 0, as Parquet
    out = f.export_parquet()
    nbytes, hlen = sb.parse_parquet_header(out)
    assert nbytes == 32 * B and out.size == hlen + nbytes
    assert out[:hlen].tobytes() == sb.parquet_header(32 * B)
    ref = oracle.new_filter(B)
    oracle.insert(ref, B, oracle.xxh64_fixed(keys))
    assert np.array_equal(out[hlen:].view("<u4"), oracle.swap_lane_pairs(ref))


def test_parquet_import():
    B = 2048
    vals = inp.stream(157, 0, 30_000)
    ref = oracle.new_filter(B)
    oracle.insert(ref, B, oracle.xxh64_fixed(vals))
    blob = sb.parquet_header(32 * B) + oracle.swap_lane_pairs(ref).astype("<u4").tobytes()
    f, used = sb.Filter.import_parquet(blob + b"trailing")
    assert used == len(blob) and f.lanes == 8 and f.num_blocks == B
    assert np.array_equal(f.to_numpy(), ref)
    bits = bits_np(f.find_keys(to_dev(vals)))
    assert np.all(np.unpackbits(bits.view(np.uint8), bitorder="little")[:vals.size] == 1)
    with pytest.raises(ValueError):
        sb.Filter(16, lanes=4).export_parquet()
    with pytest.raises(sb.SbbfError):
        sb.Filter.import_parquet(blob[:-1])
