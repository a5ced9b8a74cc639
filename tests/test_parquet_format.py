"""Parquet's Bloom-filter header as the library writes and parses it (host-only
entry points; no GPU).  Apache Arrow's Parquet writer (pyarrow, where
installed) is the independent reference: the library's header must equal the
bytes it writes, and the library must parse its files."""
import os
import tempfile

import numpy as np
import pytest

import sbbf_inputs as inp


@pytest.fixture(scope="module")
def sb():
    from paper_2101_01719_gb300 import build
    build.build()
    import paper_2101_01719_gb300 as sb
    return sb


def _arrow_filter_bytes(ndv, fpp):
    pa = pytest.importorskip("pyarrow")
    pq = pytest.importorskip("pyarrow.parquet")
    vals = inp.stream(8, 5, ndv).view(np.int64)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "t.parquet")
        pq.write_table(pa.table({"c": pa.array(vals, type=pa.int64())}), path,
                       bloom_filter_options={"c": {"ndv": ndv, "fpp": fpp}})
        cc = pq.ParquetFile(path).metadata.row_group(0).column(0)
        raw = open(path, "rb").read()[cc.bloom_filter_offset:
                                      cc.bloom_filter_offset + cc.bloom_filter_length]
    return raw


@pytest.mark.parametrize("ndv,fpp", [(10, 0.1), (1000, 0.01), (200_000, 0.001)])
def test_header_bytes_match_arrow(sb, ndv, fpp):
    raw = _arrow_filter_bytes(ndv, fpp)
    num_bytes, hlen = sb.parse_parquet_header(raw)
    assert hlen + num_bytes == len(raw)
    assert sb.parquet_header(num_bytes) == raw[:hlen]


@pytest.mark.parametrize("num_bytes", [32, 64, 2048, 1 << 20, (1 << 31) - 32])
def test_header_round_trip(sb, num_bytes):
    h = sb.parquet_header(num_bytes)
    assert sb.parse_parquet_header(h + b"\0" * 7) == (num_bytes, len(h))


def test_header_rejects(sb):
    good = sb.parquet_header(4096)
    for bad in (b"", good[:1], good[:-1],              # truncated
                good.replace(b"\x1c\x1c\x00\x00", b"\x1c\x2c\x00\x00", 1),  # algorithm member 2
                bytes([0x15, 0xC8, 0x01]) + good[3:],                      # 100 bytes: not x32
                bytes([0x15, 0x01]) + good[3:]):                            # negative size
        with pytest.raises(sb.SbbfError):
            sb.parse_parquet_header(bad)
    for n in (0, 16, 33, 1 << 31):
        with pytest.raises(sb.SbbfError):
            sb.parquet_header(n)


def test_header_skips_unknown_fields(sb):
    """A field the library does not know (here field 5: a binary, then a list
    of i32) is skipped; nesting deeper than the parser allows is an error."""
    good = sb.parquet_header(64)
    extra = bytes([0x18, 0x03]) + b"abc" + bytes([0x19, 0x35, 0x02, 0x04, 0x06])
    assert sb.parse_parquet_header(good[:-1] + extra + b"\0") == (64, len(good) + len(extra))
    deep = good[:-1] + bytes([0x1c]) * 40 + b"\0" * 41
    with pytest.raises(sb.SbbfError):
        sb.parse_parquet_header(deep)
