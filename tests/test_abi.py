"""The C-ABI library builds for sm_103a, loads, and exports every entry point
its headers declare.  No compute calls here: these run without a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for m in re.finditer(r"\b(sbbf_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2101_01719_gb300 import build
    return build.build()


def test_headers_declare_entry_points():
    names = _declared()
    for core in ("sbbf_create", "sbbf_destroy", "sbbf_insert_hashes", "sbbf_find_hashes",
                 "sbbf_union"):
        assert core in names


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True,
                         text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert _declared() <= exported


def test_binding_covers_every_symbol(built):
    from paper_2101_01719_gb300 import sbbf
    assert set(sbbf.SIGNATURES) == _declared()
    L = sbbf.lib()
    assert L.sbbf_version() >> 16 == 1
    assert L.sbbf_status_string(0) == b"SBBF_OK"
    assert b"EINVAL" in L.sbbf_status_string(1)


def test_argument_checks_need_no_gpu(built):
    """Invalid arguments are rejected on the host before any CUDA call."""
    from paper_2101_01719_gb300 import sbbf
    L = sbbf.lib()
    P = ctypes.c_void_p
    h = P()
    assert L.sbbf_create(0, ctypes.byref(h)) == sbbf.SBBF_EINVAL
    assert L.sbbf_wrap(None, 10, ctypes.byref(h)) == sbbf.SBBF_EINVAL
    assert L.sbbf_wrap(ctypes.c_void_p(0x1004), 10, ctypes.byref(h)) == sbbf.SBBF_EINVAL
    assert L.sbbf_insert_hashes(None, None, 0, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_find_hashes(None, None, 5, None, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_union(None, None, None) == sbbf.SBBF_EINVAL
    flag = ctypes.c_int(7)
    assert L.sbbf_partition_applies(None, 10, 0, ctypes.byref(flag)) == sbbf.SBBF_EINVAL
    assert flag.value == 7  # untouched on error
    assert L.sbbf_set_partitioning(None, 0) == sbbf.SBBF_EINVAL
    passes = ctypes.c_uint32(9)
    assert L.sbbf_region_passes(None, 10, 1, ctypes.byref(passes)) == sbbf.SBBF_EINVAL
    assert passes.value == 9  # untouched on error
    assert L.sbbf_device_status(None, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_record_device_status(None, 1, None) == sbbf.SBBF_EINVAL
    lo, hi = ctypes.c_uint32(7), ctypes.c_uint32(7)
    assert L.sbbf_shard_range(0, 2, 0, ctypes.byref(lo), ctypes.byref(hi)) == sbbf.SBBF_EINVAL
    assert L.sbbf_shard_range(10, 1025, 0, ctypes.byref(lo), ctypes.byref(hi)) == sbbf.SBBF_EINVAL
    assert lo.value == 7 and hi.value == 7  # untouched on error
    assert L.sbbf_shard_range(10, 3, 2, ctypes.byref(lo), ctypes.byref(hi)) == sbbf.SBBF_OK
    assert (lo.value, hi.value) == (8, 10)
    assert L.sbbf_shard_routed_capacity(100, 4, 1) == 100 + 31 * 4
    assert L.sbbf_shard_routed_capacity(100, 4, 0) == 100
    assert L.sbbf_shard_route(None, 5, 0, 2, 0, None, None, None, None, 0, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_shard_insert(None, 10, 0, None, 0, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_shard_find(None, 10, 0, None, 5, None, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_shard_unpermute(None, None, 5, 5, None, None) == sbbf.SBBF_EINVAL
    out = ctypes.c_void_p(0x2000)
    words = ctypes.c_void_p(0x3000)
    assert L.sbbf_range_digest(words, 10, 5, 4, out, out, out, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_range_digest(words, 10, 8, 0, out, out, out, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_range_digest(words, 10, 8, 4, None, out, out, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_range_digest(words, 2**40 + 1, 8, 4, out, out, out, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_range_digest(ctypes.c_void_p(0x3004), 10, 8, 4, out, out, out, None) \
        == sbbf.SBBF_EINVAL  # words not 16-byte aligned
    assert L.sbbf_range_digest(None, 10, 8, 4, out, out, out, None) == sbbf.SBBF_EINVAL
    assert L.sbbf_range_digest(None, 0, 8, 4, out, out, out, None) == sbbf.SBBF_OK  # nothing
    assert L.sbbf_destroy(None) == sbbf.SBBF_OK
    assert L.sbbf_num_blocks(None) == 0
    assert L.sbbf_host_pipe_create(100, ctypes.byref(h)) == sbbf.SBBF_EINVAL  # not /64
    assert L.sbbf_fill_queries(ctypes.c_void_p(0x1000), 10, 0, 1, 0, 0, 2, 3, 5, None) \
        == sbbf.SBBF_EINVAL  # members requested from an empty inserted set


def test_ptxas_reports_no_spills(built):
    reports = glob.glob(os.path.join(ROOT, "_build", "ptxas_*.txt"))
    assert reports
    for r in reports:
        text = open(r).read()
        for m in re.finditer(r"(\d+) bytes spill stores", text):
            assert int(m.group(1)) == 0, r


def test_product_path_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_2101_01719_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cc")):
            text = open(path).read()
            assert "import oracle" not in text and "sbbf_oracle" not in text, path
