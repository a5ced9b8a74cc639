"""GB300 (sm_103a) split block Bloom filters: batched insert and lookup of
64-bit hash values, or of raw keys hashed on the device (Apple, "Split block
Bloom filters", arXiv 2101.01719).

The compute runs in ``libsbbf.so`` (hand-written CUDA behind the C ABI in
``include/sbbf.h``); this package is its thin Python binding.
"""
from .sbbf import (  # noqa: F401
    FORM_SEGMENTS,
    FORM_TAGGED,
    OP_FIND,
    OP_INSERT,
    PARTITION_AUTO,
    PARTITION_OFF,
    PARTITION_ON,
    PARTITION_REGIONS,
    PIPE_AUTO,
    PIPE_COPY,
    PIPE_DIRECT,
    Filter,
    HostPipe,
    MultiFilter,
    REQUEST_DTYPE,
    Server,
    SbbfError,
    check,
    count_bits,
    fill_queries,
    fill_segment_ids,
    fill_segment_queries,
    fill_splitmix64,
    hash_bytes,
    hash_keys,
    lib,
    out_words,
    parquet_header,
    parse_parquet_header,
    stream_handle,
)
