"""The native input generator produces exactly the numpy generator's streams
(which tests/test_oracle.py pins to the published splitmix64 outputs)."""
import numpy as np

import sbbf_inputs as inp


def test_native_splitmix64_equals_numpy():
    for seed, start, n in ((1234567, 0, 10), (0, 0, 1000), (inp.stream_seed(3, 1), 12345, 300_001)):
        for threads in (1, 3, 16):
            assert np.array_equal(inp.fast_splitmix64(seed, start, n, threads),
                                  inp.splitmix64(seed, start, n))


def test_native_workload_queries_equal_numpy():
    for cfg, n_ins, frac, prefix, start, n in ((2, 100_000_000, 0.1, 0, 0, 200_000),
                                              (1, 1_000_000, 0.5, 0, 777_777, 150_001),
                                              (0, 100_000, 0.0, 100_000, 0, 1_100_000),
                                              (0, 100_000, 0.0, 100_000, 99_990, 20),
                                              (5, 1, 1.0, 0, 0, 1000)):
        for threads in (1, 7):
            assert np.array_equal(
                inp.fast_workload_queries(cfg, n_ins, frac, prefix, start, n, threads),
                inp.workload_queries(cfg, n_ins, frac, prefix, start, n)), (cfg, threads)


def test_native_segment_queries_equal_numpy():
    n_keys = np.array([1000, 0, 5, 200_000, 1, 64, 3000], np.int64)
    ins_off, q_off = inp.multi_offsets(n_keys, 4)
    for t0, t1 in ((0, 7), (1, 4), (3, 4), (6, 7)):
        for threads in (1, 5, 16):
            got = inp.fast_segment_queries(9, ins_off, q_off, 0.5, t0, t1, threads)
            exp = np.concatenate([inp.segment_queries(9, ins_off, q_off, 0.5, t)
                                  for t in range(t0, t1)])
            assert np.array_equal(got, exp), (t0, t1, threads)
