"""Helpers for GPU parity tests: move seeded host inputs to the device and
bring packed results back as uint32 numpy arrays."""
import numpy as np
import torch


def dev():
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    return torch.device("cuda", torch.cuda.current_device())


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64)).to(dev())


def bits_np(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def u64_np(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def bit_at(bits: np.ndarray, k) -> np.ndarray:
    k = np.asarray(k, dtype=np.int64)
    return (bits[k // 32] >> (k % 32).astype(np.uint32)) & 1


def compare_all_lookups(w, ref_words, q_dev, bits_dev, chunk=1 << 26):
    """Every lookup answer of single-filter workload w against the oracle,
    chunk by chunk: the oracle's queries come from the host generator (and
    must equal the device-generated ones the GPU looked up), its answers from
    its multithreaded find over ref_words."""
    import oracle
    import sbbf_inputs as inp

    threads = oracle.num_cores()
    n = w.n_lookup
    assert chunk % 32 == 0
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        qh = inp.fast_workload_queries(w.cfg, w.n_insert, w.member_frac, w.member_prefix, s, m)
        assert np.array_equal(u64_np(q_dev[s:s + m]), qh), "queries %d.." % s
        exp, _ = oracle.find_mt(ref_words, w.num_blocks, qh, threads)
        got = bits_np(bits_dev[s // 32:(s + m + 31) // 32])
        assert np.array_equal(got, exp), "answers %d..%d" % (s, s + m)


def oracle_filter_of_stream(w, chunk=1 << 27):
    """The oracle's filter for all of w's inserted hashes (the role-0 stream),
    built chunk by chunk on all host cores (threads own block ranges)."""
    import oracle
    import sbbf_inputs as inp

    threads = oracle.num_cores()
    ref = oracle.new_filter(w.num_blocks)
    for s in range(0, w.n_insert, chunk):
        keys = inp.fast_stream(w.cfg, inp.ROLE_INSERT, min(chunk, w.n_insert - s), s)
        oracle.insert_mt(ref, w.num_blocks, keys, threads)
    return ref


def compare_words(words_dev, ref, chunk_words=1 << 28):
    """A device filter's words against the oracle's, whole, in chunks."""
    flat = words_dev.reshape(-1)
    assert flat.numel() == ref.size
    for s in range(0, ref.size, chunk_words):
        e = min(ref.size, s + chunk_words)
        assert np.array_equal(flat[s:e].cpu().numpy().view(np.uint32), ref[s:e]), \
            "words %d..%d" % (s, e)
