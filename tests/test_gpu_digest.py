"""The device block-range verification digest (sbbf_range_digest) against
the oracle's: every range's digest, set-bit count and partial-block count,
for 4, 8 and 16 lanes, ragged block counts, ranges from one block to more
than the filter, filters spanning many CTAs' chunks, words with planted
all-zero lanes and blocks, and filters built by the device's inserts (no
partial block)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2101_01719_gb300 as sb
from paper_2101_01719_gb300 import sbbf
import sbbf_inputs as inp
from gpu_util import dev, to_dev

pytestmark = pytest.mark.gpu


def _words(cfg, lanes, nb):
    """Seeded words with sparse and dense lanes, whole zero blocks and zero
    lanes inside non-zero blocks."""
    w = inp.stream(cfg, lanes, -(-nb * lanes // 2)).view(np.uint32)[: nb * lanes].copy()
    blocks = w.reshape(nb, lanes)
    blocks[::5] &= blocks[::5] >> np.uint32(7)
    blocks[1::11] = 0
    blocks[2::13, 1] = 0
    blocks[3::17, lanes - 1] = 0
    return w


def _device_digest(words, lanes, R):
    t = torch.from_numpy(words.view(np.int32)).to(dev())
    return [x.cpu().numpy().view(np.uint64) for x in sbbf.range_digest(t, lanes, R)]


@pytest.mark.parametrize("lanes", [4, 8, 16])
@pytest.mark.parametrize("nb,R", [(1, 1), (37, 5), (1000, 1), (1000, 7), (100_003, 4096),
                                  (100_003, 10**9), (2**20 + 13, 2**16 + 1), (2**22 + 3, 2**20)])
def test_device_digest_equals_oracle(lanes, nb, R):
    w = _words(200 + lanes, lanes, nb)
    got = _device_digest(w, lanes, R)
    exp = oracle.range_digest(w, lanes, R, threads=8)
    for name, g, e in zip(("digest", "bits", "partial"), got, exp):
        assert np.array_equal(g, e), name
    assert exp[2].any() or nb < 20


def test_device_digest_of_built_filters():
    """Device-built filters (random and slice-ordered inserts) against the
    oracle's filter of the same hashes: equal digests, no partial block."""
    for B, n, mode in ((4096, 100_000, sb.PARTITION_OFF), (2**23 + 5, 5_000_001, sb.PARTITION_ON)):
        keys = inp.stream(210, 0, n)
        f = sb.Filter(B).set_partitioning(mode)
        f.insert(to_dev(keys))
        ref = oracle.new_filter(B)
        oracle.insert_mt(ref, B, keys, oracle.num_cores())
        R = 4099
        got = [x.cpu().numpy().view(np.uint64) for x in f.range_digest(R)]
        exp = oracle.range_digest(ref, 8, R, threads=8)
        for g, e in zip(got, exp):
            assert np.array_equal(g, e)
        assert not got[2].any()
        # one flipped bit shows in its range and no other
        f.words[8 * 1234 + 3] ^= 1 << 9
        d2 = f.range_digest(R)[0].cpu().numpy().view(np.uint64)
        diff = np.flatnonzero(d2 != got[0])
        assert diff.tolist() == [1234 // R]


def test_device_digest_lane_variants_and_empty():
    for lanes in (4, 16):
        B = 70_001
        keys = inp.stream(220 + lanes, 0, 200_000)
        f = sb.Filter(B, lanes=lanes)
        f.insert(to_dev(keys))
        ref = np.zeros(B * lanes, np.uint32)
        oracle.insert_k(ref, B, lanes, keys)
        got = [x.cpu().numpy().view(np.uint64) for x in f.range_digest(1000)]
        for g, e in zip(got, oracle.range_digest(ref, lanes, 1000)):
            assert np.array_equal(g, e)
        assert not got[2].any()
    f = sb.Filter(10)
    d, b, p = f.range_digest(3)
    zero = oracle.range_digest(np.zeros(80, np.uint32), 8, 3)
    assert np.array_equal(d.cpu().numpy().view(np.uint64), zero[0])
    assert not b.any() and not p.any()
    with pytest.raises(ValueError):
        f.range_digest(0)
