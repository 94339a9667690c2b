"""CPU checks of the 64-bit input generators in synth (they feed the uint64
parity tests and the bench's uint64 leg, so both sides see the same inputs):

* uniform64 is floor(w * p / 2^64) of each SplitMix64 word w, checked with
  Python's exact integers, including across the generator's internal chunk
  boundary, and stays below p for primes from 3 to 2^64 - 59;
* rank_deficient64 keeps the untouched rows of the uniform stream and drops
  the rank by exactly the number of replaced rows.
"""
import numpy as np
import pytest

import oracle
from paper_2605_25863_gb300 import synth

PRIMES = [3, 2**31 - 1, 2**32 + 15, 2**61 - 1, 2**63 - 25, 2**64 - 59]


@pytest.mark.parametrize("p", PRIMES)
def test_uniform64_is_multiply_shift_of_the_stream(p):
    key = synth.stream_key(5, "u64test")
    got = synth.uniform64((37, 11), p, key, start=123)
    w = synth.words(key, 37 * 11, start=123)
    want = np.asarray([(int(x) * p) >> 64 for x in w], dtype=np.uint64).reshape(37, 11)
    assert np.array_equal(got, want)
    assert int(got.max()) < p


def test_uniform64_across_the_chunk_boundary():
    p = 2**64 - 59
    key = synth.stream_key(6, "u64chunk")
    n = (1 << 22) + 7
    got = synth.uniform64((n,), p, key)
    for i in (0, (1 << 22) - 1, 1 << 22, n - 1):
        w = int(synth.words(key, 1, start=i)[0])
        assert int(got[i]) == (w * p) >> 64


def test_uniform64_is_roughly_uniform():
    p = 2**64 - 59
    v = synth.uniform64((200000,), p, synth.stream_key(7, "u64mean")).astype(np.float64)
    assert abs(v.mean() / p - 0.5) < 0.01
    assert abs((v < p / 4).mean() - 0.25) < 0.01


@pytest.mark.parametrize("p", [5, 2**32 + 15, 2**64 - 59])
def test_rank_deficient64(p):
    m, n, d = 30, 34, 4
    M, targets = synth.rank_deficient64(m, n, d, p, seed=3)
    U = synth.uniform64((m, n), p, synth.stream_key(3, "rank_deficient64"))
    keep = np.setdiff1d(np.arange(m), targets)
    assert len(targets) == d
    assert np.array_equal(M[keep], U[keep])
    _, rank, _ = oracle.rref64(M, p)
    assert rank == m - d
