"""Parity with the oracle at primes whose 2^32 mod p is dense.

The plain trailing update (section 3.2, "Row reduce", blocked to rank k)
folds its signed 64-bit accumulator H*2^32 + L to H*(2^32 mod p) + L.  When
2^32 mod p has at most three set bits the fold is shifts and adds on the ALU
pipe, otherwise two multiply-adds; the per-output reduction is then Barrett's
instead of the multiply-free one.  The benchmark primes 2^31 - 1 and
2^31 - 19 (2^32 mod p = 2 and 38) take the shift fold, so these tests run
linac_rref, linac_solve and linac_rref_batched, element by element against
the oracle, at primes that take the other branches:

  P_BIGFOLD  1431655777  the first prime above 2^32/3: 2^32 mod p =
                         1431655742 (17 set bits), multiply fold every 8
                         products, Barrett reduction
  P_DENSE31  1908903247  a 31-bit prime with 2^32 mod p = 477160802
                         (14 set bits): multiply fold every 8, Barrett
  P_DENSE16  1381576943  2^32 mod p = 150236467 (15 set bits): the smaller
                         p allows a fold every 16 products
  251                    2^32 mod p = 123 (6 set bits), fold every 16
  P_SPARSE   2147418079  2^32 mod p = 131138 = 2^17 + 2^6 + 2 (3 set bits):
                         shift fold, but the multiply-free reduction's
                         bounds fail (c32 (c32 + 1)/2 > p), so Barrett

The batched kernel (its own fold and reduction choices) is also run at

  P_EDGE_IN  2147450923  2^32 mod p = 65450 (12 set bits): the largest such
                         value below 2^16 whose two-fold reduction bounds
                         (c32 (c32 + 1)/2 <= p, 2^32 - 1 + c32 (c32/2 + 1) < 3p)
                         still hold, so the batched kernel folds on the
                         multiply pipe and reduces by two folds and two
                         conditional subtractions; fold every 8 products
  P_EDGE_OUT 2147450861  2^32 mod p = 65574: just outside those bounds, so
                         Barrett; fold every 8
  2^31 - 19              2^32 mod p = 38: multiply-pipe fold every 8 with the
                         two-fold reduction

The CPU test at the end checks those properties of the primes themselves.
Shapes span two or more panels with ragged tails, at panel widths 128 and 32;
one matrix has entries (p - 1)/2 and (p + 1)/2 only, the balanced
representatives of largest magnitude, so the first panel's products all sit
at the accumulator bound ((p - 1)/2)^2.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_25863_gb300 import linac, synth
from modmath import matmul_mod

NTH = min(16, os.cpu_count() or 1)

P_BIGFOLD = 1431655777
P_DENSE31 = 1908903247
P_DENSE16 = 1381576943
P_SPARSE = 2147418079
DENSE_PRIMES = [P_BIGFOLD, P_DENSE31, P_DENSE16, 251, P_SPARSE]
P_EDGE_IN = 2147450923
P_EDGE_OUT = 2147450861
BATCHED_PRIMES = DENSE_PRIMES + [P_EDGE_IN, P_EDGE_OUT, 2**31 - 19]


def _is_prime(n):
    if n < 2:
        return False
    d = 2
    while d * d <= n:
        if n % d == 0:
            return False
        d += 1
    return True


def _fold_cadence(p):
    """Products a folded accumulator may take before the next fold: the
    largest of 16, 8, 4 that keeps |acc| below 2^63 (balanced operands)."""
    c32 = (1 << 32) % p
    half = (p - 1) // 2
    amax = max(((1 << 31) - 1) * c32 + (1 << 32) - 1, (1 << 31) * c32)
    k = ((1 << 63) - 1 - amax) // (half * half)
    return 16 if k >= 16 else (8 if k >= 8 else 4)


def test_primes_take_the_dense_fold_branches():
    """CPU: the primes above have the properties the tests rely on."""
    for p in DENSE_PRIMES:
        assert _is_prime(p) and p < 2**31
    bits = {p: bin((1 << 32) % p).count("1") for p in DENSE_PRIMES}
    assert all(bits[p] > 3 for p in (P_BIGFOLD, P_DENSE31, P_DENSE16, 251))
    assert _fold_cadence(P_BIGFOLD) == 8 and _fold_cadence(P_DENSE31) == 8
    assert _fold_cadence(P_DENSE16) == 16 and _fold_cadence(251) == 16
    c = (1 << 32) % P_SPARSE
    assert bits[P_SPARSE] == 3 and c * (c + 1) // 2 > P_SPARSE and _fold_cadence(P_SPARSE) == 8
    # the benchmark primes take the shift fold with the multiply-free reduction
    for p in (2**31 - 1, 2**31 - 19):
        c = (1 << 32) % p
        assert bin(c).count("1") <= 3 and c * (c + 1) // 2 <= p
    # the edge primes of the two-fold reduction's bounds
    two_fold = lambda p, c: c * (c + 1) // 2 <= p and (1 << 32) - 1 + c * (c // 2 + 1) < 3 * p
    for p, inside in ((P_EDGE_IN, True), (P_EDGE_OUT, False)):
        c = (1 << 32) % p
        assert _is_prime(p) and p < 2**31 and bin(c).count("1") > 3 and _fold_cadence(p) == 8
        assert two_fold(p, c) == inside
    assert _fold_cadence(2**31 - 19) == 8 and two_fold(2**31 - 19, 38)


def _gpu_rref(M, p, **kw):
    A = linac.to_device(M)
    rank, piv = linac.linac_rref(A, p, **kw)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 0
    return A.cpu().numpy().view(np.uint32)[:, :M.shape[1]].copy(), int(rank.item()), piv.cpu().numpy()


def _check(M, p, **kw):
    R, r, piv = _gpu_rref(M, p, **kw)
    R0, r0, piv0, _ = oracle.rref(M, p, nthreads=NTH)
    assert r == r0
    assert np.array_equal(piv[:r], piv0) and (piv[r:] == -1).all()
    assert np.array_equal(R, R0)
    return r


@pytest.mark.gpu
@pytest.mark.parametrize("nb", [128, 32])
@pytest.mark.parametrize("shape", [(513, 700), (1000, 1100)])
@pytest.mark.parametrize("p", DENSE_PRIMES)
def test_rref_vs_oracle_dense_fold(p, shape, nb):
    m, n = shape
    M = synth.uniform(shape, p, synth.stream_key(m + n + nb, f"dense_fold{p}"))
    _check(M, p, nb=nb, path="plain")


@pytest.mark.gpu
@pytest.mark.parametrize("p", DENSE_PRIMES)
def test_rank_deficient_vs_oracle_dense_fold(p):
    M, _ = synth.rank_deficient(m=600, n=640, d=25, p=p, seed=p % 1000)
    assert _check(M, p) == 575


@pytest.mark.gpu
@pytest.mark.parametrize("path", ["plain", "crt", "hybrid"])
@pytest.mark.parametrize("nb", [128, 32])
@pytest.mark.parametrize("p", DENSE_PRIMES + [2**31 - 1])
def test_balanced_extremes_vs_oracle(p, nb, path):
    """Entries (p - 1)/2 and (p + 1)/2 only: every product of the first
    panel's update is +-((p - 1)/2)^2, the accumulator's worst case."""
    g = np.random.default_rng(p % 9973 + nb)
    half = (p - 1) // 2
    M = np.where(g.integers(0, 2, size=(700, 760)) == 1, half, half + 1).astype(np.uint32)
    _check(M, p, nb=nb, path=path)


@pytest.mark.gpu
@pytest.mark.parametrize("p", [P_BIGFOLD, 251, P_SPARSE])
def test_limb_path_vs_oracle_dense_fold(p):
    M = synth.uniform((513, 700), p, synth.stream_key(7, f"limb_dense{p}"))
    _check(M, p, path="limb")


@pytest.mark.gpu
@pytest.mark.parametrize("p", DENSE_PRIMES)
def test_solve_vs_oracle_dense_fold(p):
    """Section 5.2: [A | B] reduced with the search restricted to A, X read
    off; rank-deficient A with one inconsistent right-hand side."""
    g = np.random.default_rng(p % 7919)
    A, _ = synth.rank_deficient(m=520, n=530, d=11, p=p, seed=p % 991)
    x0 = synth.uniform((530, 4), p, synth.stream_key(3, f"solve_dense{p}"))
    B = matmul_mod(A, x0, p)
    B[:, 2] = (B[:, 2].astype(np.int64) + 1 + g.integers(0, p - 1)) % p   # almost surely inconsistent
    X, cons, rank, piv = linac.linac_solve(linac.to_device(A), linac.to_device(B), p)
    torch.cuda.synchronize()
    X0, cons0, r0, piv0, _ = oracle.solve(A, B, p, nthreads=NTH)
    assert int(rank.item()) == r0 == 509
    assert np.array_equal(piv.cpu().numpy()[:r0], piv0)
    assert np.array_equal(cons.cpu().numpy(), cons0) and list(cons0) == [True, True, False, True]
    assert np.array_equal(X.cpu().numpy().view(np.uint32), X0)


@pytest.mark.gpu
@pytest.mark.parametrize("p", BATCHED_PRIMES)
def test_batched_vs_oracle_dense_fold(p):
    """linac_rref_batched (its own Montgomery and fold arithmetic) at the same
    primes, systems in every size bucket."""
    g = np.random.default_rng(p % 4999)
    shapes = [(1, 1), (7, 9), (40, 44), (64, 68), (100, 104), (129, 133), (200, 204), (257, 261),
              (300, 304), (511, 515), (600, 604), (1020, 1024)]
    systems = []
    for i, (m, n) in enumerate(shapes):
        S = synth.uniform((m, n), p, synth.stream_key(i, f"bt_dense{p}"))
        if m > 8 and i % 3 == 0:   # a few dependent rows
            S[m - 3:] = matmul_mod(g.integers(0, p, size=(3, m - 3), dtype=np.int64).astype(np.uint32),
                                   S[:m - 3], p)
        systems.append(S)
    _batched_check(systems, p)


def _batched_check(systems, p):
    """linac_rref_batched on the systems (4 right-hand-side columns outside the
    search where the system has more than 4 columns), every system compared
    with the oracle element by element."""
    B = synth._pack(systems, p, [s.shape[1] - 4 if s.shape[1] > 4 else s.shape[1] for s in systems],
                    [0] * len(systems))
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    data = t(B.data.view(np.int32))
    ranks, piv, poff, st = linac.linac_rref_batched(data, t(B.offsets), t(B.m), t(B.n), t(B.ld), p,
                                                    nsearch=t(B.nA))
    torch.cuda.synchronize()
    out = data.cpu().numpy().view(np.uint32)
    ranks, piv, poff = ranks.cpu().numpy(), piv.cpu().numpy(), poff.cpu().numpy()
    for s in range(B.count):
        o, m, n, ld = int(B.offsets[s]), int(B.m[s]), int(B.n[s]), int(B.ld[s])
        R0, r0, piv0, _ = oracle.rref(B.system(s), p, col_limit=int(B.nA[s]), nthreads=NTH)
        assert ranks[s] == r0, f"system {s}"
        assert np.array_equal(piv[poff[s]:poff[s] + r0], piv0), f"system {s}"
        assert np.array_equal(out[o:o + m * ld].reshape(m, ld)[:, :n], R0), f"system {s}"


@pytest.mark.gpu
@pytest.mark.parametrize("p", [P_EDGE_IN, P_EDGE_OUT, 2**31 - 19])
def test_batched_balanced_extremes(p):
    """Entries (p - 1)/2 and (p + 1)/2 only, so the first panel's products sit
    at the accumulator bound, in systems of every size bucket, through the
    batched kernel's fold and its two-fold or Barrett reduction."""
    g = np.random.default_rng(p % 6007)
    half = (p - 1) // 2
    shapes = [(40, 44), (100, 104), (200, 204), (300, 304), (511, 515), (700, 704)]
    systems = [np.where(g.integers(0, 2, size=sh) == 1, half, half + 1).astype(np.uint32) for sh in shapes]
    _batched_check(systems, p)
