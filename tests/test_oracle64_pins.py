"""Pins for the oracle's 64-bit residues (paper section 2.3: uint64 storage
for primes that do not fit 32 bits, up to 2^64 - 1).

Facts fixed by the mathematics, each computed with Python integers (exact,
no 64-bit wrap-around) and never by the oracle itself:

* known RREF by construction: R is a random RREF, A = G R with G = P L U
  invertible; the RREF is unique (section 5.1), so RREF(A) must be R;
* h * (1/h) = 1 mod p for the Fermat inverse, at both ends of the range;
* for primes below 2^31 the 64-bit oracle agrees with the 32-bit oracle,
  whose own pins are in test_oracle_pins.py;
* solve: A X = B exactly for consistent right-hand sides, a right-hand side
  built outside the column space is flagged inconsistent, free variables
  are zero (section 5.2);
* special matrices: zero, identity, p - 1 everywhere, one row, one column;
* null space and rank factorisation (section 5.1): A K = 0 with the free rows
  of K equal to -I, and A = C R.
The primes span the range: tiny (3, 5), below 2^31, just above 2^32, the
Mersenne prime 2^61 - 1, the largest primes below 2^63 and 2^64.
"""
import numpy as np
import pytest

import oracle
from paper_2605_25863_gb300 import synth

P64 = [3, 5, 2**31 - 1, 2**32 + 15, 2**61 - 1, 2**63 - 25, 2**64 - 59]


def is_prime(n):
    """Deterministic Miller-Rabin with the first twelve prime bases (exact
    for every n < 3.3e24, far beyond 2^64)."""
    if n < 2:
        return False
    bases = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for q in bases:
        if n % q == 0:
            return n == q
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in bases:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def test_primes_are_prime():
    for p in P64:
        assert is_prime(p), p
    assert not is_prime(2**64 - 1) and not is_prime(2**61 + 1)


def matmul_exact(A, B, p):
    A = np.asarray(A, dtype=object)
    B = np.asarray(B, dtype=object)
    return np.asarray((A.dot(B)) % p, dtype=np.uint64)


def rand64(g, shape, p):
    """Residues in [0, p) from Python's integers (p may exceed int64)."""
    flat = [int(g.integers(0, 1 << 62)) * 4 + int(g.integers(0, 4)) for _ in range(int(np.prod(shape)))]
    return np.asarray([v % p for v in flat], dtype=np.uint64).reshape(shape)


def random_rref64(g, m, n, rank, p):
    piv = np.sort(g.choice(n, size=rank, replace=False)) if rank else np.zeros(0, dtype=np.int64)
    R = np.zeros((m, n), dtype=np.uint64)
    for t, c in enumerate(piv):
        R[t, c] = 1
        for j in range(c + 1, n):
            if j not in piv:
                R[t, j] = rand64(g, (1,), p)[0]
    return R, piv


def random_invertible64(g, m, p):
    L = np.zeros((m, m), dtype=object)
    U = np.zeros((m, m), dtype=object)
    for i in range(m):
        L[i, i] = 1
        for j in range(i):
            L[i, j] = int(rand64(g, (1,), p)[0])
        U[i, i] = 1 + int(rand64(g, (1,), p - 1)[0])
        for j in range(i + 1, m):
            U[i, j] = int(rand64(g, (1,), p)[0])
    P = np.eye(m, dtype=object)[g.permutation(m)]
    return np.asarray(P.dot(L.dot(U) % p) % p, dtype=object)


@pytest.mark.parametrize("p", P64)
@pytest.mark.parametrize("mnr", [(1, 1, 1), (1, 1, 0), (6, 9, 4), (12, 7, 7), (20, 20, 20), (15, 40, 9),
                                 (30, 12, 5), (9, 9, 0)])
def test_known_rref_by_construction(mnr, p):
    m, n, r = mnr
    g = np.random.default_rng(m * 131 + n * 7 + r + p % 1000)
    R, piv = random_rref64(g, m, n, r, p)
    G = random_invertible64(g, m, p)
    A = matmul_exact(G, R, p)
    got, rank, pivots = oracle.rref64(A, p)
    assert rank == r
    assert list(pivots) == list(piv)
    assert np.array_equal(got, R)


@pytest.mark.parametrize("p", P64)
def test_inverse_times_value_is_one(p):
    g = np.random.default_rng(p % 99991)
    hs = {1, p - 1, 2 % p or 1, (p - 1) // 2 or 1} | {int(v) or 1 for v in rand64(g, (20,), p)}
    for h in hs:
        assert h * oracle.inverse64(h, p) % p == 1


@pytest.mark.parametrize("p", [3, 7, 65537, 2**31 - 1, 2147483629])
@pytest.mark.parametrize("mnd", [(40, 60, 7), (60, 40, 0), (33, 33, 33), (70, 90, 12)])
def test_agrees_with_32bit_oracle(mnd, p):
    m, n, d = mnd
    if d >= m:
        M = np.zeros((m, n), dtype=np.uint32)
    else:
        M, _ = synth.rank_deficient(m=m, n=n, d=d, p=p, seed=m + n)
    R32, r32, piv32, _ = oracle.rref(M, p)
    R64, r64, piv64 = oracle.rref64(M.astype(np.uint64), p)
    assert r64 == r32
    assert np.array_equal(piv64, piv32)
    assert np.array_equal(R64, R32.astype(np.uint64))


@pytest.mark.parametrize("p", P64)
def test_special_matrices(p):
    Z = np.zeros((5, 7), dtype=np.uint64)
    R, r, piv = oracle.rref64(Z, p)
    assert r == 0 and not R.any()
    I = np.eye(6, dtype=np.uint64)
    R, r, piv = oracle.rref64(I, p)
    assert r == 6 and np.array_equal(R, I)
    # p - 1 everywhere: rank 1, first row all ones
    F = np.full((4, 5), p - 1, dtype=np.uint64)
    R, r, piv = oracle.rref64(F, p)
    assert r == 1 and list(piv) == [0]
    assert (R[0] == 1).all() and not R[1:].any()
    # one row: divided by its first nonzero entry
    g = np.random.default_rng(p % 777)
    row = rand64(g, (1, 9), p)
    row[0, :2] = 0
    row[0, 2] = max(int(row[0, 2]), 1)
    R, r, piv = oracle.rref64(row, p)
    inv = pow(int(row[0, 2]), p - 2, p)
    assert r == 1 and list(piv) == [2]
    assert [int(v) for v in R[0]] == [int(v) * inv % p for v in row[0]]
    # one column: unit vector
    col = rand64(g, (7, 1), p)
    col[3, 0] = max(int(col[3, 0]), 1)
    R, r, piv = oracle.rref64(col, p)
    assert r == 1 and R[0, 0] == 1 and not R[1:].any()


@pytest.mark.parametrize("p", P64)
def test_solve_consistency_and_solutions(p):
    g = np.random.default_rng(p % 4093 + 1)
    m, n, r, k = 14, 11, 8, 3
    Rr, piv = random_rref64(g, m, n, r, p)
    G = random_invertible64(g, m, p)
    A = matmul_exact(G, Rr, p)
    X0 = rand64(g, (n, 2), p)
    B = np.zeros((m, k), dtype=np.uint64)
    B[:, :2] = matmul_exact(A, X0, p)                       # in the column space
    B[:, 2] = np.asarray(G[:, r] % p, dtype=np.uint64)        # G e_r: outside span(G[:, :r])
    X, cons, rank, pv, _ = oracle.solve64(A, B, p)
    assert rank == r and list(pv) == list(piv)
    assert list(cons) == [True, True, False]
    AX = matmul_exact(A, X, p)
    assert np.array_equal(AX[:, :2], B[:, :2])
    free = [c for c in range(n) if c not in set(piv)]
    assert not X[free].any()
    assert not X[:, 2].any()


@pytest.mark.parametrize("p", [2**32 + 15, 2**63 - 25, 2**64 - 59])
def test_square_full_rank_solve_reproduces_solution(p):
    g = np.random.default_rng(p % 65521)
    n = 16
    A = np.asarray(random_invertible64(g, n, p) % p, dtype=np.uint64)
    x = rand64(g, (n, 1), p)
    b = matmul_exact(A, x, p)
    X, cons, rank, pv, M = oracle.solve64(A, b, p)
    assert rank == n and cons[0]
    assert np.array_equal(X, x)
    assert np.array_equal(M[:, :n], np.eye(n, dtype=np.uint64))


@pytest.mark.parametrize("p", [5, 2**32 + 15, 2**64 - 59])
@pytest.mark.parametrize("mnr", [(9, 14, 5), (14, 9, 9), (10, 10, 0), (12, 12, 12)])
def test_null_space_and_rank_factor(mnr, p):
    """Section 5.1 in exact integers: A K = 0, the free rows of K are -I, and
    A = C R with C = A[:, J] and R the RREF's first rank rows."""
    m, n, r = mnr
    g = np.random.default_rng(m * 7 + n + r)
    Rr, piv = random_rref64(g, m, n, r, p)
    A = matmul_exact(random_invertible64(g, m, p), Rr, p)
    R, rank, pivots = oracle.rref64(A, p)
    K = oracle.null_space64(R, pivots, p)
    assert K.shape == (n, n - rank)
    if n - rank:
        assert not matmul_exact(A, K, p).any()
        free = [c for c in range(n) if c not in set(pivots)]
        assert np.array_equal(K[free], np.eye(n - rank, dtype=np.uint64) * np.uint64(p - 1))
    C = oracle.rank_factor64(A, pivots)
    if rank:
        assert np.array_equal(matmul_exact(C, R[:rank], p), A)
