"""Pins of the oracle's LUP factorisation (oracle.lup), independent of its
code: P A = L U checked in Python's exact integers, the shapes of L and U,
brute-force ranks that fix the pivot columns and the canonical pivot rows,
the factorisation of a product L0 U0 that needs no row exchange, and the
Vandermonde determinant read off U.

The paper names an LUP factorisation as the option to add beside the rank
decomposition (section 6, "Conclusions and Outlook") without defining its
pivot rule; the reading pinned here: the pivot of each column is the
lowest-index row, in the original order, among the rows not yet used whose
current entry is nonzero, so P lists the pivot rows in pivot order, then the
other rows in increasing order.
"""
import itertools

import numpy as np
import pytest

import oracle
from test_oracle_pins import det_leibniz, matmul_mod, rank_bruteforce, rand_residues, rng

PRIMES = [3, 5, 7, 65537, 2**31 - 1, 2147483629]


def check_factorisation(A, p, L, U, perm, r, piv):
    m, n = A.shape
    mn = min(m, n)
    assert sorted(perm.tolist()) == list(range(m))
    assert L.shape == (m, mn) and U.shape == (m, n)
    # L: unit diagonal, zero above it, columns at or beyond the rank unit vectors
    for i in range(m):
        for t in range(mn):
            if t == i:
                assert L[i, t] == 1
            elif t > i or t >= r:
                assert L[i, t] == 0
    # U: row echelon with heads at the pivot columns, zero rows from the rank
    assert len(piv) == r and all(piv[t] < piv[t + 1] for t in range(r - 1))
    for t in range(m):
        nz = np.flatnonzero(U[t])
        if t < r:
            assert len(nz) and nz[0] == piv[t]
        else:
            assert len(nz) == 0
    # P A = L U: the stored columns suffice because U's rows from min(m, n) are zero
    PA = A[perm]
    LU = matmul_mod(L, U[:mn], p) if mn else np.zeros((m, n), dtype=np.uint32)
    assert np.array_equal(PA, LU)


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("shape_rank", [(6, 9, 4), (12, 12, 12), (15, 10, 7), (1, 5, 1), (8, 1, 1),
                                        (20, 31, 0), (17, 40, 17), (33, 21, 21), (30, 30, 11)])
def test_pa_equals_lu(p, shape_rank):
    m, n, rank = shape_rank
    g = rng(m * 101 + n * 7 + rank + p % 13)
    A = matmul_mod(rand_residues(g, (m, rank), p), rand_residues(g, (rank, n), p), p) if rank else \
        np.zeros((m, n), dtype=np.uint32)
    L, U, perm, r, piv = oracle.lup(A, p)
    if p > 7:   # a random product of full-rank factors keeps the rank for large p
        assert r == rank
    check_factorisation(A, p, L, U, perm, r, piv)


@pytest.mark.parametrize("p", [3, 5, 7, 2**31 - 1])
@pytest.mark.parametrize("seed", range(6))
def test_rank_pivots_and_pivot_rows_bruteforce(p, seed):
    """On tiny matrices: the rank and pivot columns from all minors, and the
    pivot rows: row perm[t] is the lowest-index unused row whose prefix
    A[i, :c_t + 1] is independent of the earlier pivot rows' prefixes."""
    g = rng(seed * 17 + p % 97)
    m, n = int(g.integers(1, 5)), int(g.integers(1, 6))
    A = rand_residues(g, (m, n), p)
    if seed % 2:   # sparse entries make rows and columns vanish
        A[g.random((m, n)) < 0.5] = 0
    L, U, perm, r, piv = oracle.lup(A, p)
    assert r == rank_bruteforce(A, p)
    prev, want = 0, []
    for c in range(n):
        rc = rank_bruteforce(A[:, :c + 1], p)
        if rc > prev:
            want.append(c)
        prev = rc
    assert list(piv) == want
    used = []
    for t, c in enumerate(piv):
        cand = [i for i in range(m) if i not in used
                and rank_bruteforce(A[np.ix_(used + [i], range(c + 1))], p) == t + 1]
        assert perm[t] == min(cand)
        used.append(int(perm[t]))
    assert list(perm[r:]) == sorted(set(range(m)) - set(used))
    check_factorisation(A, p, L, U, perm, r, piv)


@pytest.mark.parametrize("p", [7, 65537, 2**31 - 1])
@pytest.mark.parametrize("n", [1, 4, 19, 40])
def test_product_without_exchanges_is_recovered(p, n):
    """A = L0 U0 with unit lower L0 and upper U0 of nonzero diagonal: every
    leading head is nonzero, no row moves, so P = I, L = L0 and U = U0."""
    g = rng(n * 13 + p % 11)
    L0 = np.tril(rand_residues(g, (n, n), p), -1) + np.eye(n, dtype=np.uint32)
    U0 = np.triu(rand_residues(g, (n, n), p), 1)
    U0[np.arange(n), np.arange(n)] = g.integers(1, p, size=n)
    A = matmul_mod(L0, U0, p)
    L, U, perm, r, piv = oracle.lup(A, p)
    assert r == n and list(perm) == list(range(n)) and list(piv) == list(range(n))
    assert np.array_equal(L, L0) and np.array_equal(U, U0)


@pytest.mark.parametrize("p", [65537, 2**31 - 1])
@pytest.mark.parametrize("n", [2, 5, 16, 33])
def test_vandermonde_determinant_from_u(p, n):
    """det A = sign(P) * prod of U's diagonal = prod_{i<j} (x_j - x_i)."""
    g = rng(n * 3 + p % 5)
    x = g.choice(p, size=n, replace=False)
    V = np.array([[pow(int(xi), j, p) for j in range(n)] for xi in x], dtype=np.uint32)
    g.shuffle(V)   # rows in any order: P must undo the exchanges the rule makes
    L, U, perm, r, piv = oracle.lup(V, p)
    inversions = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
    det = 1
    for t in range(n):
        det = det * int(U[t, t]) % p
    if inversions % 2:
        det = (p - det) % p
    xs = [int(row[1]) if n > 1 else 0 for row in V]
    expect = 1
    for i in range(n):
        for j in range(i + 1, n):
            expect = expect * ((xs[j] - xs[i]) % p) % p
    assert r == n and det == expect
    if n <= 5:
        assert det == det_leibniz(V, p)


@pytest.mark.parametrize("p", [3, 2**31 - 1])
def test_special_matrices(p):
    Z = np.zeros((5, 7), dtype=np.uint32)
    L, U, perm, r, piv = oracle.lup(Z, p)
    assert r == 0 and list(perm) == list(range(5)) and not U.any()
    assert np.array_equal(L, np.eye(5, 5, dtype=np.uint32))
    I = np.eye(6, dtype=np.uint32)
    L, U, perm, r, piv = oracle.lup(I[::-1].copy(), p)
    # column 0's only nonzero is in the last row: the rows come out reversed
    assert r == 6 and list(perm) == list(range(5, -1, -1))
    assert np.array_equal(L, I) and np.array_equal(U, I)
    row = np.array([[0, 0, 2, 1]], dtype=np.uint32)
    L, U, perm, r, piv = oracle.lup(row, p)
    assert r == 1 and list(piv) == [2] and np.array_equal(U, row) and L.tolist() == [[1]]
    col = np.array([[0], [0], [p - 1], [1]], dtype=np.uint32)
    L, U, perm, r, piv = oracle.lup(col, p)
    assert r == 1 and list(perm) == [2, 0, 1, 3] and U[0, 0] == p - 1
    assert L[:, 0].tolist() == [1, 0, 0, p - 1]   # 1 = (p - 1) * (p - 1)
    check_factorisation(col, p, L, U, perm, r, piv)
