"""Pins for the CPU oracle: facts fixed by the mathematics, not by the oracle.

Each check would fail for a plausible slip in the oracle (a dropped update
term, a wrong sign, a wrong pivot index, an LU-style update that skips the
rows above the pivot, a wrong inverse, a transposed operand, a consistency
test read from the wrong rows):

* known RREF by construction: R is built first (random pivot pattern,
  identity at the pivot columns, zero rows at the bottom), A = G R for a
  random invertible G; the RREF is unique (paper section 5.1: the rows of
  the RREF are a basis of the row space), so RREF(A) must be R exactly;
* brute-force rank from all square minors (Leibniz expansion mod p) and
  pivot columns from prefix ranks -- no elimination involved;
* brute-force null spaces and solution sets over tiny fields (enumerate all
  of F_p^n), checked against section 5.1 (A K = 0, free columns -1) and
  section 5.2 (consistency iff rank(A) = rank(A|b), free variables 0);
* closed-form determinants: Vandermonde prod_{i<j}(x_j - x_i) and L*D*U;
* Vandermonde interpolation: the solve recovers a polynomial's coefficients;
* special matrices (zero, identity, permutations, duplicated rows, p - 1
  everywhere, 1 x N, N x 1, wide and tall).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2605_25863_gb300 import synth

PRIMES = [3, 5, 7, 65537, 2**31 - 1, 2147483629]


def rng(seed):
    return np.random.default_rng(seed)


def matmul_mod(A, B, p):
    """Exact (A @ B) mod p through Python integers (small sizes only)."""
    A = np.asarray(A, dtype=object)
    B = np.asarray(B, dtype=object)
    return np.asarray((A @ B) % p, dtype=np.uint64).astype(np.uint32)


def rand_residues(g, shape, p):
    return g.integers(0, p, size=shape, dtype=np.int64).astype(np.uint32)


def random_rref(g, m, n, rank, p):
    """A random RREF with ``rank`` pivots: identity at the pivot columns,
    arbitrary residues right of each pivot in non-pivot columns, zero rows
    at the bottom."""
    piv = np.sort(g.choice(n, size=rank, replace=False))
    R = np.zeros((m, n), dtype=np.uint32)
    for t, c in enumerate(piv):
        R[t, c] = 1
        for j in range(c + 1, n):
            if j not in piv:
                R[t, j] = g.integers(0, p)
    return R, piv


def random_invertible(g, m, p):
    """P L U with unit lower L, upper U with nonzero diagonal, permutation P."""
    L = np.eye(m, dtype=np.int64)
    U = np.zeros((m, m), dtype=np.int64)
    for i in range(m):
        for j in range(i):
            L[i, j] = g.integers(0, p)
        U[i, i] = g.integers(1, p)
        for j in range(i + 1, m):
            U[i, j] = g.integers(0, p)
    P = np.eye(m, dtype=np.int64)[g.permutation(m)]
    return matmul_mod(P, matmul_mod(L, U, p), p)


def det_leibniz(M, p):
    """Determinant mod p by the Leibniz permutation expansion (tiny sizes)."""
    n = len(M)
    if n == 0:
        return 1
    total = 0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        term = 1
        for i in range(n):
            term = term * int(M[i][perm[i]]) % p
        total += -term if inv % 2 else term
    return total % p


def rank_bruteforce(A, p):
    """Largest s with a nonzero s x s minor."""
    m, n = A.shape
    for s in range(min(m, n), 0, -1):
        for rows in itertools.combinations(range(m), s):
            for cols in itertools.combinations(range(n), s):
                if det_leibniz(A[np.ix_(rows, cols)], p):
                    return s
    return 0


def pivots_bruteforce(A, p):
    """Column c is a pivot iff rank(A[:, :c+1]) > rank(A[:, :c])."""
    piv, prev = [], 0
    for c in range(A.shape[1]):
        r = rank_bruteforce(A[:, :c + 1], p)
        if r > prev:
            piv.append(c)
        prev = r
    return piv


# --------------------------------------------------------------------------
# Known RREF by construction


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("shape_rank", [(6, 9, 4), (12, 12, 12), (15, 10, 7), (1, 5, 1),
                                        (8, 1, 1), (20, 31, 0), (17, 40, 17), (33, 21, 21)])
def test_known_rref_by_construction(p, shape_rank):
    m, n, rank = shape_rank
    g = rng(hash((p, m, n, rank)) & 0xFFFF)
    R, piv = random_rref(g, m, n, rank, p)
    G = random_invertible(g, m, p)
    A = matmul_mod(G, R, p)
    out, r, pv, _ = oracle.rref(A, p)
    assert r == rank
    assert list(pv) == list(piv)
    assert np.array_equal(out, R)


@pytest.mark.parametrize("nthreads", [1, 3, 8])
def test_known_rref_threads(nthreads):
    g = rng(11)
    p = 2**31 - 1
    R, piv = random_rref(g, 70, 90, 55, p)
    A = matmul_mod(random_invertible(g, 70, p), R, p)
    out, r, pv, _ = oracle.rref(A, p, nthreads=nthreads)
    assert r == 55 and list(pv) == list(piv) and np.array_equal(out, R)


# --------------------------------------------------------------------------
# Brute force on tiny matrices


@pytest.mark.parametrize("p", [3, 5, 7, 2**31 - 1])
@pytest.mark.parametrize("seed", range(6))
def test_rank_and_pivots_bruteforce(p, seed):
    g = rng(100 + seed)
    m, n = int(g.integers(1, 5)), int(g.integers(1, 6))
    if seed % 2:   # force low rank by a product of thin factors
        k = int(g.integers(0, min(m, n) + 1))
        A = matmul_mod(rand_residues(g, (m, k), p), rand_residues(g, (k, n), p), p) if k else \
            np.zeros((m, n), dtype=np.uint32)
    else:
        A = rand_residues(g, (m, n), p)
    out, r, pv, _ = oracle.rref(A, p)
    assert r == rank_bruteforce(A, p)
    assert list(pv) == pivots_bruteforce(A, p)


def enumerate_vectors(n, p):
    return np.array(list(itertools.product(range(p), repeat=n)), dtype=np.int64)


@pytest.mark.parametrize("p", [3, 5])
@pytest.mark.parametrize("seed", range(5))
def test_null_space_bruteforce(p, seed):
    g = rng(200 + seed)
    m, n = int(g.integers(1, 5)), int(g.integers(1, 6))
    k = int(g.integers(0, min(m, n) + 1))
    A = matmul_mod(rand_residues(g, (m, k), p), rand_residues(g, (k, n), p), p) if k else \
        np.zeros((m, n), dtype=np.uint32)
    R, r, pv, _ = oracle.rref(A, p)
    X = enumerate_vectors(n, p)
    kernel = X[((A.astype(np.int64) @ X.T) % p == 0).all(axis=0)]
    assert len(kernel) == p ** (n - r)
    K = oracle.null_space(R, pv, p)
    assert K.shape == (n, n - r)
    assert not matmul_mod(A, K, p).any()
    free = [c for c in range(n) if c not in set(pv.tolist())]
    for f_idx, f in enumerate(free):      # free block is minus the identity
        col = K[:, f_idx]
        assert all(col[c] == ((p - 1) if c == f else 0) for c in free)


@pytest.mark.parametrize("p", [3, 5])
@pytest.mark.parametrize("seed", range(6))
def test_solve_bruteforce(p, seed):
    g = rng(300 + seed)
    m, nA, k = int(g.integers(1, 5)), int(g.integers(1, 5)), int(g.integers(1, 3))
    rk = int(g.integers(0, min(m, nA) + 1))
    A = matmul_mod(rand_residues(g, (m, rk), p), rand_residues(g, (rk, nA), p), p) if rk else \
        np.zeros((m, nA), dtype=np.uint32)
    B = rand_residues(g, (m, k), p)
    if seed % 2:   # make the first right-hand side consistent
        B[:, 0] = matmul_mod(A, rand_residues(g, (nA, 1), p), p)[:, 0]
    X, cons, r, pv, _ = oracle.solve(A, B, p)
    assert r == rank_bruteforce(A, p)
    V = enumerate_vectors(nA, p)
    free = [c for c in range(nA) if c not in set(pv.tolist())]
    for j in range(k):
        sols = V[((A.astype(np.int64) @ V.T) % p == B[:, j:j + 1].astype(np.int64)).all(axis=0)]
        assert cons[j] == (len(sols) > 0)
        if cons[j]:
            with_free_zero = [s for s in sols if all(s[c] == 0 for c in free)]
            assert len(with_free_zero) == 1
            assert np.array_equal(X[:, j].astype(np.int64), with_free_zero[0])
        else:
            assert not X[:, j].any()


# --------------------------------------------------------------------------
# Closed forms


@pytest.mark.parametrize("p", [65537, 2**31 - 1, 2147483629])
@pytest.mark.parametrize("n", [1, 2, 5, 16, 40])
def test_vandermonde_determinant(p, n):
    g = rng(n * 7 + p % 1000)
    x = g.choice(p, size=n, replace=False).astype(object)
    V = np.array([[pow(int(xi), j, p) for j in range(n)] for xi in x], dtype=np.uint32)
    expect = 1
    for i in range(n):
        for j in range(i + 1, n):
            expect = expect * ((int(x[j]) - int(x[i])) % p) % p
    _, r, _, det = oracle.rref(V, p)
    assert r == n and det == expect


@pytest.mark.parametrize("p", [7, 65537, 2**31 - 1])
@pytest.mark.parametrize("n", [3, 9, 25])
@pytest.mark.parametrize("zeros", [0, 1, 3])
def test_ldu_determinant_and_rank(p, n, zeros):
    g = rng(n * 31 + zeros)
    L = np.eye(n, dtype=np.int64)
    U = np.eye(n, dtype=np.int64)
    for i in range(n):
        for j in range(i):
            L[i, j] = g.integers(0, p)
            U[j, i] = g.integers(0, p)
    D = g.integers(1, p, size=n)
    D[g.choice(n, size=min(zeros, n), replace=False)] = 0
    A = matmul_mod(matmul_mod(L, np.diag(D), p), U, p)
    expect = 1
    for d in D:
        expect = expect * int(d) % p
    _, r, _, det = oracle.rref(A, p)
    assert det == expect
    assert r == int(np.count_nonzero(D))


@pytest.mark.parametrize("p", [2**31 - 1, 2147483629])
@pytest.mark.parametrize("n", [4, 17, 64])
def test_vandermonde_interpolation(p, n):
    """Section 3.3: an ansatz sum_i c_i x^i fitted at n distinct points
    returns the coefficients exactly (section 5.2, [A | b] -> [I | x])."""
    g = rng(n + 5)
    x = g.choice(p, size=n, replace=False)
    coef = [int(v) for v in g.integers(0, p, size=n)]
    V = np.array([[pow(int(xi), j, p) for j in range(n)] for xi in x], dtype=np.uint32)
    b = np.array([[sum(c * pow(int(xi), j, p) for j, c in enumerate(coef)) % p] for xi in x],
                 dtype=np.uint32)
    X, cons, r, pv, M = oracle.solve(V, b, p)
    assert cons[0] and r == n
    assert [int(v) for v in X[:, 0]] == coef
    R, r2, _, _ = oracle.rref(np.concatenate([V, b], axis=1), p)
    assert r2 == n and np.array_equal(R[:, :n], np.eye(n, dtype=np.uint32))
    assert [int(v) for v in R[:, n]] == coef


def test_inverse_exhaustive_small_and_random_large():
    for p in (3, 5, 7, 11, 13):
        for h in range(1, p):
            assert oracle.inverse(h, p) * h % p == 1
    g = rng(9)
    for p in (65537, 2**31 - 1, 2147483629):
        for h in g.integers(1, p, size=200):
            assert oracle.inverse(int(h), p) * int(h) % p == 1


# --------------------------------------------------------------------------
# Structure, invariance and special matrices


@pytest.mark.parametrize("p", [5, 2**31 - 1])
@pytest.mark.parametrize("shape", [(10, 14), (14, 10), (12, 12)])
def test_rank_factorisation_and_row_space_invariance(p, shape):
    """Section 5.1: A = A[:, J] R with R the nonzero rows of the RREF; and the
    RREF depends on the row space only, so RREF(G A) = RREF(A)."""
    m, n = shape
    g = rng(m * n + p % 97)
    k = min(m, n) - 2
    A = matmul_mod(rand_residues(g, (m, k), p), rand_residues(g, (k, n), p), p)
    R, r, pv, _ = oracle.rref(A, p)
    assert r == k
    assert not R[r:].any()
    assert np.array_equal(R[:r][:, pv], np.eye(r, dtype=np.uint32))
    for t, c in enumerate(pv):
        assert not R[t, :c].any()
    assert np.array_equal(matmul_mod(A[:, pv], R[:r], p), A)
    G = random_invertible(g, m, p)
    R2, r2, pv2, _ = oracle.rref(matmul_mod(G, A, p), p)
    assert r2 == r and np.array_equal(pv2, pv) and np.array_equal(R2, R)


@pytest.mark.parametrize("p", [3, 2**31 - 1])
def test_special_matrices(p):
    g = rng(4)
    Z = np.zeros((5, 7), dtype=np.uint32)
    R, r, pv, _ = oracle.rref(Z, p)
    assert r == 0 and len(pv) == 0 and not R.any()
    I = np.eye(6, dtype=np.uint32)
    R, r, pv, det = oracle.rref(I, p)
    assert r == 6 and np.array_equal(R, I) and det == 1
    Pm = I[g.permutation(6)]
    R, r, pv, det = oracle.rref(Pm, p)
    assert np.array_equal(R, I) and det in (1, p - 1)
    F = np.full((4, 5), p - 1, dtype=np.uint32)
    R, r, pv, _ = oracle.rref(F, p)
    assert r == 1 and list(pv) == [0] and np.array_equal(R[0], np.ones(5, dtype=np.uint32))
    assert not R[1:].any()
    row = rand_residues(g, (1, 9), p)
    row[0, 0] = 0
    row[0, 1] = 3 % p or 1
    D = np.repeat(row, 4, axis=0)
    R, r, pv, _ = oracle.rref(D, p)
    assert r == 1 and list(pv) == [1]
    assert R[0, 1] == 1 and not R[1:].any()
    col = rand_residues(g, (7, 1), p)
    col[0, 0] = 0
    col[3, 0] = 5 % p or 1
    R, r, pv, _ = oracle.rref(col, p)
    assert r == 1 and R[0, 0] == 1 and not R[1:].any()


def test_inconsistent_system_has_augmented_pivot():
    """Section 5.2: an inconsistent [A | b] reduces to a row (0, ..., 0 | 1)."""
    p = 2**31 - 1
    A = np.array([[1, 2], [2, 4]], dtype=np.uint32)
    b = np.array([[1], [3]], dtype=np.uint32)
    R, r, pv, _ = oracle.rref(np.concatenate([A, b], axis=1), p)
    assert list(pv) == [0, 2]
    assert list(R[1]) == [0, 0, 1]
    X, cons, rA, pvA, _ = oracle.solve(A, b, p)
    assert not cons[0] and rA == 1 and not X.any()


def test_max_pivots_prefix_matches_full_run():
    p = 2**31 - 1
    A = synth.uniform((40, 50), p, synth.stream_key(7, "prefix"))
    _, r, pv, _ = oracle.rref(A, p)
    _, r5, pv5, _ = oracle.rref(A, p, max_pivots=5)
    assert r5 == 5 and list(pv5) == list(pv[:5])


def test_workload_ranks_match_their_construction():
    """The generators' rank-deficiency recipes give the ranks they promise."""
    p = 2**31 - 1
    M, targets = synth.rank_deficient(m=64, n=70, d=5, p=p, seed=12)
    _, r, pv, _ = oracle.rref(M, p)
    assert r == 59 and list(pv) == list(range(59))
    B = synth.batched_uneven(count=30, lo=8, hi=24, seed=5, deficient_frac=0.5)
    for s in range(B.count):
        S = B.system(s)
        nA = int(B.nA[s])
        X, cons, rA, pvA, _ = oracle.solve(S[:, :nA], S[:, nA:], B.p)
        assert rA == nA - int(B.deficiency[s])
        assert cons.all()


@pytest.mark.parametrize("p", [7, 2**31 - 1])
@pytest.mark.parametrize("shape_rank", [(12, 15, 9), (20, 12, 10), (9, 9, 6)])
def test_solve_with_scattered_pivots(p, shape_rank):
    """A = G R with R an RREF whose pivots are scattered; b = A x0 is
    consistent, and the particular solution X (free variables zero) must
    satisfy A X = b exactly (section 5.2)."""
    m, nA, rank = shape_rank
    g = rng(m * 1000 + nA * 10 + rank)
    R, piv = random_rref(g, m, nA, rank, p)
    assert list(piv) != list(range(rank)) or rank == nA
    A = matmul_mod(random_invertible(g, m, p), R, p)
    x0 = rand_residues(g, (nA, 3), p)
    B = matmul_mod(A, x0, p)
    B[:, 2] = (B[:, 2].astype(np.int64) + 1) % p     # almost surely inconsistent
    X, cons, r, pv, _ = oracle.solve(A, B, p)
    assert r == rank and list(pv) == list(piv)
    assert cons[0] and cons[1]
    assert cons[2] == (rank == m)
    free = [c for c in range(nA) if c not in set(piv.tolist())]
    for j in range(2):
        assert np.array_equal(matmul_mod(A, X[:, j:j + 1], p)[:, 0], B[:, j])
        assert not X[free, j].any()
