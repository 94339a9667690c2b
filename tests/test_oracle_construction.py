"""Pins for the oracle's matrix construction and products (paper section 3.3,
"Building linear systems on GPUs"; section 2.3, cuda_load_matrix; section
5.1, rank factorisation and null space).

Each check rests on something other than the oracle's own code:

* the product A B mod p against Python's exact integers on small shapes,
  plus identities (A I = A, (A B) C = A (B C), zero inner dimension);
* load_matrix against closed forms: d = 1 selects basis columns, a
  monomial x^a y^b equals pow(x, a, p) * pow(y, b, p) (Python's modular
  power), the constant monomial is 1, and a Vandermonde ansatz row is
  (1, x, x^2, ...);
* template evaluation against direct evaluation of every polynomial entry
  with Python's pow at each point;
* A = C R and A K = 0 for the oracle's RREF of matrices whose RREF is known
  by construction.
"""
import numpy as np
import pytest

import oracle
from tests.modmath import known_rref_matrix

PRIMES = [3, 5, 7, 65537, 2**31 - 1, 2147483629]


def exact_matmul(A, B, p):
    A = np.asarray(A, dtype=object)
    B = np.asarray(B, dtype=object)
    return np.asarray((A @ B) % p, dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 2), (7, 1, 9), (6, 13, 4), (2, 0, 3)])
def test_matmul_exact_integers(p, shape):
    g = np.random.default_rng(shape[0] * 131 + shape[1] + p % 1000)
    m, K, n = shape
    A = g.integers(0, p, size=(m, K), dtype=np.int64).astype(np.uint32)
    B = g.integers(0, p, size=(K, n), dtype=np.int64).astype(np.uint32)
    C = oracle.matmul(A, B, p)
    assert C.shape == (m, n)
    assert np.array_equal(C, exact_matmul(A, B, p))


@pytest.mark.parametrize("p", [5, 2**31 - 1])
def test_matmul_identities(p):
    g = np.random.default_rng(11)
    A = g.integers(0, p, size=(5, 6), dtype=np.int64).astype(np.uint32)
    B = g.integers(0, p, size=(6, 4), dtype=np.int64).astype(np.uint32)
    C = g.integers(0, p, size=(4, 3), dtype=np.int64).astype(np.uint32)
    assert np.array_equal(oracle.matmul(A, np.eye(6, dtype=np.uint32), p), A)
    assert np.array_equal(oracle.matmul(oracle.matmul(A, B, p), C, p), oracle.matmul(A, oracle.matmul(B, C, p), p))
    # p - 1 everywhere: (p-1)^2 * K = K mod p per entry
    F = np.full((3, 7), p - 1, dtype=np.uint32)
    G = np.full((7, 2), p - 1, dtype=np.uint32)
    assert (oracle.matmul(F, G, p) == 7 % p).all()


@pytest.mark.parametrize("p", PRIMES)
def test_load_matrix_closed_forms(p):
    g = np.random.default_rng(p % 997)
    pts = g.integers(0, p, size=(9, 2), dtype=np.int64)
    bases = np.concatenate([np.ones((9, 1), dtype=np.int64), pts], axis=1).astype(np.uint32)
    # monomials x^a y^b, a + b <= 4, as repeated indices padded with the constant 1
    mons = [(a, b) for t in range(5) for a in range(t, -1, -1) for b in [t - a]]
    lind = np.zeros((len(mons), 4), dtype=np.int32)
    for u, (a, b) in enumerate(mons):
        idx = [1] * a + [2] * b
        lind[u, :len(idx)] = idx
    A = oracle.load_matrix(bases, lind, p)
    for r in range(9):
        x, y = int(pts[r, 0]), int(pts[r, 1])
        for u, (a, b) in enumerate(mons):
            assert int(A[r, u]) == pow(x, a, p) * pow(y, b, p) % p
    # d = 1 selects basis columns
    sel = np.array([[2], [0], [1], [2]], dtype=np.int32)
    assert np.array_equal(oracle.load_matrix(bases, sel, p), bases[:, [2, 0, 1, 2]] % p)
    # Vandermonde ansatz: column c is x^c (c repeated indices of x, rest the constant)
    d = 6
    lv = np.array([[1] * c + [0] * (d - c) for c in range(d + 1)], dtype=np.int32)
    V = oracle.load_matrix(bases, lv, p)
    for r in range(9):
        assert [int(v) for v in V[r]] == [pow(int(pts[r, 0]), c, p) for c in range(d + 1)]


def test_load_matrix_rejects_bad_indices():
    with pytest.raises(ValueError):
        oracle.load_matrix(np.ones((2, 3), dtype=np.uint32), np.array([[3]], dtype=np.int32), 7)


@pytest.mark.parametrize("p", [7, 2**31 - 1])
def test_eval_template_direct(p):
    g = np.random.default_rng(5)
    rows, cols = 6, 7
    mask = g.random((rows, cols)) < 0.4
    mons = [(a, t - a) for t in range(4) for a in range(t, -1, -1)]
    nnz = int(mask.sum())
    coefs = g.integers(0, p, size=(nnz, len(mons)), dtype=np.int64).astype(np.uint32)
    pts = g.integers(0, p, size=(5, 2), dtype=np.int64).astype(np.uint32)
    out = oracle.eval_template(pts, coefs, mons, mask, p)
    pos = list(zip(*np.nonzero(mask)))
    for s in range(5):
        x, y = int(pts[s, 0]), int(pts[s, 1])
        want = np.zeros((rows, cols), dtype=np.uint32)
        for e, (i, j) in enumerate(pos):
            want[i, j] = sum(int(coefs[e, u]) * pow(x, a, p) * pow(y, b, p) for u, (a, b) in enumerate(mons)) % p
        assert np.array_equal(out[s], want)


@pytest.mark.parametrize("p", [5, 2**31 - 1])
@pytest.mark.parametrize("shape_rank", [(6, 9, 4), (9, 6, 6), (8, 8, 3), (5, 5, 0)])
def test_rank_factorisation_and_null_space(p, shape_rank):
    m, n, rank = shape_rank
    g = np.random.default_rng(m * 17 + n + rank)
    A, R_known, piv_known = known_rref_matrix(g, m, n, rank, p)
    R, r, piv, _ = oracle.rref(A, p)
    assert r == rank and np.array_equal(piv, piv_known)
    C = oracle.rank_factor(A, piv)
    assert C.shape == (m, r)
    if r:
        assert np.array_equal(exact_matmul(C, R[:r], p), A)            # A = C R
    K = oracle.null_space(R, piv, p)
    assert K.shape == (n, n - r)
    if n - r:
        assert not exact_matmul(A, K, p).any()                        # A K = 0
        free = [c for c in range(n) if c not in set(piv.tolist())]
        assert np.array_equal(K[free], (np.eye(n - r, dtype=np.int64) * (p - 1)).astype(np.uint32))
