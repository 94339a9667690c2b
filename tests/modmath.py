"""Exact modular helpers for the tests (independent of the oracle and of the
CUDA library): matrix products mod p through int64 with a 16-bit split, and
random constructions whose RREF is known in advance."""
import numpy as np


def matmul_mod(A, B, p):
    """(A @ B) mod p exactly for residues < 2^31 and inner dimension < 2^16."""
    A = np.asarray(A, dtype=np.int64)
    B = np.asarray(B, dtype=np.uint64)
    assert A.shape[1] < (1 << 16)
    lo = (B & np.uint64(0xFFFF)).astype(np.int64)
    hi = (B >> np.uint64(16)).astype(np.int64)
    r_lo = (A @ lo) % p
    r_hi = (A @ hi) % p
    return ((r_lo + (r_hi << 16) % p) % p).astype(np.uint32)


def random_rref(g, m, n, rank, p, pivots=None):
    """Random RREF: identity at the pivot columns, random residues right of
    each pivot in the non-pivot columns, zero rows below the rank."""
    piv = np.sort(g.choice(n, size=rank, replace=False)) if pivots is None else np.asarray(pivots)
    R = np.zeros((m, n), dtype=np.uint32)
    mask = np.ones(n, dtype=bool)
    mask[piv] = False
    for t, c in enumerate(piv):
        R[t, c] = 1
        cols = np.nonzero(mask & (np.arange(n) > c))[0]
        R[t, cols] = g.integers(0, p, size=len(cols), dtype=np.int64).astype(np.uint32)
    return R, piv


def random_invertible(g, m, p):
    """P L U with unit lower L, upper U with nonzero diagonal, permutation P."""
    L = np.tril(g.integers(0, p, size=(m, m), dtype=np.int64), -1) + np.eye(m, dtype=np.int64)
    U = np.triu(g.integers(0, p, size=(m, m), dtype=np.int64), 1)
    U[np.arange(m), np.arange(m)] = g.integers(1, p, size=m, dtype=np.int64)
    G = matmul_mod(L.astype(np.uint32), U.astype(np.uint32), p)
    return G[g.permutation(m)]


def known_rref_matrix(g, m, n, rank, p, pivots=None):
    """(A, R, pivots) with RREF(A) = R by construction (A = G R, G invertible)."""
    R, piv = random_rref(g, m, n, rank, p, pivots)
    G = random_invertible(g, m, p)
    return matmul_mod(G, R, p), R, piv
