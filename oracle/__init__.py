"""Plain CPU oracle for exact Gauss-Jordan elimination over Z/pZ.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module; the library itself
never does.  It shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (uint64 ``%`` reductions, Fermat
inverses, lowest-index nonzero pivots); this module compiles it with gcc on
first use and wraps it with ctypes.  Every function follows paper section
3.2 (the elimination loop) or section 5 (reading solutions, null spaces and
rank factorisations off the RREF), cited where it is defined.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no arch flags)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # ORACLE_LIB lets the mutation test load a deliberately broken build
        path = os.environ.get("ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        i64, u32, i32p = ctypes.c_int64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)
        vp = ctypes.c_void_p
        lib.oracle_rref.argtypes = [vp, i64, i64, i64, u32, i64, i64, ctypes.c_int,
                                    i32p, i32p, ctypes.POINTER(ctypes.c_uint32)]
        lib.oracle_rref.restype = ctypes.c_int
        lib.oracle_solve.argtypes = [vp, i64, i64, i64, i64, u32, ctypes.c_int,
                                     vp, i64, vp, i32p, i32p]
        lib.oracle_solve.restype = ctypes.c_int
        lib.oracle_inverse.argtypes = [u32, u32]
        lib.oracle_inverse.restype = u32
        lib.oracle_load_matrix.argtypes = [vp, i64, i64, i64, vp, i64, i64, u32, vp, i64]
        lib.oracle_load_matrix.restype = ctypes.c_int
        lib.oracle_matmul.argtypes = [vp, i64, i64, i64, vp, i64, i64, u32, vp, i64]
        lib.oracle_matmul.restype = ctypes.c_int
        u64 = ctypes.c_uint64
        lib.oracle_lup.argtypes = [vp, i64, i64, i64, u32, vp, i64, vp, i64, i32p, i32p, i32p, vp, vp, vp]
        lib.oracle_lup.restype = ctypes.c_int
        lib.oracle_rref64.argtypes = [vp, i64, i64, i64, u64, i64, ctypes.c_int, i32p, i32p]
        lib.oracle_rref64.restype = ctypes.c_int
        lib.oracle_solve64.argtypes = [vp, i64, i64, i64, i64, u64, ctypes.c_int, vp, i64, vp, i32p, i32p]
        lib.oracle_solve64.restype = ctypes.c_int
        lib.oracle_inverse64.argtypes = [u64, u64]
        lib.oracle_inverse64.restype = u64
        _lib = lib
        return lib


def _as_matrix(A) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.uint32))
    if A.ndim != 2:
        raise ValueError("expected a 2-D matrix")
    return A


def _as_matrix64(A) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.uint64))
    if A.ndim != 2:
        raise ValueError("expected a 2-D matrix")
    return A


def inverse(h: int, p: int) -> int:
    """h^(p-2) mod p (Fermat); the pivot inverse of section 3.2."""
    return int(_load().oracle_inverse(int(h), int(p)))


def rref(A, p: int, col_limit: int | None = None, max_pivots: int = -1,
         nthreads: int = 1):
    """Reduced row-echelon form of A over Z/pZ (paper section 3.2).

    Returns (R, rank, pivots, det) where R has A's shape with zero rows at the
    bottom, pivots is an int32 array of length rank, and det is
    (-1)^swaps * (product of the heads before scaling) -- det(A) for square A
    searched over all columns, 0 when the rank is short.  Pivot search is
    limited to columns [0, col_limit); max_pivots >= 0 stops early (a bounded
    sample used only for timing).
    """
    R = _as_matrix(A).copy()
    m, n = R.shape
    if col_limit is None:
        col_limit = n
    piv = np.full(max(min(m, n), 1), -1, dtype=np.int32)
    rank = ctypes.c_int32(0)
    det = ctypes.c_uint32(0)
    rc = _load().oracle_rref(R.ctypes.data, m, n, n, p, col_limit, max_pivots, nthreads,
                             ctypes.byref(rank), piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             ctypes.byref(det))
    if rc != 0:
        raise ValueError("oracle_rref rejected its arguments")
    return R, int(rank.value), piv[: rank.value].copy(), int(det.value)


def solve(A, B, p: int, nthreads: int = 1):
    """Particular solution of A X = B over Z/pZ (paper section 5.2).

    Pivots are restricted to A's columns; right-hand side j is consistent iff
    rank(A) == rank(A | b_j).  Free variables are set to zero; inconsistent
    columns of X are zero.  Returns (X, consistent, rank, pivots, reduced
    augmented matrix).
    """
    A = _as_matrix(A)
    B = _as_matrix(B)
    m, nA = A.shape
    if B.shape[0] != m:
        raise ValueError("A and B need the same number of rows")
    k = B.shape[1]
    M = np.ascontiguousarray(np.concatenate([A, B], axis=1))
    X = np.zeros((max(nA, 1), max(k, 1)), dtype=np.uint32)
    cons = np.zeros(max(k, 1), dtype=np.uint8)
    piv = np.full(max(min(m, nA + k), 1), -1, dtype=np.int32)
    rank = ctypes.c_int32(0)
    rc = _load().oracle_solve(M.ctypes.data, m, nA, k, nA + k, p, nthreads,
                              X.ctypes.data, X.shape[1], cons.ctypes.data,
                              ctypes.byref(rank),
                              piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != 0:
        raise ValueError("oracle_solve rejected its arguments")
    return (X[:nA, :k].copy(), cons[:k].astype(bool), int(rank.value),
            piv[: rank.value].copy(), M)


def lup(A, p: int):
    """LUP factorisation P A = L U (the option paper section 6 names beside
    the rank decomposition; see oracle_lup in oracle.c for the reading).

    Returns (L, U, perm, rank, pivots): L is m x min(m, n) (the first columns
    of the unit lower triangular factor), U is m x n in row-echelon form (rows
    at and beyond the rank zero), row i of P A is row perm[i] of A, and pivots
    (length rank) are the pivot columns.
    """
    A = _as_matrix(A)
    m, n = A.shape
    mn = min(m, n)
    L = np.zeros((m, max(mn, 1)), dtype=np.uint32)
    U = np.zeros((m, max(n, 1)), dtype=np.uint32)
    perm = np.zeros(max(m, 1), dtype=np.int32)
    piv = np.full(max(mn, 1), -1, dtype=np.int32)
    W = np.zeros(max(m * n, 1), dtype=np.uint32)
    Lo = np.zeros(max(m * mn, 1), dtype=np.uint32)
    isp = np.zeros(max(m, 1), dtype=np.uint8)
    rank = ctypes.c_int32(0)
    i32p = ctypes.POINTER(ctypes.c_int32)
    rc = _load().oracle_lup(A.ctypes.data, m, n, n, p, L.ctypes.data, L.shape[1], U.ctypes.data, U.shape[1],
                            perm.ctypes.data_as(i32p), ctypes.byref(rank), piv.ctypes.data_as(i32p),
                            W.ctypes.data, Lo.ctypes.data, isp.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_lup rejected its arguments")
    r = int(rank.value)
    return L[:, :mn].copy(), U[:, :n].copy(), perm[:m].copy(), r, piv[:r].copy()


def null_space(R: np.ndarray, pivots: np.ndarray, p: int) -> np.ndarray:
    """Canonical null-space basis read off an RREF (paper section 5.1).

    The non-pivot columns are the free variables; their coefficients form
    minus the identity.  Returns K (n x (n - rank)) with A K = 0 mod p.
    """
    R = np.asarray(R, dtype=np.uint64)
    n = R.shape[1]
    piv = [int(c) for c in pivots]
    free = [c for c in range(n) if c not in set(piv)]
    K = np.zeros((n, len(free)), dtype=np.uint64)
    for f_idx, f in enumerate(free):
        K[f, f_idx] = (p - 1) % p
        for t, c in enumerate(piv):
            K[c, f_idx] = R[t, f]
    return K.astype(np.uint32)


def rank_factor(A, pivots) -> np.ndarray:
    """C = A[:, J], the pivot columns of the ORIGINAL matrix (paper section
    5.1): with R the RREF without its zero rows, A = C R is a rank
    factorisation."""
    A = _as_matrix(A)
    J = np.asarray(pivots, dtype=np.int64)
    return np.ascontiguousarray(A[:, J])


def load_matrix(bases, lindices, p: int) -> np.ndarray:
    """A[r][c] = prod_t bases[r][lindices[c][t]] mod p (paper sections 2.3 and
    3.3: rows are sampling points, columns monomials)."""
    bases = _as_matrix(bases)
    L = np.ascontiguousarray(np.asarray(lindices, dtype=np.int32))
    if L.ndim != 2:
        raise ValueError("lindices must be n_cols x d")
    n_rows, n_basis = bases.shape
    n_cols, d = L.shape
    A = np.zeros((n_rows, max(n_cols, 1)), dtype=np.uint32)
    rc = _load().oracle_load_matrix(bases.ctypes.data, n_rows, n_basis, n_basis, L.ctypes.data,
                                    n_cols, d, p, A.ctypes.data, A.shape[1])
    if rc != 0:
        raise ValueError("oracle_load_matrix rejected its arguments")
    return A[:, :n_cols].copy()


def matmul(A, B, p: int) -> np.ndarray:
    """A B mod p, every product reduced before it is added."""
    A = _as_matrix(A)
    B = _as_matrix(B)
    m, K = A.shape
    if B.shape[0] != K:
        raise ValueError("inner dimensions differ")
    n = B.shape[1]
    C = np.zeros((m, max(n, 1)), dtype=np.uint32)
    rc = _load().oracle_matmul(A.ctypes.data, m, K, K, B.ctypes.data, n, n, p, C.ctypes.data, C.shape[1])
    if rc != 0:
        raise ValueError("oracle_matmul rejected its arguments")
    return C[:, :n].copy()


def eval_template(points, coefs, monomials, mask, p: int) -> np.ndarray:
    """Evaluate a template of polynomial entries at many points (paper
    section 3.3: a system is built by evaluating the same monomials at
    different numerical points).

    points: count x nv residues (one row per point); monomials: list of
    exponent tuples, one per monomial; coefs: nnz x n_monomials coefficients
    of the template's nonzero entries, in row-major order of the boolean
    mask (rows x cols).  Each monomial's value at a point is a load_matrix
    product of the point's variables (exponents unrolled into repeated
    indices, padded with the constant 1); entry values are the monomial
    values times the coefficients, summed mod p.  Returns count x rows x cols.
    """
    pts = _as_matrix(points)
    count, nv = pts.shape
    bases = np.concatenate([np.ones((count, 1), dtype=np.uint32), pts], axis=1)
    deg = max(sum(e) for e in monomials)
    lind = np.zeros((len(monomials), max(deg, 1)), dtype=np.int32)
    for u, e in enumerate(monomials):
        idx = [1 + v for v in range(nv) for _ in range(e[v])]
        lind[u, :len(idx)] = idx
    V = load_matrix(bases, lind, p)                               # count x n_monomials
    vals = matmul(V, np.ascontiguousarray(np.asarray(coefs, dtype=np.uint32).T), p)   # count x nnz
    mask = np.asarray(mask, dtype=bool)
    out = np.zeros((count,) + mask.shape, dtype=np.uint32)
    out[:, mask] = vals
    return out


# ---------------------------------------------------------------------------
# 64-bit residues (paper section 2.3: uint64 storage for primes that do not
# fit 32 bits, up to 2^64 - 1)

def inverse64(h: int, p: int) -> int:
    """h^(p-2) mod p for a 64-bit prime p (Fermat)."""
    return int(_load().oracle_inverse64(int(h), int(p)))


def rref64(A, p: int, col_limit: int | None = None, nthreads: int = 1):
    """RREF over Z/pZ of a uint64 matrix, 3 <= p < 2^64 prime (section 3.2's
    column loop with 128-bit products).  Returns (R, rank, pivots)."""
    R = _as_matrix64(A).copy()
    m, n = R.shape
    if col_limit is None:
        col_limit = n
    piv = np.full(max(min(m, n), 1), -1, dtype=np.int32)
    rank = ctypes.c_int32(0)
    rc = _load().oracle_rref64(R.ctypes.data, m, n, n, p, col_limit, nthreads, ctypes.byref(rank),
                               piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != 0:
        raise ValueError("oracle_rref64 rejected its arguments")
    return R, int(rank.value), piv[: rank.value].copy()


def solve64(A, B, p: int, nthreads: int = 1):
    """Particular solution of A X = B over Z/pZ with uint64 residues
    (section 5.2).  Returns (X, consistent, rank, pivots, reduced [A | B])."""
    A = _as_matrix64(A)
    B = _as_matrix64(B)
    m, nA = A.shape
    if B.shape[0] != m:
        raise ValueError("A and B need the same number of rows")
    k = B.shape[1]
    M = np.ascontiguousarray(np.concatenate([A, B], axis=1))
    X = np.zeros((max(nA, 1), max(k, 1)), dtype=np.uint64)
    cons = np.zeros(max(k, 1), dtype=np.uint8)
    piv = np.full(max(min(m, nA + k), 1), -1, dtype=np.int32)
    rank = ctypes.c_int32(0)
    rc = _load().oracle_solve64(M.ctypes.data, m, nA, k, nA + k, p, nthreads, X.ctypes.data, X.shape[1],
                                cons.ctypes.data, ctypes.byref(rank),
                                piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != 0:
        raise ValueError("oracle_solve64 rejected its arguments")
    return (X[:nA, :k].copy(), cons[:k].astype(bool), int(rank.value), piv[: rank.value].copy(), M)


def null_space64(R, pivots, p: int) -> np.ndarray:
    """Canonical null-space basis of a uint64 RREF (section 5.1): for the q-th
    free column f, -1 (that is, p - 1) in row f and R[t][f] in row pivots[t]."""
    R = _as_matrix64(R)
    n = R.shape[1]
    piv = [int(c) for c in pivots]
    free = [c for c in range(n) if c not in set(piv)]
    K = np.zeros((n, len(free)), dtype=np.uint64)
    for q, f in enumerate(free):
        K[f, q] = p - 1
        for t, c in enumerate(piv):
            K[c, q] = R[t, f]
    return K


def rank_factor64(A, pivots) -> np.ndarray:
    """C = A[:, J] for uint64 residues (section 5.1: A = C R)."""
    A = _as_matrix64(A)
    return np.ascontiguousarray(A[:, np.asarray(pivots, dtype=np.int64)])
