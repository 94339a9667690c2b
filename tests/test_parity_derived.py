"""GPU parity of system construction and of the outputs read off an RREF,
bit for bit against the CPU oracle:

* linac_load_matrix: A[r][c] = prod_t bases[r][lindices[c][t]] mod p (paper
  sections 2.3 and 3.3), both the shared-memory and the global-memory basis
  paths, ragged tiles, d = 0, and an out-of-range index (written as 0, status
  LINAC_ERR_RANGE, nothing read out of bounds);
* linac_matmul: A B mod p at ragged sizes, K = 0, entries p - 1 everywhere and
  a prime whose 2^32 mod p is large (the fold's worst case);
* the template pipeline: monomial values of many points (load_matrix) times a
  block-banded template's coefficients (matmul) gives the shared-pattern
  batch, then its RREF;
* linac_null_space and linac_rank_factor (section 5.1) against the oracle's
  null space and rank factor, plus A K = 0 and A = C R on the device at
  4096 x 4160.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_25863_gb300 import linac, synth

pytestmark = pytest.mark.gpu

P31 = synth.P31
PB = synth.P_BATCH
NTH = min(16, os.cpu_count() or 1)


def _is_prime(n):
    if n < 2:
        return False
    for q in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % q == 0:
            return n == q
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7, 11, 13, 17):
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


def _prime_above(x):
    x += 1
    while not _is_prime(x):
        x += 1
    return x


# 2^32 mod p = 2^32 - 2p is about p for p just above 2^32 / 3: the largest
# fold multiplier among primes below 2^31
P_BIGFOLD = _prime_above((1 << 32) // 3)


def host(t):
    return t.cpu().numpy().view(np.uint32)


def dev_int32(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.int32))).cuda()


@pytest.mark.parametrize("p", [3, P31, PB])
@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (37, 5, 300, 4), (129, 40, 1000, 7), (20, 2000, 70, 3),
                                   (9, 3, 15, 0), (300, 64, 257, 12)])
def test_load_matrix_vs_oracle(shape, p):
    n_rows, n_basis, n_cols, d = shape
    g = np.random.default_rng(n_rows * 7 + n_cols + d)
    bases = synth.uniform((n_rows, n_basis), p, synth.stream_key(n_rows + n_basis, "lm_bases"))
    lind = g.integers(0, n_basis, size=(n_cols, d), dtype=np.int64).astype(np.int32)
    A = linac.linac_load_matrix(linac.to_device(bases), dev_int32(lind), p)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 0
    want = oracle.load_matrix(bases, lind, p)
    assert np.array_equal(host(A), want)


def test_load_matrix_rejects_bad_index_without_reading_it():
    p = P31
    bases = synth.uniform((16, 6), p, synth.stream_key(1, "lm_bad"))
    lind = np.array([[0, 1], [2, 6], [5, -1], [3, 3]], dtype=np.int32)   # columns 1, 2 name no basis value
    A = linac.linac_load_matrix(linac.to_device(bases), dev_int32(lind), p)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 7   # LINAC_ERR_RANGE
    got = host(A)
    ok = oracle.load_matrix(bases, lind[[0, 3]], p)
    assert np.array_equal(got[:, [0, 3]], ok)
    assert not got[:, [1, 2]].any()


@pytest.mark.parametrize("p", [3, 65537, P31, PB, P_BIGFOLD])
@pytest.mark.parametrize("shape", [(1, 1, 1), (130, 17, 70), (257, 100, 129), (64, 0, 5), (3, 300, 2)])
def test_matmul_vs_oracle(shape, p):
    m, K, n = shape
    A = synth.uniform((m, K), p, synth.stream_key(m + K, "mm_a"))
    B = synth.uniform((K, n), p, synth.stream_key(K + n, "mm_b"))
    C = linac.linac_matmul(linac.to_device(A), linac.to_device(B), p)
    torch.cuda.synchronize()
    assert np.array_equal(host(C), oracle.matmul(A, B, p))


@pytest.mark.parametrize("p", [3, 65537, P31, PB, P_BIGFOLD])
def test_matmul_extreme_entries(p):
    # balanced residues of magnitude (p-1)/2: (p-1)/2 is +half, (p+1)/2 is -half,
    # so even rows of A times B give +half^2 per product and odd rows -half^2,
    # the accumulator bounds' worst cases in both directions, at K = 257
    half = (p - 1) // 2
    A = np.full((129, 257), half, dtype=np.uint32)
    A[1::2] = (p + 1) // 2
    B = np.full((257, 65), (p + 1) // 2, dtype=np.uint32)
    B[:, 1::2] = half
    C = linac.linac_matmul(linac.to_device(A), linac.to_device(B), p)
    torch.cuda.synchronize()
    assert np.array_equal(host(C), oracle.matmul(A, B, p))


def _template_inputs(count):
    mask, coefs, mons = synth.shared_pattern_template()
    p = P31
    pts = synth.uniform((count, 2), p, synth.stream_key(4, "sp_points"))
    rows, cols = mask.shape
    # dense coefficient matrix: one row per monomial, one column per template entry
    Cd = np.zeros((len(mons), rows * cols), dtype=np.uint32)
    flat = np.flatnonzero(mask.ravel())
    Cd[:, flat] = coefs.T
    deg = max(a + b for a, b in mons)
    lind = np.zeros((len(mons), deg), dtype=np.int32)
    for u, (a, b) in enumerate(mons):
        idx = [1] * a + [2] * b
        lind[u, :len(idx)] = idx
    bases = np.concatenate([np.ones((count, 1), dtype=np.uint32), pts], axis=1)
    return p, mask, coefs, mons, pts, bases, lind, Cd


def test_template_pipeline_vs_oracle():
    count = 48
    p, mask, coefs, mons, pts, bases, lind, Cd = _template_inputs(count)
    rows, cols = mask.shape
    V = linac.linac_load_matrix(linac.to_device(bases), dev_int32(lind), p)
    out = linac.padded(count, rows * cols)
    linac.linac_matmul(V, linac.to_device(Cd), p, out=out)
    torch.cuda.synchronize()
    got = host(out).reshape(count, rows, cols)
    want = oracle.eval_template(pts, coefs, mons, mask, p)
    assert np.array_equal(got, want)
    # the constructed systems reduce exactly as the oracle reduces its own
    data = out.contiguous().view(-1)
    offs = torch.arange(count, dtype=torch.int64, device="cuda") * (rows * cols)
    mm = torch.full((count,), rows, dtype=torch.int32, device="cuda")
    nn = torch.full((count,), cols, dtype=torch.int32, device="cuda")
    ns = torch.full((count,), cols - 16, dtype=torch.int32, device="cuda")
    ranks, piv, poff, st = linac.linac_rref_batched(data, offs, mm, nn, nn.clone(), p, nsearch=ns,
                                                     flags=linac.LINAC_SHARED_PATTERN)
    torch.cuda.synchronize()
    red = data.cpu().numpy().view(np.uint32).reshape(count, rows, cols)
    for s in (0, 1, count - 1):
        R0, r0, piv0, _ = oracle.rref(want[s], p, col_limit=cols - 16, nthreads=NTH)
        assert int(ranks[s].item()) == r0 == rows
        assert np.array_equal(red[s], R0)


def _rref_on_gpu(M, p):
    A = linac.to_device(M)
    rank, piv = linac.linac_rref(A, p)
    return A, rank, piv


@pytest.mark.parametrize("p", [5, P31, PB])
@pytest.mark.parametrize("mnd", [(40, 60, 15), (60, 40, 0), (50, 50, 50), (1, 1, 1), (200, 230, 9),
                                 (130, 300, 70)])
def test_null_space_and_rank_factor_vs_oracle(mnd, p):
    m, n, d = mnd
    if d >= m:
        M = np.zeros((m, n), dtype=np.uint32)
    else:
        M, _ = synth.rank_deficient(m=m, n=n, d=d, p=p, seed=m + n + d)
    R, rank, piv = _rref_on_gpu(M, p)
    K, free, nullity = linac.linac_null_space(R, rank, piv, p)
    C = linac.linac_rank_factor(linac.to_device(M), rank, piv)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 0
    R0, r0, piv0, _ = oracle.rref(M, p, nthreads=NTH)
    assert int(rank.item()) == r0
    assert int(nullity.item()) == n - r0
    K0 = oracle.null_space(R0, piv0, p)
    assert np.array_equal(host(K)[:, :n - r0], K0)
    assert not host(K)[:, n - r0:].any()
    fr = free.cpu().numpy()
    assert np.array_equal(fr[:n - r0], np.setdiff1d(np.arange(n), piv0))
    assert (fr[n - r0:] == -1).all()
    C0 = oracle.rank_factor(M, piv0)
    assert np.array_equal(host(C)[:, :r0], C0)
    assert not host(C)[:, r0:].any()
    if r0:
        assert np.array_equal(oracle.matmul(C0, R0[:r0], p), M)     # A = C R
    if n - r0:
        assert not oracle.matmul(M, K0, p).any()                     # A K = 0


def test_null_space_column_bound_reports_range():
    p = P31
    M, _ = synth.rank_deficient(m=64, n=80, d=10, p=p, seed=3)      # nullity 26
    R, rank, piv = _rref_on_gpu(M, p)
    K, free, nullity = linac.linac_null_space(R, rank, piv, p, kcols=8)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 7
    assert int(nullity.item()) == 26
    R0, r0, piv0, _ = oracle.rref(M, p)
    assert np.array_equal(host(K), oracle.null_space(R0, piv0, p)[:, :8])


def test_null_space_and_rank_factor_identities_at_4096():
    """4096 x 4160 with 64 rows replaced by combinations (rank 4032, nullity
    128): A K = 0 and C R = A on the device through linac_matmul."""
    p = P31
    M, _ = synth.rank_deficient(m=4096, n=4160, d=64, p=p, seed=2)
    A0 = linac.to_device(M)
    R, rank, piv = _rref_on_gpu(M, p)
    K, free, nullity = linac.linac_null_space(R, rank, piv, p, kcols=128)
    C = linac.linac_rank_factor(A0, rank, piv, ccols=4032)
    AK = linac.linac_matmul(A0, K, p)
    CR = linac.linac_matmul(C, R[:4032], p)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 0
    assert int(rank.item()) == 4032 and int(nullity.item()) == 128
    assert not host(AK).any()
    assert torch.equal(CR, A0)
    # sampled rows of A K on the CPU, through the oracle's product
    Kh = host(K)
    for i in (0, 1777, 4095):
        assert not oracle.matmul(M[i:i + 1], Kh, p).any()
