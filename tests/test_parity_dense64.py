"""GPU parity of the uint64 elimination (primes below 2^64, paper section 2.3)
against the CPU oracle, bit for bit:

* RREF, rank and pivots at seven primes from 3 to 2^64 - 59, at sizes that
  span several 32-column panels and 48-row windows with ragged tails, square,
  wide, tall and rank-deficient;
* structured inputs that force the full-height pivot search: the window's
  rows are zero in the panel columns while lower rows are not, zero columns,
  duplicated rows, the zero matrix, p - 1 everywhere;
* the pivot-search limit (ncols_search) and solve (section 5.2): X,
  consistency flags, rank and pivots;
* for primes below 2^31, the uint64 path agrees with the uint32 path;
* 1024 x 1056 against the oracle, and at 4096 x 4097 the identity block and
  A x = b on sampled rows checked with Python integers;
* the range validation option, and a capture into a CUDA graph (the panel
  kernels run on a second stream forked from the caller's);
* null space and rank factorisation of uint64 RREFs (section 5.1) against the
  oracle's.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_25863_gb300 import linac, synth

pytestmark = pytest.mark.gpu

P64 = [3, 5, 2**31 - 1, 2**32 + 15, 2**61 - 1, 2**63 - 25, 2**64 - 59]
NTH = min(16, os.cpu_count() or 1)


def run(M, p, ncols_search=None):
    A = linac.to_device64(M)
    rank, piv = linac.linac_rref64(A, p, ncols_search=ncols_search)
    torch.cuda.synchronize()
    return linac.host64(A), int(rank.item()), piv.cpu().numpy()


def check(M, p, ncols_search=None):
    got, rank, piv = run(M, p, ncols_search)
    R0, r0, piv0 = oracle.rref64(M, p, col_limit=ncols_search, nthreads=NTH)
    assert rank == r0
    assert np.array_equal(piv[:r0], piv0)
    assert (piv[r0:] == -1).all()
    assert np.array_equal(got, R0)


@pytest.mark.parametrize("p", P64)
@pytest.mark.parametrize("mnd", [(1, 1, 0), (5, 3, 0), (3, 5, 0), (40, 70, 6), (100, 33, 0), (33, 100, 0),
                                 (129, 161, 9), (200, 200, 0), (97, 97, 40), (300, 40, 0)])
def test_rref64_vs_oracle(mnd, p):
    m, n, d = mnd
    if d:
        M, _ = synth.rank_deficient64(m, n, d, p, seed=m + 3 * n + d)
    else:
        M = synth.uniform64((m, n), p, synth.stream_key(m * 1000 + n, "r64"))
    check(M, p)


@pytest.mark.parametrize("p", [5, 2**31 - 1, 2**64 - 59])
def test_full_height_search_when_window_rows_vanish(p):
    # rows 0..99 are zero in every column, so the 48-row window holds no pivot
    M = np.zeros((300, 70), dtype=np.uint64)
    M[100:] = synth.uniform64((200, 70), p, synth.stream_key(11, "low64"))
    M[:, 5] = 0                      # a zero column inside the first panel
    M[250] = M[180]                  # a duplicated row
    M[7, 40] = 1                     # a single entry high up in the second panel
    check(M, p)


@pytest.mark.parametrize("p", [3, 2**63 - 25, 2**64 - 59])
def test_special_matrices(p):
    check(np.zeros((50, 45), dtype=np.uint64), p)
    check(np.full((70, 90), p - 1, dtype=np.uint64), p)
    check(np.eye(65, dtype=np.uint64), p)
    M = synth.uniform64((60, 80), p, synth.stream_key(3, "dup64"))
    M[30:] = M[:30]
    check(M, p)
    # alternating p - 1 and 1: every product in the update is (p-1)^2 or 1
    B = np.ones((90, 96), dtype=np.uint64)
    B[::2, ::3] = p - 1
    B[1::3, 1::2] = p - 1
    check(B, p)


@pytest.mark.parametrize("p", [2**31 - 1, 2**64 - 59])
def test_ncols_search_limit(p):
    M = synth.uniform64((50, 90), p, synth.stream_key(5, "ns64"))
    check(M, p, ncols_search=37)
    check(M, p, ncols_search=0)


@pytest.mark.parametrize("p", [7, 2**32 + 15, 2**64 - 59])
@pytest.mark.parametrize("mnk", [(64, 64, 3), (80, 50, 2), (50, 80, 4), (120, 100, 1)])
def test_solve64_vs_oracle(mnk, p):
    m, nA, k = mnk
    M, _ = synth.rank_deficient64(m, nA + k, min(m, nA) // 8, p, seed=m + nA + k)
    A, B = M[:, :nA].copy(), M[:, nA:].copy()
    B[:, -1] = synth.uniform64((m,), p, synth.stream_key(m, "rhs64"))   # generally inconsistent
    X, cons, rank, piv = linac.linac_solve64(linac.to_device64(A), linac.to_device64(B), p)
    torch.cuda.synchronize()
    X0, cons0, r0, piv0, _ = oracle.solve64(A, B, p, nthreads=NTH)
    assert int(rank.item()) == r0
    assert np.array_equal(piv.cpu().numpy()[:r0], piv0)
    assert np.array_equal(cons.cpu().numpy(), cons0)
    assert np.array_equal(linac.host64(X), X0)


@pytest.mark.parametrize("p", [3, 65537, 2**31 - 1, 2147483629])
def test_agrees_with_uint32_path(p):
    M, _ = synth.rank_deficient(m=150, n=170, d=12, p=p, seed=9)
    A32 = linac.to_device(M)
    r32, piv32 = linac.linac_rref(A32, p)
    got64, r64, piv64 = run(M.astype(np.uint64), p)
    assert r64 == int(r32.item())
    assert np.array_equal(piv64, piv32.cpu().numpy())
    assert np.array_equal(got64, A32.cpu().numpy().view(np.uint32).astype(np.uint64))


def test_1024_vs_oracle():
    p = 2**64 - 59
    M, _ = synth.rank_deficient64(1024, 1056, 16, p, seed=21)
    check(M, p)


def test_4096_identity_and_sampled_solution():
    """[A | b], A 4096 x 4096 uniform: RREF = [I | x] (rank 4096 whp), and
    A x = b holds on sampled rows in exact integer arithmetic."""
    p = 2**64 - 59
    n = 4096
    M = synth.uniform64((n, n + 1), p, synth.stream_key(4096, "big64"))
    got, rank, piv = run(M, p)
    assert rank == n
    assert np.array_equal(piv, np.arange(n))
    assert np.array_equal(got[:, :n], np.eye(n, dtype=np.uint64))
    x = [int(v) for v in got[:, n]]
    for i in (0, 1, 2047, 4095):
        row = [int(v) for v in M[i, :n]]
        assert sum(a * b for a, b in zip(row, x)) % p == int(M[i, n])


def test_validate_flags_entries_not_below_p():
    p = 2**61 - 1
    M = synth.uniform64((20, 20), p, synth.stream_key(1, "val64"))
    M[3, 4] = p
    A = linac.to_device64(M)
    linac.linac_rref64(A, p, validate=True)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 7


def test_rref64_captured_in_a_cuda_graph():
    """The panel kernels run on a second stream forked from the caller's;
    the fork and join must hold inside a CUDA graph capture too."""
    p = 2**61 - 1
    M, _ = synth.rank_deficient64(200, 230, 7, p, seed=8)
    R0, r0, piv0 = oracle.rref64(M, p, nthreads=NTH)
    src = linac.to_device64(M)
    A = src.clone()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        linac.linac_rref64(A, p)        # uncaptured call on this stream: scratch exists
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rank, piv = linac.linac_rref64(A, p)
    for _ in range(2):
        A.copy_(src)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert int(rank.item()) == r0
        assert np.array_equal(piv.cpu().numpy()[:r0], piv0)
        assert np.array_equal(linac.host64(A), R0)


@pytest.mark.parametrize("p", [5, 2**32 + 15, 2**64 - 59])
@pytest.mark.parametrize("mnd", [(40, 60, 15), (60, 40, 0), (50, 50, 50), (130, 300, 70), (1, 1, 0)])
def test_null_space64_and_rank_factor64_vs_oracle(mnd, p):
    m, n, d = mnd
    if d >= m:
        M = np.zeros((m, n), dtype=np.uint64)
    else:
        M, _ = synth.rank_deficient64(m, n, d, p, seed=m + n + d)
    A0 = linac.to_device64(M)
    R = A0.clone()
    rank, piv = linac.linac_rref64(R, p)
    K, free, nullity = linac.linac_null_space64(R, rank, piv, p)
    C = linac.linac_rank_factor64(A0, rank, piv)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 0
    R0, r0, piv0 = oracle.rref64(M, p, nthreads=NTH)
    assert int(rank.item()) == r0 and int(nullity.item()) == n - r0
    Kh = linac.host64(K)
    assert np.array_equal(Kh[:, :n - r0], oracle.null_space64(R0, piv0, p))
    assert not Kh[:, n - r0:].any()
    fr = free.cpu().numpy()
    assert np.array_equal(fr[:n - r0], np.setdiff1d(np.arange(n), piv0))
    assert (fr[n - r0:] == -1).all()
    Ch = linac.host64(C)
    assert np.array_equal(Ch[:, :r0], oracle.rank_factor64(M, piv0))
    assert not Ch[:, r0:].any()
