"""GPU parity of linac_lup (P A = L U, the option of paper section 6) with
the oracle's LUP, bit for bit: P, L, U, rank and pivots, on shapes that span
several panels with ragged tails, rank-deficient, tall and wide matrices,
small primes (many vanishing entries and pivot rows from deep in the list)
and panels whose pivot window lacks a pivot (the grid-wide search).  One
larger case also checks P A = L U on the device with linac_matmul."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_25863_gb300 import linac, synth

pytestmark = pytest.mark.gpu

NTH = min(16, os.cpu_count() or 1)
P31 = synth.P31


def check_lup(M, p):
    A = linac.to_device(M)
    L, U, perm, rank, piv = linac.linac_lup(A, p)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 0
    L0, U0, perm0, r0, piv0 = oracle.lup(M, p)
    r = int(rank.item())
    assert r == r0
    pv = piv.cpu().numpy()
    assert np.array_equal(pv[:r], piv0) and (pv[r:] == -1).all()
    assert np.array_equal(perm.cpu().numpy(), perm0)
    assert np.array_equal(U.cpu().numpy().view(np.uint32), U0)
    assert np.array_equal(L.cpu().numpy().view(np.uint32), L0)
    assert np.array_equal(A.cpu().numpy().view(np.uint32), M)   # the input is left alone
    return r


@pytest.mark.parametrize("p", [3, 251, 65537, P31, 1431655777])
@pytest.mark.parametrize("shape", [(1, 1), (5, 3), (3, 5), (64, 64), (100, 257), (257, 100), (300, 300),
                                   (513, 700)])
def test_lup_uniform_vs_oracle(shape, p):
    m, n = shape
    M = synth.uniform(shape, p, synth.stream_key(m * 1013 + n, f"lup{p}"))
    check_lup(M, p)


@pytest.mark.parametrize("mnd", [(600, 640, 25), (700, 600, 40), (400, 900, 0), (2100, 2200, 30)])
def test_lup_rank_deficient_vs_oracle(mnd):
    m, n, d = mnd
    M, _ = synth.rank_deficient(m=m, n=n, d=d, p=P31, seed=m + d)
    assert check_lup(M, P31) == min(m - d, n)


def test_lup_window_fallback_and_zero_columns():
    """Column 3 vanishes in the first 300 rows and columns 100..160 vanish
    everywhere: the first panel's pivot window lacks a pivot (the grid-wide
    search runs on the row list), later panels have no pivot in some columns."""
    M = synth.uniform((700, 400), 65537, synth.stream_key(3, "lup_fallback"))
    M[:300, 3] = 0
    M[:, 100:160] = 0
    check_lup(M, 65537)


def test_lup_special_matrices():
    check_lup(np.zeros((70, 90), dtype=np.uint32), P31)
    I = np.eye(150, dtype=np.uint32)
    check_lup(I[::-1].copy(), P31)
    check_lup(I[np.random.default_rng(4).permutation(150)], P31)
    check_lup(np.full((40, 50), P31 - 1, dtype=np.uint32), P31)
    check_lup(np.repeat(synth.uniform((1, 90), P31, 77), 33, axis=0), P31)


@pytest.mark.parametrize("p", [P31, 7])
def test_lup_product_on_device(p):
    """P A = L U at 1500 x 1600 (the oracle's factors compared too): the
    product L U[:min(m, n)] on linac_matmul equals A's rows in P's order."""
    M, _ = synth.rank_deficient(m=1500, n=1600, d=12, p=p, seed=5)
    r = check_lup(M, p)
    A = linac.to_device(M)
    L, U, perm, rank, piv = linac.linac_lup(A, p)
    LU = linac.linac_matmul(L, U[:min(M.shape)], p)
    PA = A[perm.long()]
    torch.cuda.synchronize()
    assert torch.equal(LU, PA)
