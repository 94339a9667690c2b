"""linac_rref_host: the RREF of a matrix in page-locked host memory with the
transfers inside the call, compared bit for bit with the oracle (section 3.2
elimination, section 2.3 output shape)."""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_25863_gb300 import linac, synth

NTH = min(16, os.cpu_count() or 1)
P31 = synth.P31


def host_matrix(M):
    H = linac.padded_host(*M.shape)
    H.copy_(torch.from_numpy(np.ascontiguousarray(M).view(np.int32)))
    return H


@pytest.mark.gpu
@pytest.mark.parametrize("shape_d", [((900, 950), 17), ((300, 257), 0), ((129, 700), 3), ((1, 5), 0)])
def test_host_rref_vs_oracle(shape_d):
    (m, n), d = shape_d
    M = synth.rank_deficient(m=m, n=n, d=d, p=P31, seed=m + n)[0] if d else \
        synth.uniform((m, n), P31, synth.stream_key(m * 3 + n, "host_io"))
    H = host_matrix(M)
    rank, piv = linac.linac_rref_host(H, P31)
    torch.cuda.synchronize()
    R0, r0, piv0, _ = oracle.rref(M, P31, nthreads=NTH)
    assert int(rank.item()) == r0
    assert np.array_equal(piv.numpy()[:r0], piv0) and (piv.numpy()[r0:] == -1).all()
    assert np.array_equal(H.numpy().view(np.uint32), R0)


@pytest.mark.gpu
def test_host_rref_calls_in_a_row_and_on_a_side_stream():
    s = torch.cuda.Stream()
    for i, (m, n) in enumerate([(600, 640), (1200, 700), (64, 2000)]):
        M = synth.uniform((m, n), 65537, synth.stream_key(i, "host_io_row"))
        H = host_matrix(M)
        rank, piv = linac.linac_rref_host(H, 65537, stream=s)
        s.synchronize()
        R0, r0, piv0, _ = oracle.rref(M, 65537, nthreads=NTH)
        assert int(rank.item()) == r0 and np.array_equal(piv.numpy()[:r0], piv0)
        assert np.array_equal(H.numpy().view(np.uint32), R0)


@pytest.mark.gpu
def test_host_rref_rejects_pageable_memory():
    lib = linac.lib()
    A = np.zeros((8, 8), dtype=np.uint32)
    rank = np.zeros(1, dtype=np.int32)
    piv = np.zeros(8, dtype=np.int32)
    code = lib.linac_rref_host(A.ctypes.data, 8, 8, 8, P31, rank.ctypes.data, piv.ctypes.data, None)
    assert code == 1   # LINAC_ERR_ARG: not page-locked


def test_host_rref_argument_checks():
    """CPU: shape, alignment and prime errors come back before any CUDA call."""
    from paper_2605_25863_gb300 import build
    build.build()
    lib = linac.lib()
    fake = ctypes.c_void_p(0x1000)
    assert lib.linac_rref_host(fake, -1, 4, 4, P31, fake, fake, None) == 1
    assert lib.linac_rref_host(fake, 4, 5, 6, P31, fake, fake, None) == 3
    assert lib.linac_rref_host(fake, 4, 4, 4, 15, fake, fake, None) == 2
