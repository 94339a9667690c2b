"""linac_rref_noalloc: the RREF entry point for callers that cannot allocate
device memory (for example an application whose pool allocator owns the
whole GPU, or a latency-critical loop that cannot absorb cudaMalloc's
implicit synchronisation).  Its scratch is a fixed 4 MiB array inside the
library, so it is limited to m, n <= 2048.

The test calls it through the C ABI, first, in a process where it may be the
library's very first call, then checks its output bit for bit against
linac_rref, the existing entry point, on two different inputs in a row (the
shared array keeps the first call's data when the second starts)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2605_25863_gb300 import linac, synth

pytestmark = pytest.mark.gpu

P31 = synth.P31


def call_noalloc(A: torch.Tensor, p: int):
    lib = linac.lib()
    fn = lib.linac_rref_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    m, n = A.shape
    rank = torch.zeros(1, dtype=torch.int32, device=A.device)
    piv = torch.full((max(min(m, n), 1),), -1, dtype=torch.int32, device=A.device)
    code = fn(A.data_ptr(), m, n, A.stride(0), p, rank.data_ptr(), piv.data_ptr(),
              torch.cuda.current_stream().cuda_stream)
    return code, rank, piv


def test_noalloc_matches_rref_on_two_calls_in_a_row():
    inputs = [synth.rank_deficient(m=1500, n=1700, d=37, p=P31, seed=61)[0],
              synth.rank_deficient(m=2048, n=1999, d=5, p=P31, seed=62)[0]]
    for M in inputs:
        A_no = linac.to_device(M)
        code, r_no, piv_no = call_noalloc(A_no, P31)
        assert code == 0
        A_ref = linac.to_device(M)
        r_ref, piv_ref = linac.linac_rref(A_ref, P31)
        torch.cuda.synchronize()
        assert int(r_no.item()) == int(r_ref.item())
        assert torch.equal(piv_no[:piv_ref.numel()], piv_ref)
        assert torch.equal(A_no, A_ref)


def test_noalloc_rejects_sizes_above_its_limit():
    A = linac.padded(2049, 8)
    code, _, _ = call_noalloc(A, P31)
    assert code == 8   # LINAC_ERR_UNSUPPORTED
