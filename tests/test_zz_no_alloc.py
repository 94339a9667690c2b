"""linac_rref_noalloc: the RREF entry point for callers that cannot allocate
device memory (for example an application whose pool allocator owns the
whole GPU, or a latency-critical loop that cannot absorb cudaMalloc's
implicit synchronisation).  Its scratch is a fixed 4 MiB array inside the
library, so it is limited to m, n <= 2048.

The tests call it through the C ABI and compare its output bit for bit with
the oracle and with linac_rref, the existing entry point, on several inputs
in a row (the shared array keeps the previous call's data when the next one
starts), with output buffers filled with junk first so that stale pivots
would show.  One test runs it in a fresh Python process as the library's
very first call, where it looks up the array's device address.  This file is
named to be collected last, so a run that stops at the first failure has
already run every other test.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2605_25863_gb300 import linac, synth

pytestmark = pytest.mark.gpu

P31 = synth.P31
NTH = min(16, os.cpu_count() or 1)
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def call_noalloc(A: torch.Tensor, p: int, junk: bool = True):
    lib = linac.lib()
    fn = lib.linac_rref_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    m, n = A.shape
    fill = 12345 if junk else -1
    rank = torch.full((1,), fill, dtype=torch.int32, device=A.device)
    piv = torch.full((max(min(m, n), 1),), fill, dtype=torch.int32, device=A.device)
    code = fn(A.data_ptr(), m, n, A.stride(0), p, rank.data_ptr(), piv.data_ptr(),
              torch.cuda.current_stream().cuda_stream)
    return code, rank, piv


def check_one(M, p):
    m, n = M.shape
    A_no = linac.to_device(M)
    code, r_no, piv_no = call_noalloc(A_no, p)
    assert code == 0
    A_ref = linac.to_device(M)
    r_ref, piv_ref = linac.linac_rref(A_ref, p)
    torch.cuda.synchronize()
    R0, r0, piv0, _ = oracle.rref(M, p, nthreads=NTH)
    rank = int(r_no.item())
    piv_no = piv_no.cpu().numpy()[:min(m, n)]
    assert rank == int(r_ref.item()) == r0
    assert np.array_equal(piv_no[:rank], piv0) and (piv_no[rank:] == -1).all()
    assert np.array_equal(piv_no, piv_ref.cpu().numpy())
    got = A_no.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, R0)
    assert torch.equal(A_no, A_ref)


def test_noalloc_matches_oracle_and_rref_on_calls_in_a_row():
    inputs = [synth.rank_deficient(m=1500, n=1700, d=37, p=P31, seed=61)[0],
              synth.rank_deficient(m=2048, n=1999, d=5, p=P31, seed=62)[0],
              # full-rank wide: the panels run out of rows before columns
              synth.uniform((256, 257), P31, synth.stream_key(63, "noalloc_wide")),
              # short and wide: one window holds every row
              synth.uniform((100, 2048), P31, synth.stream_key(64, "noalloc_short")),
              # a window that lacks a pivot: the grid-wide search runs
              synth.uniform((700, 400), P31, synth.stream_key(65, "noalloc_fallback"))]
    inputs[-1][:300, 5] = 0
    for M in inputs:
        check_one(M, P31)


def test_noalloc_rejects_sizes_above_its_limit():
    A = linac.padded(2049, 8)
    code, _, _ = call_noalloc(A, P31)
    assert code == 8   # LINAC_ERR_UNSUPPORTED


def test_noalloc_reports_a_wait_that_ran_out_as_negative_rank():
    """A device-side wait that gives up is reported through the rank output
    (-LINAC_ERR_TIMEOUT); the next call is exact again."""
    M = synth.uniform((600, 300), P31, synth.stream_key(66, "noalloc_timeout"))
    M[:300, 3] = 0          # the first panel's window lacks a pivot in column 3
    linac.linac_set_wait_limit(200_000)
    linac.linac_debug_inject_wait_failure(True)
    try:
        A = linac.to_device(M)
        code, rank, _ = call_noalloc(A, P31)
        torch.cuda.synchronize()
        assert code == 0 and int(rank.item()) == -6
    finally:
        linac.linac_debug_inject_wait_failure(False)
        linac.linac_set_wait_limit(0)
    check_one(M, P31)


FIRST_CALL = r"""
import sys, ctypes
import numpy as np, torch
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle
from paper_2605_25863_gb300 import linac, synth
from test_zz_no_alloc import call_noalloc
p = synth.P31
M = synth.rank_deficient(m=900, n=950, d=12, p=p, seed=67)[0]
A = linac.to_device(M)
code, rank, piv = call_noalloc(A, p)      # the library's first call in this process
torch.cuda.synchronize()
R0, r0, piv0, _ = oracle.rref(M, p, nthreads=8)
r = int(rank.item())
piv = piv.cpu().numpy()
ok = (code == 0 and r == r0 == 888 and np.array_equal(piv[:r], piv0) and (piv[r:] == -1).all()
      and np.array_equal(A.cpu().numpy().view(np.uint32), R0))
print("FIRST_CALL_OK" if ok else f"FIRST_CALL_BAD code={{code}} rank={{r}} oracle={{r0}}")
"""


def test_noalloc_as_first_call_in_a_fresh_process():
    script = FIRST_CALL.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "FIRST_CALL_OK" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
