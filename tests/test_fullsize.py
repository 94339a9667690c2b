"""Full-size check of the dense workload in the launch configuration the
benchmark times: the 32768 x 33024 system (A 32768 x 32768 plus 256
right-hand sides, uniform residues, p = 2^31 - 1), panel width 128, default
path.  The oracle cannot reduce it in test time (1.8e13 multiply-adds), so
the result is checked through properties that hold at any size:

* rank 32768 and pivot columns 0..32767 (a uniform square matrix over
  F_p is invertible with probability > 1 - 1/p);
* the left block of the RREF is exactly the identity (section 5.2:
  [A | B] reduces to [I | X]);
* A X = B (mod p) for all 256 right-hand sides, exactly: the product A X
  (2.7e14 multiply-adds) runs on linac_matmul, the library's exact mod-p
  product (its own kernel, pinned against the oracle in
  test_parity_derived.py), and is compared with B entry by entry.  Because A
  is invertible, X is then the unique solution and the RREF [I | X] is
  determined, so the check is deterministic;
* the same identity by Freivalds' test with three random vectors v,
  A (X v) = B v, in exact integer arithmetic on the CPU (numpy int64 with a
  16-bit split), independent of the CUDA code.
"""
import numpy as np
import pytest
import torch

from paper_2605_25863_gb300 import linac, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

P = synth.P31
M_ROWS, RHS = 32768, 256


def matmul_mod(A: np.ndarray, Y: np.ndarray, p: int, chunk: int = 2048) -> np.ndarray:
    """(A @ Y) mod p exactly for A uint32 (rows x cols) and Y residues
    (cols x t): Y is split into 16-bit halves so every partial dot product
    stays below 2^62 for cols <= 2^15."""
    Y = np.asarray(Y, dtype=np.uint64).reshape(A.shape[1], -1)
    t = Y.shape[1]
    parts = np.concatenate([(Y & np.uint64(0xFFFF)), (Y >> np.uint64(16))], axis=1).astype(np.int64)
    out = np.empty((A.shape[0], t), dtype=np.int64)
    for r0 in range(0, A.shape[0], chunk):
        blk = A[r0:r0 + chunk].astype(np.int64) @ parts
        out[r0:r0 + chunk] = (blk[:, :t] % p + ((blk[:, t:] % p) << 16) % p) % p
    return out


def test_dense_32768_bench_configuration():
    dev = torch.device("cuda")
    n = M_ROWS + RHS
    key = synth.stream_key(5, "large_dense")           # the benchmark's input stream
    A = synth.uniform_torch(M_ROWS, n, P, key, device=dev)
    orig = A.cpu().numpy().view(np.uint32).copy()
    rank, piv = linac.linac_rref(A, P, nb=128)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 0
    assert int(rank.item()) == M_ROWS
    assert torch.equal(piv.cpu(), torch.arange(M_ROWS, dtype=torch.int32))
    eye_ok = True
    for r0 in range(0, M_ROWS, 4096):
        blk = A[r0:r0 + 4096, :M_ROWS]
        ref = torch.zeros_like(blk)
        ref[torch.arange(blk.shape[0], device=dev), torch.arange(r0, r0 + blk.shape[0], device=dev)] = 1
        eye_ok &= bool(torch.equal(blk, ref))
    assert eye_ok, "left block is not the identity"
    # exact A X = B on the device (A kept in its original state on the host)
    A0 = torch.from_numpy(orig.view(np.int32)).to(dev)
    AX = linac.linac_matmul(A0[:, :M_ROWS], A[:, M_ROWS:], P)
    torch.cuda.synchronize()
    assert torch.equal(AX, A0[:, M_ROWS:]), "A X != B (mod p) on the device product"
    del A0, AX
    X = A[:, M_ROWS:].cpu().numpy().view(np.uint32)
    V = np.random.default_rng(2026).integers(0, P, size=(RHS, 3), dtype=np.int64)
    XV = matmul_mod(X, V, P)
    lhs = matmul_mod(orig[:, :M_ROWS], XV, P)
    rhs = matmul_mod(orig[:, M_ROWS:], V, P)
    assert np.array_equal(lhs, rhs), "A X != B (mod p)"
