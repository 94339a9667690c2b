"""Failure detection without a GPU fault.

The dense elimination's one wait on other thread blocks is the arrival
barrier of the full-height pivot search (the grid-wide search of section 3.2,
"Pivoting", that runs when a panel's pivot window lacks a pivot).  It is
bounded: after the wait limit every block records LINAC_ERR_TIMEOUT in the
device status word and returns.  These tests make that wait run out on
purpose -- the injected failure raises the barrier's target by one arrival
that no block ever makes, a flag that nothing sets -- with a short limit,
then check that the status word says so and that the next, normal call on the
same stream is bit-exact with the oracle.  No kernel faults, traps or hangs:
every block returns after about the limit.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_25863_gb300 import linac, synth

NTH = min(16, os.cpu_count() or 1)
P31 = synth.P31
LINAC_ERR_TIMEOUT = 6


def _window_missing_pivot(m=520, n=300, zero_rows=300, seed=8):
    """Column 3 is zero in the first zero_rows rows, more than the first
    panel's pivot window holds, so the full-height search must run."""
    M = synth.uniform((m, n), P31, synth.stream_key(seed, "wait_failure"))
    M[:zero_rows, 3] = 0
    return M


def test_wait_limit_argument_checked():
    """CPU: a negative limit is rejected on the host."""
    from paper_2605_25863_gb300 import build
    build.build()
    assert linac.lib().linac_set_wait_limit(-5) == 1   # LINAC_ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("nb", [128, 32])
def test_injected_wait_failure_reports_timeout_then_recovers(nb):
    M = _window_missing_pivot()
    linac.linac_set_wait_limit(200_000)          # about 0.1 ms of SM clocks
    linac.linac_debug_inject_wait_failure(True)
    try:
        A = linac.to_device(M)
        linac.linac_rref(A, P31, nb=nb)          # the host call itself succeeds
        assert linac.linac_last_device_status() == LINAC_ERR_TIMEOUT
    finally:
        linac.linac_debug_inject_wait_failure(False)
        linac.linac_set_wait_limit(0)
    # the next call on the same stream runs normally and is exact
    A = linac.to_device(M)
    rank, piv = linac.linac_rref(A, P31, nb=nb)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 0
    R0, r0, piv0, _ = oracle.rref(M, P31, nthreads=NTH)
    assert int(rank.item()) == r0
    assert np.array_equal(piv.cpu().numpy()[:r0], piv0)
    assert np.array_equal(A.cpu().numpy().view(np.uint32), R0)


@pytest.mark.gpu
def test_injected_failure_in_solve_reports_timeout():
    M = _window_missing_pivot(m=400, n=260, zero_rows=250, seed=9)
    A, B = M[:, :256], M[:, 256:]
    linac.linac_set_wait_limit(200_000)
    linac.linac_debug_inject_wait_failure(True)
    try:
        linac.linac_solve(linac.to_device(A), linac.to_device(B), P31)
        assert linac.linac_last_device_status() == LINAC_ERR_TIMEOUT
    finally:
        linac.linac_debug_inject_wait_failure(False)
        linac.linac_set_wait_limit(0)
    X, cons, rank, piv = linac.linac_solve(linac.to_device(A), linac.to_device(B), P31)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 0
    X0, cons0, r0, _, _ = oracle.solve(A, B, P31, nthreads=NTH)
    assert int(rank.item()) == r0
    assert np.array_equal(X.cpu().numpy().view(np.uint32), X0)
    assert np.array_equal(cons.cpu().numpy(), cons0)


@pytest.mark.gpu
def test_window_only_elimination_never_waits():
    """With the failure injected but a matrix whose every panel window holds
    its pivots, the grid-wide search (and its wait) never runs: the result is
    exact and the status stays clean."""
    M = synth.uniform((300, 340), P31, synth.stream_key(10, "no_wait"))
    linac.linac_set_wait_limit(200_000)
    linac.linac_debug_inject_wait_failure(True)
    try:
        A = linac.to_device(M)
        rank, piv = linac.linac_rref(A, P31)
        torch.cuda.synchronize()
        assert linac.linac_last_device_status() == 0
    finally:
        linac.linac_debug_inject_wait_failure(False)
        linac.linac_set_wait_limit(0)
    R0, r0, _, _ = oracle.rref(M, P31, nthreads=NTH)
    assert int(rank.item()) == r0 and np.array_equal(A.cpu().numpy().view(np.uint32), R0)
