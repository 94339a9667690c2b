"""GPU parity of the dense path (linac_rref / linac_solve) with the CPU
oracle, bit for bit, plus RREFs known by construction.  Sizes span several
panels and update tiles with ragged tails."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_25863_gb300 import linac, synth
from modmath import known_rref_matrix, matmul_mod

pytestmark = pytest.mark.gpu

P31 = synth.P31
PB = synth.P_BATCH
NTH = min(16, os.cpu_count() or 1)


def gpu_rref(M, p, **kw):
    A = linac.to_device(M)
    rank, piv = linac.linac_rref(A, p, **kw)
    torch.cuda.synchronize()
    assert linac.linac_last_device_status() == 0
    R = A.cpu().numpy().view(np.uint32)[:, :M.shape[1]].copy()
    return R, int(rank.item()), piv.cpu().numpy()


def check_against_oracle(M, p, **kw):
    R, r, piv = gpu_rref(M, p, **kw)
    ns = kw.get("ncols_search")
    R0, r0, piv0, _ = oracle.rref(M, p, col_limit=ns, nthreads=NTH)
    assert r == r0
    assert np.array_equal(piv[:r], piv0)
    assert (piv[r:] == -1).all()
    assert np.array_equal(R, R0)
    return R, r, piv


@pytest.mark.parametrize("p", [3, 65537, P31, PB])
@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (5, 3), (17, 33), (64, 64), (100, 257), (257, 100),
                                   (300, 300), (513, 700)])
def test_uniform_vs_oracle(shape, p):
    m, n = shape
    M = synth.uniform(shape, p, synth.stream_key(m * 1009 + n, f"u{p}"))
    check_against_oracle(M, p)


@pytest.mark.parametrize("nb", [16, 32, 64, 128])
@pytest.mark.parametrize("path", ["plain", "auto", "limb", "crt", "hybrid"])
def test_panel_widths(nb, path):
    M, _ = synth.rank_deficient(m=333, n=401, d=21, p=P31, seed=nb)
    check_against_oracle(M, P31, nb=nb, path=path)


@pytest.mark.parametrize("p", [7, P31, PB])
@pytest.mark.parametrize("mnr", [(200, 300, 150), (300, 200, 170), (260, 260, 259), (129, 700, 90),
                                 (700, 129, 129), (400, 64, 13)])
def test_known_rref_by_construction(p, mnr):
    m, n, rank = mnr
    g = np.random.default_rng(m * 7 + n * 3 + rank + p % 101)
    A, R, piv = known_rref_matrix(g, m, n, rank, p)
    Rg, rg, pg = gpu_rref(A, p)
    assert rg == rank and np.array_equal(pg[:rank], piv) and np.array_equal(Rg, R)


def test_small_prime_forces_many_swaps():
    """p = 3: a third of the entries vanish, so pivot rows come from deep in
    the slab and from other blocks' slabs."""
    M = synth.uniform((600, 650), 3, synth.stream_key(5, "p3"))
    check_against_oracle(M, 3)


def test_late_pivots_and_zero_columns():
    g = np.random.default_rng(3)
    m, n = 300, 500
    piv = np.sort(np.concatenate([g.choice(np.arange(130, 500), size=150, replace=False)]))
    A, R, pv = known_rref_matrix(g, m, n, len(piv), P31, pivots=piv)
    Rg, rg, pg = gpu_rref(A, P31, nb=32)
    assert rg == len(piv) and np.array_equal(pg[:rg], pv) and np.array_equal(Rg, R)


def test_special_matrices():
    p = P31
    Z = np.zeros((70, 90), dtype=np.uint32)
    R, r, piv = gpu_rref(Z, p)
    assert r == 0 and not R.any() and (piv == -1).all()
    I = np.eye(150, dtype=np.uint32)
    R, r, piv = gpu_rref(I, p)
    assert r == 150 and np.array_equal(R, I)
    perm = np.random.default_rng(1).permutation(150)
    R, r, piv = gpu_rref(I[perm], p)
    assert np.array_equal(R, I)
    F = np.full((40, 50), p - 1, dtype=np.uint32)
    check_against_oracle(F, p)
    D = np.repeat(synth.uniform((1, 90), p, 77), 33, axis=0)
    check_against_oracle(D, p)


@pytest.mark.parametrize("shape", [(0, 5), (5, 0), (0, 0)])
def test_empty(shape):
    m, n = shape
    A = linac.padded(m, n)
    rank, piv = linac.linac_rref(A, P31)
    torch.cuda.synchronize()
    assert int(rank.item()) == 0


def test_ncols_search_limits_pivots():
    M = synth.uniform((120, 150), P31, synth.stream_key(9, "ns"))
    M[:, 60:] = 0
    M[:, 100:] = synth.uniform((120, 50), P31, synth.stream_key(9, "ns2"))
    check_against_oracle(M, P31, ncols_search=80)


def test_workload_dense_system_256():
    """The 256 x 256 system with one right-hand side: RREF of [A | b] and the
    solve both match the oracle; x solves A x = b."""
    S = synth.dense_system(n=256, k=1, p=P31, seed=1)
    R, r, piv = check_against_oracle(S, P31)
    assert r == 256 and np.array_equal(piv, np.arange(256))
    A, b = S[:, :256], S[:, 256:]
    X, cons, rank, pv = linac.linac_solve(linac.to_device(A), linac.to_device(b), P31)
    torch.cuda.synchronize()
    X = X.cpu().numpy().view(np.uint32)
    X0, cons0, r0, _, _ = oracle.solve(A, b, P31)
    assert int(rank.item()) == r0 == 256 and cons.cpu().numpy().all()
    assert np.array_equal(X, X0) and np.array_equal(X[:, 0], R[:, 256])
    assert np.array_equal(matmul_mod(A, X, P31), b)


def test_workload_rank_deficient_4096():
    """4096 x 4160 with 64 rows replaced by combinations of others: rank 4032,
    pivots 0..4031, RREF identical to the oracle's."""
    M, _ = synth.rank_deficient()
    R, r, piv = check_against_oracle(M, P31)
    assert r == 4032 and np.array_equal(piv[:r], np.arange(4032))


def test_solve_inconsistent_and_underdetermined():
    p = P31
    g = np.random.default_rng(12)
    A, R, piv = known_rref_matrix(g, 90, 120, 70, p)
    x0 = synth.uniform((120, 3), p, 4)
    B = matmul_mod(A, x0, p)
    B[:, 1] = (B[:, 1].astype(np.int64) + 5) % p
    X, cons, rank, pv = linac.linac_solve(linac.to_device(A), linac.to_device(B), p)
    torch.cuda.synchronize()
    X = X.cpu().numpy().view(np.uint32)
    X0, cons0, r0, pv0, _ = oracle.solve(A, B, p)
    assert int(rank.item()) == r0 == 70
    assert np.array_equal(cons.cpu().numpy(), cons0) and list(cons0) == [True, False, True]
    assert np.array_equal(X, X0)
    for j in (0, 2):
        assert np.array_equal(matmul_mod(A, X[:, j:j + 1], p)[:, 0], B[:, j])


def test_validation_flags_out_of_range_entries():
    M = synth.uniform((40, 44), P31, 3)
    M[7, 9] = P31 + 5
    A = linac.to_device(M)
    linac.linac_rref(A, P31, validate=True)
    assert linac.linac_last_device_status() == 7   # LINAC_ERR_RANGE


def test_repeated_calls_reuse_scratch_and_match():
    M, _ = synth.rank_deficient(m=500, n=520, d=10, p=P31, seed=44)
    R1, r1, p1 = gpu_rref(M, P31)
    R2, r2, p2 = gpu_rref(M, P31)
    assert r1 == r2 and np.array_equal(R1, R2) and np.array_equal(p1, p2)


@pytest.mark.parametrize("p", [3, 251, 65537, P31, PB])
@pytest.mark.parametrize("shape", [(37, 45), (300, 300), (513, 700), (1000, 1100)])
def test_limb_path_vs_oracle(shape, p):
    """The u8-limb integer-tensor update gives the same RREF as the oracle."""
    m, n = shape
    M = synth.uniform(shape, p, synth.stream_key(m * 31 + n, f"limb{p}"))
    check_against_oracle(M, p, path="limb")


@pytest.mark.parametrize("nb", [16, 32, 64, 128])
def test_limb_path_rank_deficient(nb):
    M, _ = synth.rank_deficient(m=700, n=650, d=33, p=PB, seed=nb + 100)
    check_against_oracle(M, PB, path="limb", nb=nb)


def test_limb_and_plain_agree_on_workload_4096():
    M, _ = synth.rank_deficient()
    Rl, rl, pl = gpu_rref(M, P31, path="limb")
    Rp, rp, pp = gpu_rref(M, P31, path="plain")
    assert rl == rp == 4032 and np.array_equal(pl, pp) and np.array_equal(Rl, Rp)


@pytest.mark.parametrize("p", [P31, 65537])
@pytest.mark.parametrize("zero_rows", [150, 300])
def test_pivot_window_fallback(p, zero_rows):
    """Column 3 is zero in the first `zero_rows` rows, so the pivot window of
    the first panel (its first w + 16 remaining rows) has no pivot there and
    the grid-wide panel search must supply it; later panels use the window
    again.  Bit-exact against the oracle either way."""
    m, n = 520, 300
    M = synth.uniform((m, n), p, synth.stream_key(zero_rows, "window_fallback"))
    M[:zero_rows, 3] = 0
    M[:zero_rows // 2, 140] = 0
    check_against_oracle(M, p)
    check_against_oracle(M, p, nb=32)


@pytest.mark.parametrize("p", [3, 251, 65537, P31, PB, 1431655777, 1908903247])
@pytest.mark.parametrize("shape", [(37, 45), (300, 300), (513, 700), (1000, 1100)])
def test_crt_path_vs_oracle(shape, p):
    """The multi-modular integer-tensor update (nine s8 residue GEMMs and an
    exact Chinese-remainder reconstruction) gives the oracle's RREF."""
    m, n = shape
    M = synth.uniform(shape, p, synth.stream_key(m * 37 + n, f"crt{p}"))
    check_against_oracle(M, p, path="crt")


@pytest.mark.parametrize("nb", [16, 64, 128])
def test_crt_path_rank_deficient(nb):
    M, _ = synth.rank_deficient(m=700, n=650, d=33, p=PB, seed=nb + 200)
    check_against_oracle(M, PB, path="crt", nb=nb)


@pytest.mark.parametrize("p", [P31, PB, 1431655777, 251])
@pytest.mark.parametrize("sign", [1, -1])
def test_crt_path_extreme_products(p, sign):
    """The reconstruction's worst case: A = [[I, X], [Y, Z]] with a 128 x 128
    identity, so the first panel's pivot rows are [I | X] unchanged and its
    update subtracts Y X; with every entry of X and Y at the balanced extreme
    (p - 1)/2 (or -(p - 1)/2 in X) each output is +-128 ((p - 1)/2)^2, the
    largest |F R| a 128-column panel can produce."""
    half = (p - 1) // 2
    m, n = 600, 640
    M = synth.uniform((m, n), p, synth.stream_key(p % 1000 + sign, "crt_extreme"))
    M[:128, :128] = np.eye(128, dtype=np.uint32)
    M[:128, 128:] = half if sign > 0 else half + 1
    M[128:, :128] = half
    check_against_oracle(M, p, path="crt", nb=128)


def test_crt_and_plain_agree_on_workload_4096():
    M, _ = synth.rank_deficient()
    Rc, rc, pc = gpu_rref(M, P31, path="crt")
    Rp, rp, pp = gpu_rref(M, P31, path="plain")
    assert rc == rp == 4032 and np.array_equal(pc, pp) and np.array_equal(Rc, Rp)


@pytest.mark.parametrize("path", ["plain", "crt", "hybrid"])
def test_rref_replays_in_a_cuda_graph(path):
    """linac_rref is stream-ordered with no host synchronisation: after one
    uncaptured call (which creates the scratch), the call captures into a
    CUDA graph; replays on restored input are exact."""
    M, _ = synth.rank_deficient(m=700, n=660, d=9, p=P31, seed=71)
    pristine = linac.to_device(M)
    A = linac.padded(*M.shape)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        A.copy_(pristine)
        rank, piv = linac.linac_rref(A, P31, path=path, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        A.copy_(pristine)
        rank, piv = linac.linac_rref(A, P31, path=path, stream=s)
    R0, r0, piv0, _ = oracle.rref(M, P31, nthreads=NTH)
    for _ in range(2):
        A.zero_()
        with torch.cuda.stream(s):
            g.replay()
        s.synchronize()
        assert int(rank.item()) == r0 == 660
        assert np.array_equal(piv.cpu().numpy()[:r0], piv0)
        assert np.array_equal(A.cpu().numpy().view(np.uint32), R0)


@pytest.mark.parametrize("p", [3, 251, 65537, P31, PB, 1431655777])
@pytest.mark.parametrize("shape", [(37, 45), (300, 300), (513, 700), (1000, 1100), (2100, 2300)])
def test_hybrid_path_vs_oracle(shape, p):
    """CUDA-core and multi-modular tiles of one update, taken from one work
    counter by the two warp groups of each block: the oracle's RREF."""
    m, n = shape
    M = synth.uniform(shape, p, synth.stream_key(m * 41 + n, f"hybrid{p}"))
    check_against_oracle(M, p, path="hybrid")


def test_hybrid_and_plain_agree_on_workload_4096():
    M, _ = synth.rank_deficient()
    Rh, rh, ph = gpu_rref(M, P31, path="hybrid")
    Rp, rp, pp = gpu_rref(M, P31, path="plain")
    assert rh == rp == 4032 and np.array_equal(ph, pp) and np.array_equal(Rh, Rp)
