"""GPU parity of linac_rref_batched with the CPU oracle, system by system,
bit for bit: uneven batches over every size bucket, rectangular and
degenerate systems, and the shared-pivot-pattern mode including systems that
must leave the pattern."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_25863_gb300 import linac, synth
from modmath import matmul_mod

pytestmark = pytest.mark.gpu

NTH = min(16, os.cpu_count() or 1)


def pack(systems, nA=None):
    B = synth._pack(systems, synth.P31, nA if nA is not None else [s.shape[1] for s in systems],
                    [0] * len(systems))
    return B


def run_batched(B, p, flags=0, use_nsearch=True):
    dev = torch.device("cuda")
    data = torch.from_numpy(B.data.view(np.int32)).to(dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ranks, piv, poff, st = linac.linac_rref_batched(
        data, t(B.offsets), t(B.m), t(B.n), t(B.ld), p,
        nsearch=t(B.nA) if use_nsearch else None, flags=flags)
    torch.cuda.synchronize()
    out = data.cpu().numpy().view(np.uint32)
    return out, ranks.cpu().numpy(), piv.cpu().numpy(), poff.cpu().numpy(), st.cpu().numpy()


def check_all(B, p, out, ranks, piv, poff, which=None):
    for s in (range(B.count) if which is None else which):
        S = B.system(s)
        o, m, n, ld = int(B.offsets[s]), int(B.m[s]), int(B.n[s]), int(B.ld[s])
        got = out[o:o + m * ld].reshape(m, ld)[:, :n] if m else np.zeros((0, n), np.uint32)
        R0, r0, piv0, _ = oracle.rref(S, p, col_limit=int(B.nA[s]), nthreads=NTH)
        assert ranks[s] == r0, f"system {s}: rank {ranks[s]} vs {r0}"
        assert np.array_equal(piv[poff[s]:poff[s] + r0], piv0), f"system {s}: pivots"
        assert np.array_equal(got, R0), f"system {s}: RREF differs"


def test_uneven_batch_all_buckets():
    B = synth.batched_uneven(count=120, lo=4, hi=1000, seed=21, deficient_frac=0.3)
    out, ranks, piv, poff, st = run_batched(B, B.p)
    check_all(B, B.p, out, ranks, piv, poff)
    assert (ranks == B.nA - B.deficiency).all()


@pytest.mark.parametrize("p", [3, 65537, synth.P31])
def test_rectangular_and_degenerate_systems(p):
    g = np.random.default_rng(p % 1000)
    shapes = [(1, 1), (1, 9), (9, 1), (5, 3), (3, 5), (70, 130), (130, 70), (64, 64), (65, 65),
              (128, 200), (300, 40), (40, 300), (600, 601), (1024, 1024), (17, 1000)]
    systems = [synth.uniform(sh, p, synth.stream_key(i, f"shapes{p}")) for i, sh in enumerate(shapes)]
    systems.append(np.zeros((50, 60), dtype=np.uint32))
    systems.append(np.full((33, 44), p - 1, dtype=np.uint32))
    dup = synth.uniform((1, 80), p, 99)
    systems.append(np.repeat(dup, 90, axis=0))
    B = synth._pack(systems, p, [s.shape[1] for s in systems], [0] * len(systems))
    out, ranks, piv, poff, st = run_batched(B, p)
    check_all(B, p, out, ranks, piv, poff)


def test_nsearch_limits_pivots_per_system():
    systems = []
    for i in range(20):
        n = 30 + 7 * i
        S = synth.uniform((n - 5, n + 4), synth.P31, synth.stream_key(i, "ns"))
        systems.append(S)
    nA = [s.shape[1] - 4 - (i % 3) for i, s in enumerate(systems)]
    B = synth._pack(systems, synth.P31, nA, [0] * len(systems))
    out, ranks, piv, poff, st = run_batched(B, synth.P31)
    check_all(B, synth.P31, out, ranks, piv, poff)


def test_workload_batched_uneven_10000():
    """The full batch: 10,000 systems, n log-uniform in [32, 512], 4 RHS,
    ~10 % rank-deficient.  Every rank is checked; 200 sampled systems are
    compared with the oracle; every full-rank system of the sample solves
    A X = B."""
    B = synth.batched_uneven()
    out, ranks, piv, poff, st = run_batched(B, B.p)
    assert (ranks == B.nA - B.deficiency).all()
    sample = np.random.default_rng(7).choice(B.count, size=200, replace=False)
    check_all(B, B.p, out, ranks, piv, poff, which=sample)
    for s in sample[:60]:
        n = int(B.nA[s])
        if B.deficiency[s]:
            continue
        o, m, ld = int(B.offsets[s]), int(B.m[s]), int(B.ld[s])
        R = out[o:o + m * ld].reshape(m, ld)[:, :int(B.n[s])]
        S = B.system(s)
        assert np.array_equal(R[:, :n], np.eye(n, dtype=np.uint32))
        assert np.array_equal(matmul_mod(S[:, :n], R[:, n:], B.p), S[:, n:])


def test_shared_pattern_matches_oracle():
    B = synth.shared_pattern(count=48)
    out, ranks, piv, poff, st = run_batched(B, B.p, flags=linac.LINAC_SHARED_PATTERN)
    check_all(B, B.p, out, ranks, piv, poff)
    assert (ranks == 384).all()
    assert (st == 0).all(), "no system should leave the pattern"


def test_shared_pattern_fallbacks():
    """Systems that cannot reuse the probe's pivots fall back to the search
    (status bit 0x100) and still match the oracle: a vanished pivot, a
    different shape, and a lower rank."""
    base = synth.shared_pattern(count=12)
    systems = [base.system(s).copy() for s in range(base.count)]
    systems[3][:, 0] = 0                              # first pivot vanishes
    systems[5][10] = systems[5][11]                   # rank drops by one
    systems[7] = systems[7][:200].copy()              # different shape
    nA = [384] * len(systems)
    B = synth._pack(systems, base.p, nA, [0] * len(systems))
    out, ranks, piv, poff, st = run_batched(B, base.p, flags=linac.LINAC_SHARED_PATTERN)
    check_all(B, base.p, out, ranks, piv, poff)
    for s in (3, 5, 7):
        assert st[s] & 0x100, f"system {s} should have fallen back"
    for s in (1, 2, 4, 6, 8, 9, 10, 11):
        assert st[s] == 0


@pytest.mark.parametrize("widths", [[16, 16, 16, 16, 16], [64, 64, 64, 32, 32]])
def test_every_panel_width_matches_oracle(widths):
    """Every panel width the kernel is built for (16, 32 and 64 columns; 64
    fits systems of at most 256 rows) against the oracle, with the search
    and with the shared pattern: the pivot window's row batches, the update's
    4- and 8-row items and the pattern's pivot-row slab differ by width.  The
    widths are set explicitly, as a caller may, and restored afterwards."""
    saved = linac.linac_batched_panel_widths()
    try:
        linac.linac_batched_set_panel_widths(widths)
        assert linac.linac_batched_panel_widths() == widths
        B = synth.batched_uneven(count=60, lo=4, hi=1000, seed=33, deficient_frac=0.3)
        out, ranks, piv, poff, st = run_batched(B, B.p)
        check_all(B, B.p, out, ranks, piv, poff)
        assert (ranks == B.nA - B.deficiency).all()
        # a 240 x 256 template: systems of the 256-row bucket, reduced with
        # the shared pattern at that bucket's width
        Bs = synth.shared_pattern(count=24, rows=240, cols=256, rhs=16)
        out, ranks, piv, poff, st = run_batched(Bs, Bs.p, flags=linac.LINAC_SHARED_PATTERN)
        check_all(Bs, Bs.p, out, ranks, piv, poff)
        assert (ranks == 240).all() and (st == 0).all()
    finally:
        linac.linac_batched_set_panel_widths(saved)


def test_workload_shared_pattern_4096_sampled():
    B = synth.shared_pattern(count=4096)
    out, ranks, piv, poff, st = run_batched(B, B.p, flags=linac.LINAC_SHARED_PATTERN)
    assert (ranks == 384).all()
    sample = np.random.default_rng(3).choice(B.count, size=24, replace=False)
    check_all(B, B.p, out, ranks, piv, poff, which=sample)
    out2, ranks2, piv2, poff2, st2 = run_batched(B, B.p, flags=0)
    assert np.array_equal(out, out2) and np.array_equal(ranks, ranks2)


def test_autotuned_widths_keep_parity():
    """The autotuner picks a panel width per size bucket; results stay exact."""
    widths = linac.linac_batched_tune(synth.P_BATCH)
    assert len(widths) == 5 and all(w in (16, 32, 64) for w in widths)
    assert linac.linac_batched_panel_widths() == widths
    B = synth.batched_uneven(count=60, lo=8, hi=1000, seed=33, deficient_frac=0.3)
    out, ranks, piv, poff, st = run_batched(B, B.p)
    check_all(B, B.p, out, ranks, piv, poff)


def _graph_run(B, flags):
    """One eager call (creates the scratch), then the same call captured into
    a CUDA graph and replayed twice on restored inputs."""
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    data0 = t(B.data.view(np.int32))
    offs, mm, nn, ld, ns = t(B.offsets), t(B.m), t(B.n), t(B.ld), t(B.nA)
    max_m, max_n = int(B.m.max()), int(B.n.max())
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        data = data0.clone()
        ranks, piv, poff, st = linac.batched_outputs(mm, nn, ns)
        linac.linac_rref_batched_into(data, offs, mm, nn, ld, B.p, ranks, piv, poff, st, max_m=max_m,
                                      max_n=max_n, nsearch=ns, flags=flags)
        eager = (data.clone(), ranks.clone(), piv.clone(), st.clone())
        data.copy_(data0)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        linac.linac_rref_batched_into(data, offs, mm, nn, ld, B.p, ranks, piv, poff, st, max_m=max_m,
                                      max_n=max_n, nsearch=ns, flags=flags)
    for _ in range(2):
        data.copy_(data0)
        piv.fill_(-1)
        ranks.zero_()
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip((data, ranks, piv, st), eager):
            assert torch.equal(a, b), "graph replay differs from the eager call"
    return eager


def test_batched_cuda_graph_replay():
    """The whole batched call (sort + persistent launches) captured into one
    CUDA graph replays bit-exactly, and matches the oracle."""
    B = synth.batched_uneven(count=200, lo=8, hi=1000, seed=41, deficient_frac=0.2)
    data, ranks, piv, st = _graph_run(B, 0)
    out = data.cpu().numpy().view(np.uint32)
    npiv = np.minimum(B.m.astype(np.int64), B.nA.astype(np.int64))
    poff = np.concatenate([[0], np.cumsum(npiv)[:-1]])
    check_all(B, B.p, out, ranks.cpu().numpy(), piv.cpu().numpy(), poff, which=range(0, B.count, 7))


def test_shared_pattern_cuda_graph_replay():
    B = synth.shared_pattern(count=64)
    data, ranks, piv, st = _graph_run(B, linac.LINAC_SHARED_PATTERN)
    assert (ranks.cpu().numpy() == 384).all()
    assert (st.cpu().numpy() == 0).all()
