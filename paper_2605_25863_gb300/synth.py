"""Seeded synthetic workloads for exact mod-p row reduction.

This module only builds inputs: it holds none of the elimination arithmetic.
It serves the test suite, the benchmark and the CPU oracle alike, so both
sides of every parity check see the same matrices.

Random numbers come from the SplitMix64 finaliser (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: word i of stream (seed, tag) is
``mix(key(seed, tag) + (i + 1) * 0x9E3779B97F4A7C15)``.  A residue in [0, p) is
``(hi32(word) * p) >> 32`` (a multiply-shift map; its bias is below 2^-31 and
irrelevant for synthetic inputs).  The same map is implemented for numpy
(``uniform``) and for torch tensors on any device (``uniform_torch``); the
tests check that the two agree bit for bit.

Workloads (the paper benchmarks dense, fully random square matrices over
F_{2^31-1}, section 4.1; its linear systems come from evaluating monomial
ansatze at random points, section 3.3):

* ``dense_system``      -- [A | b] with A n x n uniform (256 x 257 by default).
* ``rank_deficient``    -- m x n uniform with ``d`` rows replaced by random
                           combinations of other rows (4096 x 4160, d = 64).
* ``batched_uneven``    -- independent [A | B] systems, n log-uniform in
                           [32, 512], 4 right-hand sides, ~10 % of them made
                           rank-deficient by 1..8 (augmented rows replaced).
* ``shared_pattern``    -- one block-banded 384 x 400 template of bivariate
                           polynomials (total degree <= 4) evaluated at many
                           random points (x, y).
* ``uniform`` at 32768 x 33024 for the large dense case.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

P31 = 2**31 - 1          # the paper's benchmark prime (section 4.1)
P_BATCH = 2147483629     # 2^31 - 19, a prime; the batched workload's modulus

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (used for stream keys)."""
    z &= _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, tag: str | int) -> int:
    """64-bit key of the stream named ``tag`` under ``seed``."""
    if isinstance(tag, str):
        h = 0xCBF29CE484222325
        for ch in tag.encode():
            h = ((h ^ ch) * 0x100000001B3) & _MASK64
        tag = h
    return _mix_int(_mix_int(seed * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) ^ (tag & _MASK64))


def words(key: int, count: int, start: int = 0) -> np.ndarray:
    """Words start .. start+count-1 of the stream ``key`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(key) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(shape, p: int, key: int, start: int = 0) -> np.ndarray:
    """Residues in [0, p) (uint32) filling ``shape`` in row-major order."""
    count = int(np.prod(shape))
    out = np.empty(count, dtype=np.uint32)
    chunk = 1 << 24
    for s in range(0, count, chunk):
        w = words(key, min(chunk, count - s), start + s)
        out[s:s + len(w)] = (((w >> np.uint64(32)) * np.uint64(p)) >> np.uint64(32)).astype(np.uint32)
    return out.reshape(shape)


def uniform64(shape, p: int, key: int, start: int = 0) -> np.ndarray:
    """Residues in [0, p) (uint64) for a modulus up to 2^64 - 1, filling
    ``shape`` in row-major order: floor(w * p / 2^64) of each 64-bit word w of
    the stream (multiply-shift; the 128-bit product is assembled from 32-bit
    halves so numpy's uint64 never overflows)."""
    count = int(np.prod(shape))
    out = np.empty(count, dtype=np.uint64)
    lo32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    ph, pl = np.uint64(p >> 32), np.uint64(p & 0xFFFFFFFF)
    chunk = 1 << 22
    for s in range(0, count, chunk):
        w = words(key, min(chunk, count - s), start + s)
        wh, wl = w >> s32, w & lo32
        hh, hl, lh, ll = wh * ph, wh * pl, wl * ph, wl * pl       # each < 2^64
        mid = (hl & lo32) + (lh & lo32) + (ll >> s32)              # < 3 * 2^32
        out[s:s + len(w)] = hh + (hl >> s32) + (lh >> s32) + (mid >> s32)
    return out.reshape(shape)


def rank_deficient64(m: int, n: int, d: int, p: int, seed: int = 2, terms: int = 8):
    """uint64 counterpart of ``rank_deficient`` for a prime up to 2^64 - 1:
    m x n uniform, ``d`` seeded rows replaced by random combinations of
    ``terms`` other rows (exact Python-integer arithmetic).  Returns
    (M, replaced_rows)."""
    M = uniform64((m, n), p, stream_key(seed, "rank_deficient64"))
    perm = np.argsort(words(stream_key(seed, "rd64_rows"), m))
    targets = np.sort(perm[:d])
    pool = np.setdiff1d(np.arange(m), targets)
    pick = words(stream_key(seed, "rd64_pick"), max(d * terms, 1), 0)
    coefs = uniform64((max(d, 1), terms), p, stream_key(seed, "rd64_coef"))
    for a, t in enumerate(targets):
        acc = np.zeros(n, dtype=object)
        for b in range(terms):
            src = int(pool[int(pick[a * terms + b] % np.uint64(len(pool)))])
            acc = (acc + M[src].astype(object) * max(int(coefs[a, b]), 1)) % p
        M[t] = np.asarray(acc, dtype=np.uint64) if n else M[t]
    return M, targets


def unit_floats(key: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits (input construction only)."""
    w = words(key, count, start)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def uniform_torch(rows: int, cols: int, p: int, key: int, device="cpu", out=None, ld: int | None = None):
    """Same stream as ``uniform`` computed with torch int64 ops on ``device``.

    Returns (or fills) an int32 tensor rows x ld whose first ``cols`` columns
    hold the residues (bit pattern of uint32; all residues are < 2^31 so the
    int32 view is the value itself).  Columns cols..ld-1 are set to zero.
    """
    import torch
    ld = cols if ld is None else ld
    if out is None:
        out = torch.empty((rows, ld), dtype=torch.int32, device=device)
    mask30 = (1 << 34) - 1   # logical >> 30 on int64 = arithmetic >> 30 then mask 34 bits
    mask27 = (1 << 37) - 1
    mask31 = (1 << 33) - 1

    def s64(v: int) -> int:
        v &= _MASK64
        return v - (1 << 64) if v >= (1 << 63) else v

    g, m1, m2, kk = s64(0x9E3779B97F4A7C15), s64(0xBF58476D1CE4E5B9), s64(0x94D049BB133111EB), s64(key)
    rows_per = max(1, (1 << 24) // max(cols, 1))
    colidx = torch.arange(cols, dtype=torch.int64, device=device)
    for r0 in range(0, rows, rows_per):
        r1 = min(rows, r0 + rows_per)
        idx = (torch.arange(r0, r1, dtype=torch.int64, device=device)[:, None] * cols + colidx[None, :]) + 1
        z = idx * g + kk
        z = (z ^ ((z >> 30) & mask30)) * m1
        z = (z ^ ((z >> 27) & mask27)) * m2
        z = z ^ ((z >> 31) & mask31)
        hi = (z >> 32) & 0xFFFFFFFF
        out[r0:r1, :cols] = ((hi * p) >> 32).to(torch.int32)
    if ld > cols:
        out[:, cols:] = 0
    return out


def _lincomb_rows(M: np.ndarray, targets, sources_pool, p: int, key: int, terms: int):
    """Replace each row in ``targets`` by a random mod-p combination of
    ``terms`` rows drawn from ``sources_pool`` (input construction only)."""
    pool = np.asarray(sources_pool)
    pick = words(key, len(targets) * terms, 0)
    coefs = uniform((len(targets), terms), p, key ^ 0x5A5A5A5A5A5A5A5A)
    for a, t in enumerate(targets):
        acc = np.zeros(M.shape[1], dtype=np.uint64)
        for b in range(terms):
            src = int(pool[int(pick[a * terms + b] % np.uint64(len(pool)))])
            c = np.uint64(max(int(coefs[a, b]), 1))
            acc = (acc + (M[src].astype(np.uint64) * c) % np.uint64(p)) % np.uint64(p)
        M[t] = acc.astype(np.uint32)


def dense_system(n: int = 256, k: int = 1, p: int = P31, seed: int = 1):
    """[A | B] with A n x n and B n x k uniform in [0, p)."""
    return uniform((n, n + k), p, stream_key(seed, "dense_system"))


def rank_deficient(m: int = 4096, n: int = 4160, d: int = 64, p: int = P31, seed: int = 2,
                   terms: int = 8):
    """m x n uniform matrix with ``d`` seeded rows replaced by random mod-p
    combinations of ``terms`` of the other rows; rank m - d with high
    probability.  Returns (M, replaced_rows)."""
    M = uniform((m, n), p, stream_key(seed, "rank_deficient"))
    perm = np.argsort(words(stream_key(seed, "rd_rows"), m))
    targets = np.sort(perm[:d])
    keep = np.setdiff1d(np.arange(m), targets)
    _lincomb_rows(M, targets, keep, p, stream_key(seed, "rd_combo"), terms)
    return M, targets


@dataclass
class Batch:
    """Packed batch of independent row-major systems.

    ``data`` holds every system back to back; system s occupies
    ``data[offsets[s] : offsets[s] + m[s] * ld[s]]`` with leading dimension
    ``ld[s]`` (a multiple of 4 words, so every row starts 16-byte aligned).
    ``nA[s]`` is the number of coefficient columns (n[s] - nA[s] right-hand
    sides).  ``deficiency[s]`` is the number of augmented rows replaced by
    combinations of the others (0 for full-rank systems).
    """
    p: int
    data: np.ndarray
    offsets: np.ndarray
    m: np.ndarray
    n: np.ndarray
    ld: np.ndarray
    nA: np.ndarray
    deficiency: np.ndarray

    @property
    def count(self) -> int:
        return len(self.m)

    def system(self, s: int) -> np.ndarray:
        o, m, n, ld = int(self.offsets[s]), int(self.m[s]), int(self.n[s]), int(self.ld[s])
        return self.data[o:o + m * ld].reshape(m, ld)[:, :n]

    def total_words(self) -> int:
        return int(len(self.data))


def _pack(systems, p, nA, deficiency):
    m = np.array([s.shape[0] for s in systems], dtype=np.int32)
    n = np.array([s.shape[1] for s in systems], dtype=np.int32)
    ld = ((n + 3) // 4 * 4).astype(np.int32)
    sizes = m.astype(np.int64) * ld.astype(np.int64)
    offsets = np.zeros(len(systems), dtype=np.int64)
    if len(systems) > 1:
        offsets[1:] = np.cumsum(sizes)[:-1]
    data = np.zeros(int(sizes.sum()) if len(systems) else 0, dtype=np.uint32)
    for s, S in enumerate(systems):
        o = int(offsets[s])
        view = data[o:o + int(sizes[s])].reshape(int(m[s]), int(ld[s]))
        view[:, :S.shape[1]] = S
    return Batch(p=p, data=data, offsets=offsets, m=m, n=n, ld=ld,
                 nA=np.asarray(nA, dtype=np.int32), deficiency=np.asarray(deficiency, dtype=np.int32))


def batched_sizes(count: int, lo: int = 32, hi: int = 512, seed: int = 3) -> np.ndarray:
    """n = round(exp(U[ln lo, ln hi])) per system."""
    u = unit_floats(stream_key(seed, "batched_n"), count)
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int32)


def batched_uneven(count: int = 10000, rhs: int = 4, lo: int = 32, hi: int = 512,
                   p: int = P_BATCH, seed: int = 3, deficient_frac: float = 0.10,
                   max_deficiency: int = 8) -> Batch:
    """Independent square systems [A | B] of uneven size (see module doc)."""
    sizes = batched_sizes(count, lo, hi, seed)
    fr = unit_floats(stream_key(seed, "batched_deficient"), count)
    dsel = words(stream_key(seed, "batched_d"), count)
    systems, defic = [], []
    for s in range(count):
        n = int(sizes[s])
        S = uniform((n, n + rhs), p, stream_key(seed, 1000003 * (s + 1)))
        d = 0
        if fr[s] < deficient_frac:
            d = 1 + int(dsel[s] % np.uint64(max_deficiency))
            d = min(d, n - 1)
            perm = np.argsort(words(stream_key(seed, 2000003 * (s + 1)), n))
            targets = np.sort(perm[:d])
            keep = np.setdiff1d(np.arange(n), targets)
            _lincomb_rows(S, targets, keep, p, stream_key(seed, 3000017 * (s + 1)), 4)
        systems.append(S)
        defic.append(d)
    return _pack(systems, p, sizes, defic)


def _pair_monomials(deg: int):
    return [(a, t - a) for t in range(deg + 1) for a in range(t, -1, -1)]


def shared_pattern_template(rows: int = 384, cols: int = 400, rhs: int = 16, blocks: int = 16,
                            band: int = 2, deg: int = 4, p: int = P31, seed: int = 4):
    """Block-banded template of bivariate polynomials.

    The coefficient part (cols - rhs columns) is cut into ``blocks`` x
    ``blocks`` blocks; block (I, J) is dense when |I - J| <= band and zero
    otherwise (about 29 % nonzero for 16 blocks and band 2).  The rhs columns
    are dense.  Every nonzero entry is a polynomial in (x, y) of total degree
    <= deg with uniform coefficients.  Returns (mask, coefs, monomials) where
    coefs has shape (nnz, n_monomials) in row-major order of the mask.
    """
    nA = cols - rhs
    assert rows % blocks == 0 and nA % blocks == 0
    br, bc = rows // blocks, nA // blocks
    I = np.arange(rows)[:, None] // br
    J = np.arange(nA)[None, :] // bc
    mask = np.zeros((rows, cols), dtype=bool)
    mask[:, :nA] = np.abs(I - J) <= band
    mask[:, nA:] = True
    mons = _pair_monomials(deg)
    nnz = int(mask.sum())
    coefs = uniform((nnz, len(mons)), p, stream_key(seed, "sp_coefs"))
    return mask, coefs, mons


def shared_pattern(count: int = 4096, rows: int = 384, cols: int = 400, rhs: int = 16,
                   p: int = P31, seed: int = 4, **kw) -> Batch:
    """``count`` evaluations of the template at random points (x, y) in [0, p)^2."""
    mask, coefs, mons = shared_pattern_template(rows, cols, rhs, p=p, seed=seed, **kw)
    pts = uniform((count, 2), p, stream_key(seed, "sp_points")).astype(np.uint64)
    P = np.uint64(p)
    # powers x^a, y^b mod p for a, b <= deg
    deg = max(a + b for a, b in mons)
    xp = np.ones((count, deg + 1), dtype=np.uint64)
    yp = np.ones((count, deg + 1), dtype=np.uint64)
    for e in range(1, deg + 1):
        xp[:, e] = (xp[:, e - 1] * pts[:, 0]) % P
        yp[:, e] = (yp[:, e - 1] * pts[:, 1]) % P
    mono = np.stack([(xp[:, a] * yp[:, b]) % P for a, b in mons], axis=1)   # count x nm
    # entries = mono @ coefs.T mod p, exactly, via a 16-bit split of mono
    lo = (mono & np.uint64(0xFFFF)).astype(np.int64)
    hi = (mono >> np.uint64(16)).astype(np.int64)
    C = coefs.astype(np.int64).T                                            # nm x nnz
    vals = np.empty((count, C.shape[1]), dtype=np.uint32)
    step = 256
    for s0 in range(0, count, step):
        s1 = min(count, s0 + step)
        lo_part = (lo[s0:s1] @ C) % p
        hi_part = (hi[s0:s1] @ C) % p
        vals[s0:s1] = ((lo_part + (hi_part << 16) % p) % p).astype(np.uint32)
    systems = []
    for s in range(count):
        S = np.zeros((rows, cols), dtype=np.uint32)
        S[mask] = vals[s]
        systems.append(S)
    nA = np.full(count, cols - rhs, dtype=np.int32)
    return _pack(systems, p, nA, np.zeros(count, dtype=np.int32))
