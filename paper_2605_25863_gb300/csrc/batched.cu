// batched.cu -- many independent systems of uneven size, each reduced to RREF
// by one thread block, in persistent launches with no inter-block traffic.
//
// Per system the block runs the same blocked Gauss-Jordan elimination as the
// dense driver (paper section 3.2, blocked by panels of NB columns):
//   panel    the pivot window (bt_window_gj): fraction-free Gauss-Jordan
//            elimination of the panel columns of the first w + 8 rows not yet
//            used, with each row's coefficients over the pivot rows, in shared
//            memory; it records the pivot rows and columns and yields
//            E = G^{-1} (G = the pivot rows at the pivot columns) with one
//            inverse per panel.  In shared-pattern mode the window holds the
//            probe's k pivot rows only.  When the window lacks a pivot for a
//            column that a row below it has, a full-height search eliminates
//            all remaining rows, and E then comes from batched inverses of
//            the heads and the panel's recurrence, scaling and back
//            substitution replayed on the identity;
//   tiles    for each 64-column tile right of the panel start: R = E W (W the
//            pivot rows' tile), move the displaced rows, and update every
//            other row: A[d] <- A[d] - F[d] R with lazy signed 64-bit
//            accumulation (F = the rows' entries at the pivot columns).
// Systems are counting-sorted by row count on the device and launched per
// size bucket (shared memory is sized by the bucket's largest system); within
// a bucket blocks pull systems, largest first, from a device work counter.
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <vector>

#include "linac_host.h"
#include "profile.h"
#include "update.cuh"

namespace linac {

constexpr int BT_THREADS = 256;
constexpr int BT_TB = 64;              // column tile of the update
constexpr int BT_NBUCKETS = 5;         // m <= 64, 128, 256, 512, 1024
// largest row count of bucket b: 64, 128, 256, 512, 1024
__host__ __device__ constexpr int bt_bucket_max(int b) { return 64 << b; }
constexpr int BT_FLAG_FALLBACK = 0x100;
constexpr int BT_WINDOW = 8;          // rows of the pivot window beyond the panel width

// The pivot window's slab: bt_win_rows_pad rows of 2 NB + 1 words (NB panel
// entries, NB coefficients over the pivot rows, one pad word against bank
// conflicts).
__host__ __device__ constexpr int bt_win_rows(int nb) { return nb + BT_WINDOW; }
// rows of the slab: bt_win_rows rounded up to whole batches of the block's
// BT_THREADS / nb row groups (the rows beyond the window hold zeros)
__host__ __device__ constexpr int bt_win_rows_pad(int nb) {
    return (bt_win_rows(nb) + BT_THREADS / nb - 1) / (BT_THREADS / nb) * (BT_THREADS / nb);
}
__host__ __device__ constexpr size_t bt_win_bytes(int nb) {
    return (size_t)bt_win_rows_pad(nb) * (2 * nb + 1) * 4;
}

// Per-call device scratch of the batched driver.
struct BatchScratch {
    unsigned int counters[2 * BT_NBUCKETS];   // work counters (search pass, fallback pass)
    int bbeg[BT_NBUCKETS], bend[BT_NBUCKETS]; // bucket segments of `order`
    int probe_m, probe_n, probe_ns;           // shape of the probe system
    int nfallback;                            // systems that left the shared pattern
    int pattern_ok;                           // the probe produced a usable pattern
    int pattern_k[1024 / 16 + 1];             // pivots per panel of the probe
};

// ---------------------------------------------------------------------------
// Sorting by row count (one block): order[] lists systems by bucket, and by
// decreasing m within a bucket.

__global__ void __launch_bounds__(1024)
batch_sort_kernel(const int32_t* __restrict__ dm, int batch, int32_t* __restrict__ order,
                  BatchScratch* bs, int skip_first) {
    __shared__ int cnt[1025];
    __shared__ int pos[1025];
    for (int i = threadIdx.x; i < 1025; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int s = threadIdx.x + skip_first; s < batch; s += blockDim.x) atomicAdd(&cnt[min(max(dm[s], 0), 1024)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        // descending m: pos[v] = number of systems with a key above v
        int acc = 0;
        for (int v = 1024; v >= 0; --v) {
            pos[v] = acc;
            acc += cnt[v];
        }
        // bucket b holds m in (max[b-1], max[b]]: positions [pos[max[b]], pos[max[b-1]])
        for (int b = 0; b < BT_NBUCKETS; ++b) {
            bs->bbeg[b] = pos[bt_bucket_max(b)];
            bs->bend[b] = b ? pos[bt_bucket_max(b - 1)] : acc;
        }
        for (int i = 0; i < 2 * BT_NBUCKETS; ++i) bs->counters[i] = 0;
        bs->nfallback = 0;
    }
    __syncthreads();
    for (int s = threadIdx.x + skip_first; s < batch; s += blockDim.x) {
        const int v = min(max(dm[s], 0), 1024);
        order[atomicAdd(&pos[v], 1)] = s;
    }
}

// ---------------------------------------------------------------------------
// Shared-memory layout of one block (sized by the bucket's largest m).  The
// panel slab is dead once the pivot rows' panel entries are copied out, so
// the multipliers F and the column tiles reuse its space.

struct BtLayout {
    int mmax, ldF;
    size_t off_p, off_ft, off_tiles, off_pu, off_e, off_isp, total;
};

__host__ __device__ inline BtLayout bt_layout(int mmax, int nb) {
    BtLayout L;
    L.mmax = mmax;
    L.ldF = (mmax + 7) / 8 * 8;
    const size_t panel = (size_t)mmax * (nb + 1) * 4;                 // panel slab (all rows)
    const size_t ftb = (size_t)nb * L.ldF * 4;                        // Ft[t][row], balanced
    const size_t tiles = (size_t)4 * nb * BT_TB * 4;                  // V, X, R, next V tiles
    L.off_p = 0;
    L.off_ft = 0;
    L.off_tiles = ftb;
    size_t o = panel > ftb + tiles ? panel : ftb + tiles;
    if (o < bt_win_bytes(nb)) o = bt_win_bytes(nb);                  // pivot window slab
    o = (o + 15) / 16 * 16;
    L.off_pu = o;  o += (size_t)nb * nb * 4;                           // pivot rows' panel entries
    L.off_e = o;   o += (size_t)nb * nb * 4;                           // E^T = (G^{-1})^T, balanced
    L.off_isp = o; o += (size_t)((mmax + 15) / 16 * 16);              // pivot flags
    L.total = (o + 15) / 16 * 16;
    return L;
}

template <int NB>
struct BtSmall {
    int J[NB], Pi[NB], own[NB], srcs[NB], dsts[NB], colt[NB];
    uint32_t hinv[NB], hs[NB];
    int red[BT_THREADS / 32];
    alignas(16) int red2[2][BT_THREADS / 32];
    int s_min, s_sys, s_npairs, s_fail, s_pat;
    uint32_t s_inv;
};

// Block-wide minimum of one int per thread (INT_MAX = none).
template <int NB>
__device__ __forceinline__ int block_min(int v, BtSmall<NB>& sm) {
    v = __reduce_min_sync(0xffffffffu, v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm.red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int x = lane < BT_THREADS / 32 ? sm.red[lane] : INT_MAX;
        x = __reduce_min_sync(0xffffffffu, x);
        if (lane == 0) sm.s_min = x;
    }
    __syncthreads();
    return sm.s_min;
}

// Barrier of the first WT threads of the block: the whole block's barrier,
// or named barrier 1 when fewer threads take part.
template <int WT>
__device__ __forceinline__ void bt_wsync() {
    if (WT == BT_THREADS) __syncthreads();
    else asm volatile("bar.sync 1, %0;" ::"n"(WT) : "memory");
}

// Minimum over the first WT threads with one barrier: each warp posts its
// minimum in one of two alternating slots and every thread reduces the posts
// itself.  A slot is written again two calls later, after another barrier,
// when every thread has read it.
template <int NB, int WT = BT_THREADS>
__device__ __forceinline__ int block_min1(int v, BtSmall<NB>& sm, int& buf) {
    static_assert(WT == 256 || WT == 128, "four or eight warp minima, read as 16-byte words");
    v = __reduce_min_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) sm.red2[buf][threadIdx.x >> 5] = v;
    bt_wsync<WT>();
    const int4 a = *reinterpret_cast<const int4*>(&sm.red2[buf][0]);
    int x = min(min(a.x, a.y), min(a.z, a.w));
    if (WT == 256) {
        const int4 b = *reinterpret_cast<const int4*>(&sm.red2[buf][4]);
        x = min(x, min(min(b.x, b.y), min(b.z, b.w)));
    }
    buf ^= 1;
    return x;
}

// Fold cadence of the lazy accumulators (fold after products t with
// (t & mask) == mask) and the shift form of 2^32 mod p (fold_any,
// reduce_acc in linac_device.cuh; nshift = 0 folds on the multiply pipe).
struct BtFold {
    int mask;
    int nshift;
    FoldShifts fs;
};

// Pivots and E = G^{-1} of one panel from a window of rows, by fraction-free
// Gauss-Jordan elimination of the panel columns c0 .. c0+w-1 augmented with
// each row's coefficients over the pivot rows (one block barrier per column).
//
// Window row i is A row r + i (forced = 0: pivot search, the lowest row with
// a nonzero entry in the column) or A row sm.Pi[i] (forced = 1: the pivot rows
// and columns sm.Pi[t], sm.J[t] of a previous search, in order; rows = k).
// A column cc with a pivot (row q, pivot number s, head h_s = row_q[cc])
// replaces EVERY other row i -- earlier pivot rows, and rows whose entry
// f = row_i[cc] is zero, included -- by h_s * row_i - f * row_q, on the panel
// columns right of cc and on the coefficients 0..s (slab columns NB + u).
// Because every row is scaled alike, the bookkeeping has a closed form: with
// H_s = h_0 h_1 ... h_{s-1},
//     current row i = H_s * (original row i) + sum_u a_iu * (original pivot row u)
// for every row that is not yet a pivot row, so pivot row s takes a_ss = H_s;
// and at the end pivot row t is zero at every other pivot column and holds
// hd_t = h_t h_{t+1} ... h_{k-1} = H_k / H_t at its own, so
// E[t][u] = a_tu / hd_t = a_tu H_t / H_k gives E G = I.  No per-row scale is
// stored, no row branches on its entry f, and one inverse (of H_k) serves the
// whole panel.
//
// The slab holds every value in Montgomery form (x R mod p, R = 2^32), so each
// update h * row_i - f * row_q is two 32 x 32 products and one Montgomery
// reduction (f = 0 enters as p - 0 = p: h x + p y < 2 p^2 < p R still holds);
// zero tests are unaffected.  The products H_s are held the same way.
//
// The w - cc - 1 panel columns and s + 1 <= cc + 1 coefficients that change
// at column cc fit in NB slab columns, so the block is laid out as NB
// columns by WT / NB row groups, and column slot cp of a thread names
// panel column cc + 1 + cp, or coefficient cp - (w - cc - 1).  A thread keeps
// the pivot flags of its own rows in one register.
//
// Only the first WT threads of the block take part (their own barrier when
// WT is below the block size).  WROWS bounds the rows: w + BT_WINDOW for the
// search, NB for the k <= NB pivot rows of shared-pattern mode, whose smaller
// padded slab saves the search window's extra row batch.
//
// Returns the number of pivots k, or -1 in forced mode when a given pivot
// vanished.  Unless forced mode, k == w or keep != 0, E is not needed and is
// not formed; otherwise Et[u * NB + t] = balanced E[t][u] for t, u < k
// rounded up to 4, zero padded.  Fills sm.J, sm.Pi, sm.own (search) and
// sm.hs[t] = H_t (held form).
template <int NB, int WT = BT_THREADS, int WROWS = bt_win_rows(NB)>
__device__ __forceinline__ int bt_window_gj(const uint32_t* __restrict__ A, int64_t ld, int r, int c0, int w, int rows,
                            int forced, int keep, const Field& f, uint32_t* __restrict__ G,
                            BtSmall<NB>& sm, int32_t* __restrict__ Et) {
    constexpr int SWG = 2 * NB + 1;
    constexpr int CW = NB;                  // column slots
    constexpr int RGN = WT / CW;            // row groups
    constexpr int UMAX = (WROWS + RGN - 1) / RGN;
    constexpr int U = UMAX <= 10 ? UMAX : 6;   // rows per batch of independent updates
    static_assert(WT % CW == 0, "column slots must divide the block");
    static_assert(UMAX <= 32, "the pivot flags of a thread's rows fit one word");
    const int tid = threadIdx.x;
    const int cp = tid % CW, rg = tid / CW;
    // load: the panel entries in Montgomery form, coefficients zero; up to 8
    // loads of a thread in flight at once
    constexpr int LPT = (WROWS * NB + WT - 1) / WT;
    constexpr int LB = LPT < 8 ? LPT : 8;
    constexpr int PR = RGN * UMAX;   // slab rows: the rows beyond `rows` hold zeros and stay zero
    static_assert((size_t)PR * SWG * 4 <= bt_win_bytes(NB), "the padded slab fits its region");
    const int nload = rows * NB;
    int cand = INT_MAX;
    for (int e = tid; e < PR * NB; e += WT) {
        const int i = e / NB, c = e % NB;
        G[i * SWG + NB + c] = 0u;
        if (i >= rows) G[i * SWG + c] = 0u;
    }
    for (int e0 = 0; e0 < nload; e0 += LB * WT) {
        uint32_t v[LB];
#pragma unroll
        for (int b = 0; b < LB; ++b) {
            const int e = e0 + b * WT + tid;
            v[b] = 0u;
            if (e < nload) {
                const int i = e / NB, c = e % NB;
                const int64_t arow = forced ? (int64_t)sm.Pi[i] : (int64_t)(r + i);
                if (c < w) v[b] = A[arow * ld + c0 + c];
            }
        }
#pragma unroll
        for (int b = 0; b < LB; ++b) {
            const int e = e0 + b * WT + tid;
            if (e < nload) {
                const int i = e / NB, c = e % NB;
                G[i * SWG + c] = to_mont(v[b], f);
                if (c == 0 && v[b] != 0u && i < cand) cand = i;
            }
        }
    }
    int buf = 0;
    int q = INT_MAX;
    if (forced) bt_wsync<WT>();
    else q = block_min1<NB, WT>(cand, sm, buf);   // also the barrier after the load
    uint32_t Hs = f.c32;   // H_0 = 1, held form R mod p
    uint32_t pmask = 0;    // bit j: window row rg + j RGN is a pivot row
    int s = 0;
    for (int cc = 0; cc < w; ++cc) {
        int qq = -1;   // window row of this column's pivot
        if (forced) {
            if (s < rows && sm.J[s] - c0 == cc) qq = s;
            else continue;   // not a pivot column of the pattern: nothing changes
        } else if (q != INT_MAX) {
            qq = q;
        }
        const bool has = qq >= 0;
        const uint32_t h = has ? G[qq * SWG + cc] : 0u;
        if (has && qq % RGN == rg) pmask |= 1u << (qq / RGN);
        const int np = w - cc - 1;
        int col = -1;
        if (cp < np) col = cc + 1 + cp;
        else if (has && cp - np <= s) col = NB + (cp - np);
        const bool act = has && col >= 0;
        const bool col_s = has && col == NB + s;
        const uint32_t pv = col_s ? Hs : (act ? G[qq * SWG + col] : 0u);
        const bool cand_col = !forced && cp == 0 && np > 0;   // col == cc + 1
        cand = INT_MAX;
        if (act || cand_col) {
            // every row of the padded slab is computed with no row tests
            // (zero padding rows stay zero and never offer a candidate); the
            // pivot row's owner does not store its row, which the other
            // threads read as pv during this step, and sets its coefficient
            // a_ss = H_s instead
            const int uq = (has && qq % RGN == rg) ? qq / RGN : -1;
#pragma unroll
            for (int b0 = 0; b0 < UMAX; b0 += U) {
                uint32_t x[U], fi[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = rg + (b0 + u) * RGN;
                    fi[u] = (b0 + u < UMAX && act) ? G[i * SWG + cc] : 0u;
                    x[u] = b0 + u < UMAX ? G[i * SWG + col] : 0u;
                }
                if (act) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (b0 + u < UMAX) {
                            x[u] = mont_mul2add(h, x[u], f.p - fi[u], pv, f);
                            if (b0 + u != uq) G[(rg + (b0 + u) * RGN) * SWG + col] = x[u];
                        }
                    }
                }
                if (cand_col) {
                    // the lowest row of this thread that is nonzero in column
                    // cc + 1 and not yet a pivot row
                    uint32_t nz = 0u;
#pragma unroll
                    for (int u = 0; u < U; ++u) nz |= (b0 + u < UMAX && x[u] != 0u) ? (1u << (b0 + u)) : 0u;
                    nz &= ~pmask;
                    if (nz != 0u && cand == INT_MAX) cand = rg + (__ffs((int)nz) - 1) * RGN;
                }
            }
            if (col_s && uq >= 0) G[qq * SWG + col] = Hs;
        }
        if (has) {
            if (tid == 0) {
                sm.hs[s] = Hs;
                if (!forced) {
                    sm.J[s] = c0 + cc;
                    sm.Pi[s] = r + qq;
                    sm.own[s] = qq;
                }
            }
            Hs = mont_mul(h, Hs, f);
            ++s;
        }
        // forced mode: a reused pivot that vanished ends the panel (h is the
        // same in every thread, so the whole block returns; a pivot found by
        // the search is nonzero)
        if (forced && h == 0u) return -1;
        if (!forced && cc + 1 < w) q = block_min1<NB, WT>(cand, sm, buf);
        else bt_wsync<WT>();
    }
    const int k = s;
    if (!forced && k < w && !keep) return k;
    // 1 / (hd_t R) = H_t / (H_k R): one inverse of the held H_k, then one
    // Montgomery product by the held H_t per pivot
    if (tid < 32) {
        const uint32_t inv = inverse_fermat(Hs, f);
        if (tid == 0) sm.s_inv = inv;
    }
    bt_wsync<WT>();
    const uint32_t invH = sm.s_inv;
    const int kp = (k + 3) & ~3;
    for (int e = tid; e < kp * kp; e += WT) {
        const int u = e / kp, t = e % kp;
        int32_t v = 0;
        if (t < k && u < k) {
            const uint32_t hinv = mont_mul(sm.hs[t], invH, f);
            v = to_balanced(mulmod(G[(forced ? t : sm.own[t]) * SWG + NB + u], hinv, f), f);
        }
        Et[u * NB + t] = v;
    }
    bt_wsync<WT>();
    return k;
}

// The K loop of a tile product: acc[a][b] += X[t][a] * Y[t][b] for t < k,
// with X rows of MR values (stride ldx) and Y rows of 4 values (stride ldy),
// all balanced residues (YBAL: Y holds raw residues, balanced on the fly).
// The loop is unrolled by the fold cadence FOLD, so the folds sit at fixed
// places and the shared-memory reads of a group issue together; the last
// group or the last k mod FOLD products need no fold before the final
// reduction (at most FOLD products after a fold keep |acc| < 2^63).
template <int FOLD, int MR, int SH, bool YBAL>
__device__ __forceinline__ void bt_kloop(int64_t (&acc)[MR][4], const int32_t* __restrict__ X, int ldx,
                                         const int32_t* __restrict__ Y, int ldy, int k, const Field& f,
                                         const FoldShifts& fs) {
    static_assert(MR == 2 || MR == 4 || MR == 8, "two, four or eight rows per item");
    auto step = [&](int t) {
        int xa[MR];
        if (MR == 2) {
            const int2 x0 = *reinterpret_cast<const int2*>(X + t * ldx);
            xa[0] = x0.x; xa[MR - 1] = x0.y;
        } else {
            const int4 x0 = *reinterpret_cast<const int4*>(X + t * ldx);
            xa[0] = x0.x; xa[1 % MR] = x0.y; xa[2 % MR] = x0.z; xa[3 % MR] = x0.w;
        }
        if (MR == 8) {
            const int4 x1 = *reinterpret_cast<const int4*>(X + t * ldx + 4);
            xa[MR - 4] = x1.x; xa[MR - 3] = x1.y; xa[MR - 2] = x1.z; xa[MR - 1] = x1.w;
        }
        const int4 yv = *reinterpret_cast<const int4*>(Y + t * ldy);
        int yb[4] = {yv.x, yv.y, yv.z, yv.w};
        if (YBAL) {
#pragma unroll
            for (int b = 0; b < 4; ++b) yb[b] = to_balanced((uint32_t)yb[b], f);
        }
#pragma unroll
        for (int a = 0; a < MR; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += (int64_t)xa[a] * yb[b];
    };
    // groups of FOLD products, each followed by a fold, except the last group
    // when no product follows it (FOLD products after a fold stay below
    // 2^63, which the final reduction accepts)
    const int kf = k - k % FOLD;
    const int kfold = k % FOLD == 0 ? kf - FOLD : kf;   // groups before kfold are folded
    int t0 = 0;
    for (; t0 < kfold; t0 += FOLD) {
#pragma unroll
        for (int tt = 0; tt < FOLD; ++tt) step(t0 + tt);
#pragma unroll
        for (int a = 0; a < MR; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fold_any<SH>(acc[a][b], f, fs);
    }
    if (t0 < kf) {
#pragma unroll
        for (int tt = 0; tt < FOLD; ++tt) step(t0 + tt);
    }
    for (int t = kf; t < k; ++t) step(t);
}

// Reduce system A (m x n, leading dimension ld) in place.  mode 0: pivot
// search; mode 1: reuse the probe's pattern (pat_J / pat_Pi / pat_k per
// panel) and report failure (returns false) when a reused pivot vanishes or
// the result leaves echelon form.  Returns true on success; writes rank and
// pivots.
template <int NB, int SH>
__device__ __forceinline__ bool bt_reduce(uint32_t* __restrict__ A, int m, int n, int64_t ld, int ns, const Field& f,
                          const BtFold& fo, int32_t* __restrict__ piv, int* rank_out, uint8_t* smem,
                          const BtLayout& L, BtSmall<NB>& sm, int mode, const int32_t* pat_J,
                          const int32_t* pat_Pi, const int* pat_k, int32_t* rec_J, int32_t* rec_Pi, int* rec_k) {
    uint32_t* P = (uint32_t*)(smem + L.off_p);
    int32_t* Ft = (int32_t*)(smem + L.off_ft);
    uint32_t* V = (uint32_t*)(smem + L.off_tiles);
    uint32_t* X = V + NB * BT_TB;
    int32_t* Rt = (int32_t*)(V + 2 * NB * BT_TB);
    uint32_t* Vnext = V + 3 * NB * BT_TB;
    uint32_t* PU = (uint32_t*)(smem + L.off_pu);
    int32_t* Et = (int32_t*)(smem + L.off_e);
    uint32_t* E = (uint32_t*)Et;
    unsigned char* isp = smem + L.off_isp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = BT_THREADS / 32;
    const int SW = NB + 1;
    const int ldF = L.ldF;

    const int npiv = min(m, ns);
    for (int i = tid; i < npiv; i += BT_THREADS) piv[i] = -1;
    // 16-byte row accesses only when the system's start and rows are aligned
    // (offsets and leading dimensions are device data the host cannot check)
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && ((ld & 3) == 0);
    int r = 0;
    int panel = 0;
    for (int c0 = 0; c0 < ns && r < m; c0 += NB, ++panel) {
        const int w = min(NB, ns - c0);
        int k = 0;
        bool e_ready = true;
        if (mode == 0) {
            // Pivots from a window of the first w + BT_WINDOW remaining rows,
            // with E from the same Gauss-Jordan pass.  The RREF does not depend
            // on which rows supply the pivots, so the window's choice stands
            // when it has a pivot in every panel column or holds every
            // remaining row; otherwise the search covers all remaining rows
            // with the fraction-free panel elimination, and E follows from its
            // record.
            const int rows_all = m - r;
            const int wrows = min(rows_all, w + BT_WINDOW);
            k = bt_window_gj<NB>(A, ld, r, c0, w, wrows, 0, wrows == rows_all, f, P, sm, Et);
            e_ready = k == w || wrows == rows_all;
            if (!e_ready) {
                const int rows = rows_all;
                k = 0;
                for (int e = tid; e < rows * w; e += BT_THREADS) {
                    const int i = e / w, j = e % w;
                    P[i * SW + j] = A[(int64_t)(r + i) * ld + c0 + j];
                }
                for (int i = tid; i < rows; i += BT_THREADS) isp[i] = 0;
                __syncthreads();
                // candidate for the first column
                int cand = INT_MAX;
                for (int i = tid; i < rows; i += BT_THREADS)
                    if (P[i * SW] != 0) { cand = i; break; }
                int q = block_min<NB>(cand, sm);
                for (int cc = 0; cc < w; ++cc) {
                    // q: lowest non-pivot row with a nonzero entry in column cc
                    if (q != INT_MAX) {
                        if (tid == 0) {
                            isp[q] = 1;
                            sm.J[k] = c0 + cc;
                            sm.Pi[k] = r + q;
                            sm.own[k] = q;
                        }
                        ++k;
                    }
                    // eliminate column cc (fraction-free) and look for the next
                    // column's candidate in the same pass over the rows
                    cand = INT_MAX;
                    const uint32_t h = q != INT_MAX ? P[q * SW + cc] : 0u;
                    for (int i = warp; i < rows; i += NW) {
                        if (i == q || isp[i]) continue;
                        uint32_t* row = P + i * SW;
                        if (q != INT_MAX) {
                            const uint32_t fi = row[cc];
                            if (fi != 0) {
                                const uint32_t nf = f.p - fi;
                                for (int j = cc + 1 + lane; j < w; j += 32)
                                    row[j] = mul2add(h, row[j], nf, P[q * SW + j], f);
                            }
                            __syncwarp();
                        }
                        if (cc + 1 < w && lane == 0 && row[cc + 1] != 0 && i < cand) cand = i;
                    }
                    if (cc + 1 < w) q = block_min<NB>(cand, sm);
                    else __syncthreads();
                }
                for (int e = tid; e < k * w; e += BT_THREADS) {
                    const int t = e / w, j = e % w;
                    PU[t * NB + j] = P[sm.own[t] * SW + j];
                }
            }
            if (rec_k && tid == 0) {
                rec_k[panel] = k;
                for (int t = 0; t < k; ++t) {
                    rec_J[panel * NB + t] = sm.J[t];
                    rec_Pi[panel * NB + t] = sm.Pi[t];
                }
            }
            __syncthreads();   // the slab is dead from here on (F and the tiles reuse it)
        } else {
            // shared pattern: the probe's pivot rows and columns, eliminated in
            // their order (the steps the search would have taken on them)
            k = pat_k[panel];
            for (int t = tid; t < k; t += BT_THREADS) {
                sm.J[t] = pat_J[panel * NB + t];
                sm.Pi[t] = pat_Pi[panel * NB + t];
            }
            if (tid == 0) sm.s_fail = 0;
            __syncthreads();
            if (bt_window_gj<NB, BT_THREADS, NB>(A, ld, r, c0, w, k, 1, 1, f, P, sm, Et) < 0) return false;
        }
        if (k == 0) continue;
        // kp = k rounded up to 4 (E^T and the tiles are zero padded to it)
        const int kp = (k + 3) & ~3;
        // the pivot rows' first column tile V (raw residues), copied with
        // cp.async now, so it lands during the F load; later tiles are copied
        // one tile ahead, during the previous tile's update (which writes only
        // its own tile's columns, so the next tile of the pivot rows is final).
        // Without 16-byte row alignment the copy is synchronous.  The window
        // slab, which the tiles may overlap, is dead here.
        uint32_t* Vcur = V;
        uint32_t* Vnxt = Vnext;
        auto fetch_v = [&](int j0v, uint32_t* dst) {
            const int twv = min(BT_TB, n - j0v);
            if (vec_ok) {
                for (int e = tid; e < kp * (BT_TB / 4); e += BT_THREADS) {
                    const int t = e / (BT_TB / 4), j = (e % (BT_TB / 4)) * 4;
                    const int bytes = (t < k && j < twv) ? min(4, twv - j) * 4 : 0;
                    const uint32_t* src = bytes ? A + (int64_t)sm.Pi[t] * ld + j0v + j : A;
                    cp_async16(dst + t * BT_TB + j, src, bytes);
                }
                cp_async_commit();
            } else {
                for (int e = tid; e < kp * BT_TB; e += BT_THREADS) {
                    const int t = e / BT_TB, j = e % BT_TB;
                    dst[t * BT_TB + j] = (t < k && j < twv) ? A[(int64_t)sm.Pi[t] * ld + j0v + j] : 0u;
                }
            }
        };
        fetch_v(c0, Vcur);
        // multipliers F (original entries at the pivot columns, all of which lie
        // in the panel's w columns): each row's panel segment is read as
        // 16-byte words, coalesced, and every entry of a pivot column is
        // written to F through the column -> pivot map colt
        if (tid < 32) {
            for (int j = tid; j < NB; j += 32) sm.colt[j] = -1;
            __syncwarp();
            for (int t = tid; t < k; t += 32) sm.colt[sm.J[t] - c0] = t;
        }
        __syncthreads();
        {
            const int wq = (w + 3) >> 2;
            const int nq = m * wq;
            constexpr int FB = 4;   // 16-byte loads of a thread in flight at once
            for (int e0 = tid; e0 < nq; e0 += FB * BT_THREADS) {
                uint4 v[FB];
#pragma unroll
                for (int b = 0; b < FB; ++b) {
                    const int e = e0 + b * BT_THREADS;
                    v[b] = make_uint4(0u, 0u, 0u, 0u);
                    if (e < nq) {
                        const int i = e / wq, q = e - i * wq;
                        const uint32_t* src = A + (int64_t)i * ld + c0 + 4 * q;   // 4 q < w
                        if (vec_ok && 4 * q + 4 <= w) {
                            v[b] = *reinterpret_cast<const uint4*>(src);
                        } else {
                            v[b].x = src[0];
                            v[b].y = 4 * q + 1 < w ? src[1] : 0u;
                            v[b].z = 4 * q + 2 < w ? src[2] : 0u;
                            v[b].w = 4 * q + 3 < w ? src[3] : 0u;
                        }
                    }
                }
#pragma unroll
                for (int b = 0; b < FB; ++b) {
                    const int e = e0 + b * BT_THREADS;
                    if (e < nq) {
                        const int i = e / wq, q = e - i * wq;
                        const uint32_t v4[4] = {v[b].x, v[b].y, v[b].z, v[b].w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int t = 4 * q + u < w ? sm.colt[4 * q + u] : -1;
                            if (t >= 0) Ft[t * ldF + i] = to_balanced(v4[u], f);
                        }
                    }
                }
            }
        }
        if (!e_ready) {
            for (int t = tid; t < k; t += BT_THREADS) {
                sm.hs[t] = PU[t * NB + (sm.J[t] - c0)];
                sm.hinv[t] = inverse_mod(sm.hs[t], f.p);
            }
            for (int e = tid; e < k * k; e += BT_THREADS) E[(e / k) * NB + (e % k)] = (e / k == e % k) ? 1u : 0u;
        }
        if (tid < 32) {
            // move plan (warp 0): the rows of [r, r+k) without a pivot, in
            // order, go to the pivot rows' old places outside [r, r+k), in
            // pivot order (k <= NB <= 64: one 64-bit occupancy mask)
            static_assert(NB <= 64, "occupancy of [r, r+k) in one 64-bit mask");
            const unsigned full = 0xffffffffu;
            unsigned long long occ = 0;
            for (int t = tid; t < k; t += 32) {
                const int d = sm.Pi[t] - r;
                if (d >= 0 && d < k) occ |= 1ull << d;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) occ |= __shfl_xor_sync(full, occ, o);
            const unsigned below = (1u << tid) - 1u;
            int na = 0, nb2 = 0;
            for (int d0 = 0; d0 < k; d0 += 32) {
                const int d = d0 + tid;
                const bool freed = d < k && !((occ >> d) & 1ull);
                const unsigned bal = __ballot_sync(full, freed);
                if (freed) sm.srcs[na + __popc(bal & below)] = r + d;
                na += __popc(bal);
            }
            for (int t0 = 0; t0 < k; t0 += 32) {
                const int t = t0 + tid;
                const bool out = t < k && (sm.Pi[t] < r || sm.Pi[t] >= r + k);
                const unsigned bal = __ballot_sync(full, out);
                if (out) sm.dsts[nb2 + __popc(bal & below)] = sm.Pi[t];
                nb2 += __popc(bal);
            }
            if (tid == 0) sm.s_npairs = na;
        }
        __syncthreads();
        if (!e_ready) {
            // E <- forward fraction-free recurrence, scaling, back substitution
            for (int s = 0; s + 1 < k; ++s) {
                const uint32_t h = sm.hs[s];
                const int cs = sm.J[s] - c0;
                for (int e = tid; e < (k - 1 - s) * k; e += BT_THREADS) {
                    const int t = s + 1 + e / k, j = e % k;
                    const uint32_t fts = PU[t * NB + cs];
                    if (fts) E[t * NB + j] = mul2add(h, E[t * NB + j], f.p - fts, E[s * NB + j], f);
                }
                __syncthreads();
            }
            for (int e = tid; e < k * k; e += BT_THREADS) {
                const int t = e / k, j = e % k;
                E[t * NB + j] = mulmod(E[t * NB + j], sm.hinv[t], f);
            }
            __syncthreads();
            for (int s = k - 1; s >= 1; --s) {
                const int cs = sm.J[s] - c0;
                for (int e = tid; e < s * k; e += BT_THREADS) {
                    const int t = e / k, j = e % k;
                    const uint32_t c = mulmod(PU[t * NB + cs], sm.hinv[t], f);
                    if (c) E[t * NB + j] = mul2add(1u, E[t * NB + j], f.p - c, E[s * NB + j], f);
                }
                __syncthreads();
            }
        }
        const int npairs = sm.s_npairs;
        for (int e = tid; e < npairs * k; e += BT_THREADS) {
            const int t = e / npairs, a = e % npairs;
            Ft[t * ldF + sm.dsts[a]] = Ft[t * ldF + sm.srcs[a]];
        }
        // E^T in balanced form (register-tiled R = E V reads 4 consecutive t),
        // zero padded to kp
        if (!e_ready) {
            // transpose through registers: each thread owns whole (t, s) entries
            uint32_t v[NB * NB / BT_THREADS + 1];
            int cnt = 0;
            for (int e = tid; e < kp * kp; e += BT_THREADS, ++cnt) {
                const int t = e / kp, s2 = e % kp;
                v[cnt] = (t < k && s2 < k) ? (uint32_t)to_balanced(E[t * NB + s2], f) : 0u;
            }
            __syncthreads();
            cnt = 0;
            for (int e = tid; e < kp * kp; e += BT_THREADS, ++cnt) {
                const int t = e / kp, s2 = e % kp;
                Et[s2 * NB + t] = (int32_t)v[cnt];
            }
        }
        // column tiles (the first barrier of the tile loop also orders the F
        // moves and E^T above before anything reads them)
        for (int j0 = c0; j0 < n; j0 += BT_TB) {
            const int tw = min(BT_TB, n - j0);
            for (int e = tid; e < npairs * tw; e += BT_THREADS) {
                const int a = e / tw, j = e % tw;
                X[a * BT_TB + j] = A[(int64_t)sm.srcs[a] * ld + j0 + j];
            }
            cp_async_wait<0>();
            __syncthreads();
            // R = E V, 2 x 4 outputs per thread (balanced operands, lazy
            // signed accumulation): k/2 x 16 items keep every thread busy
            for (int e = tid; e < (kp / 2) * (BT_TB / 4); e += BT_THREADS) {
                const int t0 = (e / (BT_TB / 4)) * 2, jq = (e % (BT_TB / 4)) * 4;
                int64_t acc[2][4];
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
                if (fo.mask == 7)
                    bt_kloop<8, 2, SH, true>(acc, Et + t0, NB, (const int32_t*)Vcur + jq, BT_TB, kp, f, fo.fs);
                else
                    bt_kloop<4, 2, SH, true>(acc, Et + t0, NB, (const int32_t*)Vcur + jq, BT_TB, kp, f, fo.fs);
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) Rt[(t0 + a) * BT_TB + jq + b] = to_balanced(reduce_acc<SH>(acc[a][b], f, fo.fs), f);
            }
            for (int e = tid; e < npairs * tw; e += BT_THREADS) {
                const int a = e / tw, j = e % tw;
                A[(int64_t)sm.dsts[a] * ld + j0 + j] = X[a * BT_TB + j];
            }
            __syncthreads();
            // the next tile's V, in flight during this tile's update
            if (j0 + BT_TB < n) fetch_v(j0 + BT_TB, Vnxt);
            {
                uint32_t* tmp = Vcur;
                Vcur = Vnxt;
                Vnxt = tmp;
            }
            // update: rows in [r, r+k) receive R, every other row A -= F R
            // (MR rows x 4 columns per work item; MR = 8 for 64-column panels,
            // whose blocks own an SM alone, 4 otherwise).  The item's
            // current values are prefetched before the products when the
            // registers allow (PREF), else read four rows at a time after the
            // products (loads cannot pass the item's earlier stores to the
            // same matrix), where the other warps' products hide their latency.
            constexpr int MR = NB >= 64 ? 8 : 4;
            constexpr bool PREF = MR == 4 || NB >= 64;
            const int rgroups = (m + MR - 1) / MR;
            constexpr int cq = BT_TB / 4;
            for (int e = tid; e < rgroups * cq; e += BT_THREADS) {
                const int d0 = (e / cq) * MR, jq = (e % cq) * 4;
                if (jq >= tw) continue;
                auto load_cur = [&](int d) {
                    uint4 c = make_uint4(0u, 0u, 0u, 0u);
                    const uint32_t* rowp = A + (int64_t)d * ld + j0 + jq;
                    if (d < m && jq + 4 <= tw && vec_ok) c = *reinterpret_cast<const uint4*>(rowp);
                    else if (d < m) {
                        c.x = rowp[0];
                        c.y = jq + 1 < tw ? rowp[1] : 0u;
                        c.z = jq + 2 < tw ? rowp[2] : 0u;
                        c.w = jq + 3 < tw ? rowp[3] : 0u;
                    }
                    return c;
                };
                uint4 cur[MR];
                if (PREF) {
#pragma unroll
                    for (int a = 0; a < MR; ++a) cur[a] = load_cur(d0 + a);
                }
                int64_t acc[MR][4];
#pragma unroll
                for (int a = 0; a < MR; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
                if (fo.mask == 7)
                    bt_kloop<8, MR, SH, false>(acc, Ft + d0, ldF, Rt + jq, BT_TB, k, f, fo.fs);
                else
                    bt_kloop<4, MR, SH, false>(acc, Ft + d0, ldF, Rt + jq, BT_TB, k, f, fo.fs);
#pragma unroll
                for (int a = 0; a < MR; ++a) {
                    // without the prefetch, the current values of four rows
                    // at a time are read before their stores
                    if (!PREF && (a & 3) == 0) {
#pragma unroll
                        for (int a2 = 0; a2 < 4; ++a2) cur[a + a2] = load_cur(d0 + a + a2);
                    }
                    const int d = d0 + a;
                    if (d >= m) continue;
                    uint32_t* row = A + (int64_t)d * ld + j0;
                    const bool prow = d >= r && d < r + k;
                    const uint32_t c4[4] = {cur[a].x, cur[a].y, cur[a].z, cur[a].w};
                    uint32_t o4[4];
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int j = jq + b;
                        uint32_t v = 0;
                        if (j < tw) {
                            if (prow) v = from_balanced(Rt[(d - r) * BT_TB + j], f);
                            else v = submod(c4[b], reduce_acc<SH>(acc[a][b], f, fo.fs), f);
                        }
                        o4[b] = v;
                        // shared pattern: rows below the new rank must vanish in the panel
                        if (mode == 1 && d >= r + k && j < tw && j0 + j < c0 + w && v != 0) sm.s_fail = 1;
                    }
                    if (jq + 4 <= tw && vec_ok) {
                        *reinterpret_cast<uint4*>(row + jq) = make_uint4(o4[0], o4[1], o4[2], o4[3]);
                    } else {
                        for (int b = 0; b < 4 && jq + b < tw; ++b) row[jq + b] = o4[b];
                    }
                }
            }
            __syncthreads();
        }
        for (int t = tid; t < k; t += BT_THREADS) piv[r + t] = sm.J[t];
        r += k;
        __syncthreads();
        if (mode == 1) {
            // echelon shape: a pivot row is zero left of its pivot within the panel
            for (int e = tid; e < k * w; e += BT_THREADS) {
                const int t = e / w, j = e % w;
                if (c0 + j < sm.J[t] && A[(int64_t)(r - k + t) * ld + c0 + j] != 0) sm.s_fail = 1;
            }
            __syncthreads();
            if (sm.s_fail) return false;
        }
    }
    if (mode == 1 && r < m) {
        // the probe's rank was reached: every remaining row must be zero in
        // the searched columns, or this system has a different pattern
        for (int e = tid; e < (m - r) * ns; e += BT_THREADS) {
            const int i = r + e / ns, j = e % ns;
            if (A[(int64_t)i * ld + j] != 0) sm.s_fail = 1;
        }
        __syncthreads();
        if (sm.s_fail) return false;
    }
    *rank_out = r;
    return true;
}

// Panel width of each size bucket for one launch.
struct BtWidths {
    int nb[BT_NBUCKETS];
};

__host__ __device__ inline int bt_bucket_of(int m) {
    int b = 0;
    while (b + 1 < BT_NBUCKETS && m > bt_bucket_max(b)) ++b;
    return b;
}

// Persistent kernel over the size buckets blo..bhi, which share the panel
// width NB (one launch for all buckets of one width whose shared-memory needs
// allow the same blocks per SM).  Blocks pull systems, largest first, from a
// device work counter.  pass 0: the buckets' systems (search, or the shared
// pattern); pass 1: systems that failed the pattern (search).
template <int NB, int SH>
__global__ void __launch_bounds__(BT_THREADS, NB >= 64 ? 1 : 2)
batched_kernel(uint32_t* __restrict__ data, const int64_t* __restrict__ offsets, const int32_t* __restrict__ dm,
               const int32_t* __restrict__ dn, const int32_t* __restrict__ dld, const int32_t* __restrict__ dns,
               const int32_t* __restrict__ order, int blo, int bhi, Field f, int32_t* __restrict__ ranks,
               int32_t* __restrict__ pivots, const int64_t* __restrict__ piv_off, int32_t* __restrict__ sys_status,
               BatchScratch* bs, int pass, int use_pattern, const int32_t* pat_J, const int32_t* pat_Pi,
               int32_t* fallback, BtFold fo, int probe) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ BtSmall<NB> sm;
    const BtLayout L = bt_layout(bt_bucket_max(bhi), NB);   // sized for the group's largest systems
    if (probe && blockIdx.x == 0) {
        // the probe: system 0 with the pivot search, recording its pattern,
        // which is then published; the other blocks meanwhile reduce their
        // systems with the search and take the pattern once it is there
        const int m0 = dm[0], n0 = dn[0];
        const int ns0 = dns ? min(dns[0], n0) : n0;
        int rank0 = 0;
        bt_reduce<NB, SH>(data + offsets[0], m0, n0, dld[0], ns0, f, fo, pivots + piv_off[0], &rank0, smem, L, sm, 0,
                          nullptr, nullptr, nullptr, (int32_t*)pat_J, (int32_t*)pat_Pi, bs->pattern_k);
        __syncthreads();
        if (threadIdx.x == 0) {
            ranks[0] = rank0;
            if (sys_status) sys_status[0] = 0;
            bs->probe_m = m0;
            bs->probe_n = n0;
            bs->probe_ns = ns0;
            __threadfence();   // the pattern and the probe's shape before the flag
            atomicExch(&bs->pattern_ok, 1);
        }
        __syncthreads();
    }
    int begin, end;
    if (pass == 0) {
        begin = bs->bbeg[bhi];
        end = bs->bend[blo];
    } else {
        begin = 0;
        end = bs->nfallback;
    }
    unsigned int* counter = &bs->counters[pass * BT_NBUCKETS + blo];
    for (;;) {
        if (threadIdx.x == 0) {
            sm.s_sys = (int)atomicAdd(counter, 1u);
            // the shared pattern, once the probe has published it (no waiting:
            // a system pulled before that is reduced with the search)
            int pat = 0;
            if (use_pattern && pass == 0) {
                pat = *(volatile int*)&bs->pattern_ok;
                if (pat) __threadfence();   // the probe's pattern is visible after the flag
            }
            sm.s_pat = pat;
        }
        __syncthreads();
        const int idx = begin + sm.s_sys;
        __syncthreads();
        if (idx >= end) return;
        const int s = pass == 0 ? order[idx] : fallback[idx];
        const int m = dm[s], n = dn[s];
        if (pass == 1) {   // fallback systems are split by bucket too
            const int b = bt_bucket_of(m);
            if (b < blo || b > bhi) continue;
        }
        const int ns = dns ? min(dns[s], n) : n;
        uint32_t* A = data + offsets[s];
        int32_t* piv = pivots + piv_off[s];
        int rank = 0;
        bool ok = false;
        // the pattern applies only to systems shaped like the probe
        const bool same_shape = m == bs->probe_m && n == bs->probe_n && ns == bs->probe_ns;
        const int mode = sm.s_pat ? 1 : 0;
        // two call sites so that each is specialised for its mode
        if (mode == 1 && !same_shape) ok = false;
        else if (mode == 1)
            ok = bt_reduce<NB, SH>(A, m, n, dld[s], ns, f, fo, piv, &rank, smem, L, sm, 1, pat_J, pat_Pi,
                               bs->pattern_k, nullptr, nullptr, nullptr);
        else
            ok = bt_reduce<NB, SH>(A, m, n, dld[s], ns, f, fo, piv, &rank, smem, L, sm, 0, nullptr, nullptr, nullptr,
                               nullptr, nullptr, nullptr);
        if (mode == 1 && !ok && threadIdx.x == 0) fallback[atomicAdd(&bs->nfallback, 1)] = s;
        __syncthreads();
        if (ok && threadIdx.x == 0) {
            ranks[s] = rank;
            if (sys_status) sys_status[s] = pass == 1 ? BT_FLAG_FALLBACK : 0;
        }
        __syncthreads();
    }
}

// Probe: system 0 with the pivot search, recording its pattern.
template <int NB>
__global__ void __launch_bounds__(BT_THREADS)
batched_probe_kernel(uint32_t* __restrict__ data, const int64_t* __restrict__ offsets, const int32_t* __restrict__ dm,
                     const int32_t* __restrict__ dn, const int32_t* __restrict__ dld, const int32_t* __restrict__ dns,
                     int mmax, Field f, int32_t* __restrict__ ranks, int32_t* __restrict__ pivots,
                     const int64_t* __restrict__ piv_off, int32_t* __restrict__ sys_status, BatchScratch* bs,
                     int32_t* pat_J, int32_t* pat_Pi, BtFold fo) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ BtSmall<NB> sm;
    const BtLayout L = bt_layout(mmax, NB);
    const int m = dm[0], n = dn[0];
    const int ns = dns ? min(dns[0], n) : n;
    for (int i = threadIdx.x; i < 1024 / 16 + 1; i += BT_THREADS) bs->pattern_k[i] = 0;
    __syncthreads();
    int rank = 0;
    bt_reduce<NB, 0>(data + offsets[0], m, n, dld[0], ns, f, fo, pivots + piv_off[0], &rank, smem, L, sm, 0, nullptr,
                  nullptr, nullptr, pat_J, pat_Pi, bs->pattern_k);
    __syncthreads();
    if (threadIdx.x == 0) {
        ranks[0] = rank;
        if (sys_status) sys_status[0] = 0;
        bs->probe_m = m;
        bs->probe_n = n;
        bs->probe_ns = ns;
        bs->pattern_ok = 1;
    }
}

// ---------------------------------------------------------------------------
// Host side: per-bucket panel width (autotuned table, see linac_batched_tune)

namespace {
std::mutex g_bt_mu;
int g_bt_nb[64][BT_NBUCKETS];   // 0 = default
}

static int bt_default_nb(int b) { (void)b; return 32; }

// The shift form is used only when 2^32 mod p is a single power of two
// (2^31 - 1): with two or three shifts the fold issues more ALU instructions
// than the multiply-pipe form it replaces, and this kernel is bound by issue
// and latency rather than by the multiply pipe.  The final reduction takes
// two folds and two conditional subtractions (reduce_alu) whenever
// c32 = 2^32 mod p is small enough, whatever its bit count (2^31 - 19:
// c32 = 38), and the Barrett reduction otherwise.
static BtFold bt_fold_params(const Field& f) {
    BtFold fo;
    fo.mask = f.fold >= 8 ? 7 : 3;
    fo.nshift = fold_shifts(f, &fo.fs);
    if (fo.nshift != 1) fo.nshift = 0;
    const unsigned __int128 cc = f.c32;
    const bool low_ok = cc * (cc + 1) / 2 <= f.p;
    const bool high_ok = (((unsigned __int128)1) << 32) - 1 + cc * (cc / 2 + 1) < (unsigned __int128)3 * f.p;
    fo.fs.alu_reduce = low_ok && high_ok;
    return fo;
}

// batched_kernel<nb, sh> (nullptr for an unsupported width).
static const void* bt_kernel_fn(int nb, int sh) {
    switch (nb) {
        case 16: return sh == 1 ? (const void*)batched_kernel<16, 1> : (const void*)batched_kernel<16, 0>;
        case 32: return sh == 1 ? (const void*)batched_kernel<32, 1> : (const void*)batched_kernel<32, 0>;
        case 64: return sh == 1 ? (const void*)batched_kernel<64, 1> : (const void*)batched_kernel<64, 0>;
        default: return nullptr;
    }
}

int bt_bucket_nb(int b) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_bt_mu);
    const int v = (dev >= 0 && dev < 64) ? g_bt_nb[dev][b] : 0;
    return v ? v : bt_default_nb(b);
}

void bt_set_bucket_nb(int b, int nb) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_bt_mu);
    if (dev >= 0 && dev < 64 && b >= 0 && b < BT_NBUCKETS) g_bt_nb[dev][b] = nb;
}

// Blocks per SM of one launch over buckets blo..bhi with widths wd (0 when
// the launch does not fit).
static int bt_group_occupancy(int blo, int bhi, const BtWidths& wd, int sh, size_t* smem_out) {
    size_t smem = 0;
    for (int b = blo; b <= bhi; ++b) {
        if (wd.nb[b] != wd.nb[blo]) return 0;   // one width per launch
        smem = std::max(smem, bt_layout(bt_bucket_max(b), wd.nb[b]).total);
    }
    int max_smem = 0;
    max_smem = max_smem_optin();
    if (max_smem <= 0) return 0;
    if (smem + sizeof(BtSmall<64>) > (size_t)max_smem) return 0;
    const void* fn = bt_kernel_fn(wd.nb[blo], sh);
    if (!fn) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, BT_THREADS, smem) != cudaSuccess) return 0;
    if (smem_out) *smem_out = smem;
    return occ;
}

static linac_status launch_group(int blo, int bhi, int pass, int use_pattern, int probe, const BtWidths& wd,
                                 uint32_t* d_data, const int64_t* d_offsets, const int32_t* d_m, const int32_t* d_n,
                                 const int32_t* d_ld, const int32_t* d_nsearch, const int32_t* order,
                                 const Field& f, int32_t* d_ranks, int32_t* d_pivots, const int64_t* d_piv_offsets,
                                 int32_t* d_status, BatchScratch* bs, const int32_t* pat_J, const int32_t* pat_Pi,
                                 int32_t* fallback, cudaStream_t stream) {
    size_t smem = 0;
    BtFold fo = bt_fold_params(f);
    const int occ = bt_group_occupancy(blo, bhi, wd, fo.nshift, &smem);
    (void)cudaGetLastError();
    if (occ < 1) return LINAC_ERR_UNSUPPORTED;
    const void* fn = bt_kernel_fn(wd.nb[blo], fo.nshift);
    if (!fn) return LINAC_ERR_ARG;
    const int grid = occ * sm_count();
    Field fv = f;
    void* args[] = {&d_data, (void*)&d_offsets, (void*)&d_m, (void*)&d_n, (void*)&d_ld, (void*)&d_nsearch,
                    (void*)&order, &blo, &bhi, &fv, &d_ranks, &d_pivots, (void*)&d_piv_offsets, &d_status, &bs,
                    &pass, &use_pattern, (void*)&pat_J, (void*)&pat_Pi, &fallback, &fo, &probe};
    ProfScope ps(stream, use_pattern ? PROF_PATTERN : PROF_BATCHED);
    LINAC_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(BT_THREADS), args, smem, stream));
    return LINAC_OK;
}

// Launch groups for buckets 0..top: consecutive buckets of one panel width
// share one launch as long as sharing keeps every one of them at its own
// blocks per SM (a larger bucket whose shared memory would cost the smaller
// ones occupancy gets a launch of its own).  Returns the number of groups; group g is
// [lo[g], hi[g]].
static int bt_groups(int top, const BtWidths& wd, int sh, int* lo, int* hi) {
    int ng = 0;
    for (int b = 0; b <= top; ++b) {
        if (ng > 0) {
            const int g = ng - 1;
            const int occ_g = bt_group_occupancy(lo[g], hi[g], wd, sh, nullptr);
            const int occ_b = bt_group_occupancy(b, b, wd, sh, nullptr);
            const int occ_m = bt_group_occupancy(lo[g], b, wd, sh, nullptr);
            if (occ_m >= 1 && occ_m == occ_g && occ_m == occ_b) {
                hi[g] = b;
                continue;
            }
        }
        lo[ng] = hi[ng] = b;
        ++ng;
    }
    (void)cudaGetLastError();
    return ng;
}

size_t bt_shared_bytes(int b, int nb) { return bt_layout(bt_bucket_max(b), nb).total; }

linac_status batched_rref(uint32_t* d_data, const int64_t* d_offsets, const int32_t* d_m,
                          const int32_t* d_n, const int32_t* d_ld, const int32_t* d_nsearch,
                          int32_t batch, int32_t max_m, int32_t max_n, const Field& f, uint32_t flags,
                          int32_t* d_ranks, int32_t* d_pivots, const int64_t* d_piv_offsets,
                          int32_t* d_status, cudaStream_t stream) {
    (void)max_n;
    const bool pattern = (flags & LINAC_SHARED_PATTERN) != 0 && batch > 1;
    // scratch: BatchScratch | order[batch] | fallback[batch] | pattern J, Pi
    const size_t pat_words = (size_t)(1024 / 16 + 1) * 64;
    const size_t bytes = align_up(sizeof(BatchScratch), 256) + align_up((size_t)batch * 4, 256) * 2 +
                         2 * pat_words * 4;
    void* buf = nullptr;
    linac_status s = scratch_get_slot(stream, 2, bytes, &buf);
    if (s != LINAC_OK) return s;
    char* p = (char*)buf;
    BatchScratch* bs = (BatchScratch*)p;
    p += align_up(sizeof(BatchScratch), 256);
    int32_t* order = (int32_t*)p;
    p += align_up((size_t)batch * 4, 256);
    int32_t* fallback = (int32_t*)p;
    p += align_up((size_t)batch * 4, 256);
    int32_t* pat_J = (int32_t*)p;
    int32_t* pat_Pi = pat_J + pat_words;

    {
        ProfScope ps(stream, PROF_BATCHED);
        batch_sort_kernel<<<1, 1024, 0, stream>>>(d_m, batch, order, bs, pattern ? 1 : 0);
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    LINAC_CUDA_TRY(cudaMemsetAsync(&bs->pattern_ok, 0, sizeof(int), stream));
    int top = 0;
    while (top + 1 < BT_NBUCKETS && max_m > bt_bucket_max(top)) ++top;
    // The probe: for batches of a few waves it runs in block 0 of the first
    // persistent launch while the other blocks reduce with the search until
    // its pattern is published; for smaller batches (which that launch would
    // take up at once) it runs first, on its own, so every later system can
    // use the pattern.
    const bool inline_probe = pattern && batch > 4 * sm_count();
    if (inline_probe) LINAC_CUDA_TRY(cudaMemsetAsync(bs->pattern_k, 0, sizeof(bs->pattern_k), stream));
    if (pattern && !inline_probe) {
        // the probe runs with the widest panel the bucket of system 0 may need
        const int nb = bt_bucket_nb(top);
        const BtLayout L = bt_layout(bt_bucket_max(top), nb);
        ProfScope ps(stream, PROF_PATTERN);
        switch (nb) {
#define LINAC_PROBE(NBV)                                                                                        \
    case NBV:                                                                                                   \
        LINAC_CUDA_TRY(cudaFuncSetAttribute(batched_probe_kernel<NBV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                            (int)L.total));                                                     \
        batched_probe_kernel<NBV><<<1, BT_THREADS, L.total, stream>>>(d_data, d_offsets, d_m, d_n, d_ld, d_nsearch, \
                                                                      bt_bucket_max(top), f, d_ranks, d_pivots,  \
                                                                      d_piv_offsets, d_status, bs, pat_J, pat_Pi,  \
                                                                      bt_fold_params(f));                          \
        break;
            LINAC_PROBE(16)
            LINAC_PROBE(32)
            LINAC_PROBE(64)
#undef LINAC_PROBE
            default: return LINAC_ERR_ARG;
        }
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    // tuned widths; every bucket uses the pattern's panel width when a
    // pattern is shared (pass 0)
    BtWidths tuned, first;
    for (int b = 0; b < BT_NBUCKETS; ++b) {
        tuned.nb[b] = bt_bucket_nb(b);
        first.nb[b] = pattern ? bt_bucket_nb(top) : tuned.nb[b];
    }
    for (int pass = 0; pass < (pattern ? 2 : 1); ++pass) {
        const BtWidths& wd = pass == 0 ? first : tuned;
        int glo[BT_NBUCKETS], ghi[BT_NBUCKETS];
        const int ng = bt_groups(top, wd, bt_fold_params(f).nshift, glo, ghi);
        for (int g = ng - 1; g >= 0; --g) {   // largest systems first
            // the first launch of the pattern pass also runs the probe (its block 0)
            const int probe = pass == 0 && inline_probe && g == ng - 1 ? 1 : 0;
            s = launch_group(glo[g], ghi[g], pass, pass == 0 && pattern ? 1 : 0, probe, wd, d_data, d_offsets, d_m, d_n,
                             d_ld, d_nsearch, order, f, d_ranks, d_pivots, d_piv_offsets, d_status, bs, pat_J,
                             pat_Pi, fallback, stream);
            if (s != LINAC_OK) return s;
        }
    }
    return LINAC_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: per size bucket, time every feasible panel width on synthetic
// systems of that bucket's sizes and keep the fastest for this device.

namespace {

// Uniform residues from a counter hash (SplitMix64 finaliser), for timing only.
__global__ void tune_fill_kernel(uint32_t* data, int64_t words, uint32_t p, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        data[i] = (uint32_t)(((z >> 32) * (uint64_t)p) >> 32);
    }
}

}  // namespace

linac_status batched_tune(const Field& f, int32_t* nb_out, cudaStream_t stream) {
    int max_smem = 0;
    max_smem = max_smem_optin();
    if (max_smem <= 0) return LINAC_ERR_CUDA;
    const int cands[3] = {16, 32, 64};
    for (int b = 0; b < BT_NBUCKETS; ++b) {
        const int hi = bt_bucket_max(b), lo = b ? bt_bucket_max(b - 1) + 1 : 8;
        // sizes spread over the bucket; enough systems to fill every SM several
        // times (throughput, not single-system latency, is what is tuned), and
        // at least a few ms of work, within a bounded footprint
        std::vector<int> ms;
        const double target = 4e9;                  // field multiply-adds per trial
        const int min_count = 6 * sm_count();
        const int64_t max_words = (int64_t)1 << 28;  // 1 GiB per copy
        int64_t work = 0, wsum = 0;
        for (int i = 0; (work < target || i < min_count) && i < 16384; ++i) {
            const int mm = lo + (int)((int64_t)(hi - lo) * ((i * 37) % 101) / 100);
            const int64_t wds = (int64_t)mm * ((mm + 4 + 3) / 4 * 4);
            if (wsum + wds > max_words) break;
            ms.push_back(mm);
            wsum += wds;
            work += (int64_t)mm * mm * mm / 2;
        }
        const int batch = (int)ms.size();
        std::vector<int64_t> off(batch), poff(batch);
        std::vector<int32_t> hm(batch), hn(batch), hld(batch), hns(batch);
        int64_t words = 0, pw = 0;
        for (int i = 0; i < batch; ++i) {
            hm[i] = ms[i];
            hns[i] = ms[i];
            hn[i] = ms[i] + 4;
            hld[i] = (hn[i] + 3) / 4 * 4;
            off[i] = words;
            words += (int64_t)hm[i] * hld[i];
            poff[i] = pw;
            pw += std::min(hm[i], hns[i]);
        }
        uint32_t *d_data = nullptr, *d_pristine = nullptr;
        int64_t *d_off = nullptr, *d_poff = nullptr;
        int32_t *d_m = nullptr, *d_n = nullptr, *d_ld = nullptr, *d_ns = nullptr, *d_ranks = nullptr, *d_piv = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        linac_status st = LINAC_OK;
        auto bail = [&](linac_status s2) { st = s2; };
        do {
            if (cudaMalloc(&d_data, words * 4) || cudaMalloc(&d_pristine, words * 4) ||
                cudaMalloc(&d_off, batch * 8) || cudaMalloc(&d_poff, batch * 8) || cudaMalloc(&d_m, batch * 4) ||
                cudaMalloc(&d_n, batch * 4) || cudaMalloc(&d_ld, batch * 4) || cudaMalloc(&d_ns, batch * 4) ||
                cudaMalloc(&d_ranks, batch * 4) || cudaMalloc(&d_piv, std::max<int64_t>(pw, 1) * 4)) {
                bail(LINAC_ERR_NOMEM);
                break;
            }
            cudaMemcpyAsync(d_off, off.data(), batch * 8, cudaMemcpyHostToDevice, stream);
            cudaMemcpyAsync(d_poff, poff.data(), batch * 8, cudaMemcpyHostToDevice, stream);
            cudaMemcpyAsync(d_m, hm.data(), batch * 4, cudaMemcpyHostToDevice, stream);
            cudaMemcpyAsync(d_n, hn.data(), batch * 4, cudaMemcpyHostToDevice, stream);
            cudaMemcpyAsync(d_ld, hld.data(), batch * 4, cudaMemcpyHostToDevice, stream);
            cudaMemcpyAsync(d_ns, hns.data(), batch * 4, cudaMemcpyHostToDevice, stream);
            tune_fill_kernel<<<1024, 256, 0, stream>>>(d_pristine, words, f.p, 0x5EEDull + b);
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            float best = 1e30f;
            int best_nb = bt_default_nb(b);
            for (int c = 0; c < 3; ++c) {
                const int nb = cands[c];
                if (bt_shared_bytes(b, nb) + 4096 > (size_t)max_smem) continue;
                bt_set_bucket_nb(b, nb);
                float t = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    cudaMemcpyAsync(d_data, d_pristine, words * 4, cudaMemcpyDeviceToDevice, stream);
                    cudaEventRecord(e0, stream);
                    linac_status s2 = batched_rref(d_data, d_off, d_m, d_n, d_ld, d_ns, batch, hi, hi + 4, f, 0,
                                                   d_ranks, d_piv, d_poff, nullptr, stream);
                    cudaEventRecord(e1, stream);
                    if (s2 != LINAC_OK) { t = 1e30f; break; }
                    cudaEventSynchronize(e1);
                    float ms_ = 0.f;
                    cudaEventElapsedTime(&ms_, e0, e1);
                    if (rep > 0) t = std::min(t, ms_);   // first run warms up
                }
                if (t < best) {
                    best = t;
                    best_nb = nb;
                }
            }
            bt_set_bucket_nb(b, best_nb);
            if (nb_out) nb_out[b] = best_nb;
            if (cudaGetLastError() != cudaSuccess) bail(LINAC_ERR_CUDA);
        } while (0);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamSynchronize(stream);
        for (void* ptr : {(void*)d_data, (void*)d_pristine, (void*)d_off, (void*)d_poff, (void*)d_m, (void*)d_n,
                          (void*)d_ld, (void*)d_ns, (void*)d_ranks, (void*)d_piv})
            if (ptr) cudaFree(ptr);
        if (st != LINAC_OK) return st;
    }
    return LINAC_OK;
}

linac_status batched_set_nb(const int32_t* nb) {
    int max_smem = 0;
    max_smem = max_smem_optin();
    if (max_smem <= 0) return LINAC_ERR_CUDA;
    for (int b = 0; b < BT_NBUCKETS; ++b) {
        const int v = nb[b];
        if (v != 0 && v != 16 && v != 32 && v != 64) return LINAC_ERR_ARG;
        if (v && bt_shared_bytes(b, v) + 4096 > (size_t)max_smem) return LINAC_ERR_UNSUPPORTED;
    }
    for (int b = 0; b < BT_NBUCKETS; ++b) bt_set_bucket_nb(b, nb[b]);
    return LINAC_OK;
}

void batched_get_nb(int32_t* nb_out) {
    for (int b = 0; b < BT_NBUCKETS; ++b) nb_out[b] = bt_bucket_nb(b);
}

}  // namespace linac
