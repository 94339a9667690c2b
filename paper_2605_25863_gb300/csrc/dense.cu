// dense.cu -- blocked right-looking Gauss-Jordan elimination of one dense
// matrix over Z/pZ on sm_103a, with every piece of state kept on the device.
//
// The paper (section 3.2) reduces one column per iteration: pivot search,
// row swap, rescale of the pivot row by the inverse of its head, and a
// rank-1 update of every other row.  Here the same elimination is blocked by
// panels of nb columns [c0, c1):
//
//   1. window_kernel  (one 8-block cluster) finds the k <= nb pivots of the
//      panel among the first nb + 16 rows not yet used, by fraction-free
//      elimination (row_i <- h * row_i - f_i * pivot_row, so no inverse is on
//      this sequential path) with one cluster barrier per column.  When the
//      window has a pivot in every column (or holds every remaining row) its
//      result is exactly that of the full search; otherwise
//      panel_kernel   (cooperative) searches every remaining row, one grid
//      arrival per column.  Either records the pivot rows Pi, the pivot
//      columns J and the pivot rows' fraction-free panel entries.
//   2. gather_*       F = M[:, J] (the multipliers of the final update, in
//      balanced signed form, stored transposed) and W = M[Pi, c0:n].
//   3. heads_inverse  batched inverses of the k pivot heads (binary extended
//      Euclid, one thread each).
//   4. einv_kernel    replays the panel's fraction-free recurrence, the
//      scaling by the heads' inverses and the back substitution on the
//      identity, giving E = G^{-1} (G = M[Pi, J]); R = E W on the update
//      kernel is the k reduced pivot rows (identity at J).
//   5. move_kernel    rows of [r, r+k) that are not pivots move to the pivot
//      rows' old places (the paper's row swap, done once per panel).
//   6. the update     every row d outside [r, r+k):  M[d, c0:n] -= F[d] * R
//      (mod p), the O(n^3) trailing update; rows r..r+k-1 receive R.  On
//      CUDA cores (update_plain), on the integer tensor pipe (update_limb,
//      update_crt), or on both at once (update_hybrid), as the path option
//      or the matrix size selects.
//   7. finish_kernel  appends J to the pivot list and advances r by k.
//
// Because R is fully reduced (identity at the pivot columns), the update
// multipliers are simply each row's entries at the pivot columns, and the
// update clears those columns in every other row, above and below: that is
// Gauss-Jordan (reduced echelon form), not LU.
#include <algorithm>
#include <climits>
#include <cstdio>

#include <cooperative_groups.h>

#include "dense_kernels.cuh"
#include "linac_host.h"
#include "profile.h"
#include "update.cuh"

namespace linac {

// ---------------------------------------------------------------------------
// Initialisation and bookkeeping

__global__ void init_kernel(DenseState* st, int32_t* d_pivots, int64_t npiv, int32_t* d_rank) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npiv;
         i += (int64_t)gridDim.x * blockDim.x)
        d_pivots[i] = -1;
    if (blockIdx.x == 0) {
        for (int t = threadIdx.x; t < NB_MAX; t += blockDim.x) st->best[t] = INT_MAX;
        if (threadIdx.x == 0) {
            st->r = 0;
            st->k = 0;
            st->win_ok = 0;
            st->bar.count = 0;
            st->bar.gen = 0;
            *d_rank = 0;
        }
    }
}

__global__ void finish_kernel(DenseState* st, int32_t* d_pivots, int32_t* d_rank) {
    const int k = st->k, r = st->r;
    __syncthreads();
    for (int t = threadIdx.x; t < k; t += blockDim.x) d_pivots[r + t] = st->J[t];
    for (int t = threadIdx.x; t < NB_MAX; t += blockDim.x) st->best[t] = INT_MAX;
    __syncthreads();
    if (threadIdx.x == 0) {
        st->r = r + k;
        st->k = 0;
        *d_rank = r + k;
    }
}

// ---------------------------------------------------------------------------
// 1. Panel factorisation (cooperative launch, one row slab per block)
//
// Shared memory: S_max x (w+1) residues (the slab, padded against bank
// conflicts), the broadcast pivot row, the owned-pivot list and pivot flags.

// Block-wide minimum of one int per thread.
__device__ __forceinline__ int panel_block_min(int v, int* red, int* out) {
    v = __reduce_min_sync(0xffffffffu, v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int x = lane < (int)(blockDim.x >> 5) ? red[lane] : INT_MAX;
        x = __reduce_min_sync(0xffffffffu, x);
        if (lane == 0) *out = x;
    }
    __syncthreads();
    return *out;
}

// Column-level look-ahead: for every column the block (1) applies the current
// pivot to the next column only and searches it, (2) lets warp 0 finish its
// candidate row, publish it and arrive at the grid barrier, and (3) while
// warp 0 waits, lets the other warps apply the current pivot to the rest of
// the panel, so the barrier latency overlaps the bulk of the elimination.
// All arithmetic is the same fraction-free step as in the plain loop:
// row_i <- h row_i - f_i pivot with f_i kept in column cc.
// Pivots of a panel from a window of its first w + WIN_EXTRA remaining rows,
// without grid-wide synchronisation.  Every column's pivot is the
// lowest-index remaining row with a nonzero entry (section 3.2: over a finite
// field any nonzero entry serves, and the RREF does not depend on the choice),
// and the window holds the lowest-index remaining rows: when it has a pivot in
// every panel column, or holds every remaining row, its pivots, their order
// and the pivot rows' fraction-free panel entries are exactly those the
// grid-wide search in panel_kernel would find.  It then writes them (k, J,
// Pi, panelU), advances panel_kernel's arrival counter by the w x G arrivals
// that kernel would have made, and sets win_ok so that panel_kernel returns
// at once; otherwise it leaves everything to panel_kernel.
//
// One cluster of WIN_CTAS blocks: block c holds window rows
// [c WIN_ROWS_CTA, (c+1) WIN_ROWS_CTA) in its shared memory (Montgomery
// form, as in panel_kernel).  Per column each block writes its lowest
// candidate row's index and its entries from the current column on into
// every block's shared memory (distributed shared memory stores), one
// cluster barrier makes them (and every block's earlier row updates)
// visible, and every block takes the minimum and eliminates its own rows
// with the winning row read locally.  A slot is reused two columns later,
// after another cluster barrier.
__global__ void __cluster_dims__(WIN_CTAS, 1, 1) __launch_bounds__(WIN_THREADS)
window_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, Field f, DenseState* st,
              uint32_t* __restrict__ panelU, int G, const int32_t* __restrict__ rowmap) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ __align__(16) uint32_t P[WIN_ROWS_CTA * (NB_MAX + 1)];
    __shared__ int posts[2][WIN_CTAS];                          // posts[par][b]: block b's candidate row
    __shared__ __align__(16) uint32_t cbuf[2][WIN_CTAS][NB_MAX];  // cbuf[par][b][j]: that row at column cc + j
    __shared__ int red[WIN_THREADS / 32];
    __shared__ unsigned char isp[WIN_ROWS_CTA];
    __shared__ int own[NB_MAX], Jc[NB_MAX];        // window row and panel column of pivot t
    constexpr int RG = WIN_THREADS / NB_MAX;        // row groups of the elimination
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = (int)cluster.block_rank();
    const int SW = w + 1;
    const int64_t r = st->r;
    const int64_t left = m - r > 0 ? m - r : 0;
    const int rows = (int)(left < w + WIN_EXTRA ? left : w + WIN_EXTRA);
    const int g0 = c * WIN_ROWS_CTA;                                   // first window row of this block
    const int lrows = max(0, min(WIN_ROWS_CTA, rows - g0));            // rows held here
    for (int e = tid; e < lrows * w; e += WIN_THREADS) {
        const int i = e / w, j = e - i * w;
        P[i * SW + j] = to_mont(M[map_row(rowmap, r, g0 + i) * ld + c0 + j], f);
    }
    for (int i = tid; i < WIN_ROWS_CTA; i += WIN_THREADS) isp[i] = 0;
    __syncthreads();
    int kk = 0, par = 0;
    const int jj = tid % NB_MAX, rg = tid / NB_MAX;
    for (int cc = 0; cc < w; ++cc) {
        // this block's lowest remaining row with a nonzero entry in column cc
        int cand = (tid < lrows && !isp[tid] && P[tid * SW + cc] != 0u) ? tid : INT_MAX;
        cand = __reduce_min_sync(0xffffffffu, cand);
        if (lane == 0) red[warp] = cand;
        __syncthreads();
        int v = INT_MAX;   // this block's lowest candidate row (local index)
#pragma unroll
        for (int x = 0; x < WIN_THREADS / 32; ++x) v = min(v, red[x]);
        // push the post and the candidate row's entries from column cc on into
        // every block of the cluster, so that after the barrier the pivot row
        // is read from local shared memory; the slots alternate by column
        // parity, and a slot is rewritten two columns later, after the next
        // barrier, when every block has finished reading it
        const int nrem = w - cc;
        if (tid < WIN_CTAS) *cluster.map_shared_rank(&posts[par][c], tid) = v == INT_MAX ? INT_MAX : g0 + v;
        if (v != INT_MAX) {
            for (int e = tid; e < WIN_CTAS * nrem; e += WIN_THREADS) {
                const int b = e % WIN_CTAS, j = e / WIN_CTAS;
                cluster.map_shared_rank(&cbuf[par][c][0], b)[j] = P[v * SW + cc + j];
            }
        }
        cluster.sync();   // posts, pushed rows and every block's row updates of column cc - 1 are visible
        int q = INT_MAX;
#pragma unroll
        for (int b = 0; b < WIN_CTAS; ++b) q = min(q, posts[par][b]);
        const int pc = par;
        par ^= 1;
        if (q == INT_MAX) continue;   // no pivot in this column (the same in every block)
        const int owner = q / WIN_ROWS_CTA, ql = q - owner * WIN_ROWS_CTA;
        const uint32_t* prow = &cbuf[pc][owner][0];   // prow[j - cc] = pivot row at column j >= cc
        const uint32_t h = prow[0];
        if (owner == c && tid == 0) isp[ql] = 1;
        if (tid == 0) {
            own[kk] = q;
            Jc[kk] = cc;
        }
        ++kk;
        // fraction-free elimination of column cc from this block's other
        // remaining rows: row_i <- h row_i - f_i row_q on the columns right of cc
        const int nc = w - cc - 1;
        if (jj < nc) {
            constexpr int U = (WIN_ROWS_CTA + RG - 1) / RG;
            const int j = cc + 1 + jj;
            const uint32_t pv = prow[j - cc];
            uint32_t fi[U], x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = rg + u * RG;
                const bool ok = i < lrows && g0 + i != q && !isp[i];
                fi[u] = ok ? P[i * SW + cc] : 0u;
                x[u] = ok ? P[i * SW + j] : 0u;
            }
            // every product computed, stored where f_i != 0: the rows'
            // chains interleave
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t xn = mont_mul2add(h, x[u], f.p - fi[u], pv, f);
                if (fi[u] != 0u) P[(rg + u * RG) * SW + j] = xn;
            }
        }
        __syncthreads();
    }
    if (kk == w || rows == left) {
        for (int t = tid; t < kk; t += WIN_THREADS) {
            const int q = own[t];
            if (q / WIN_ROWS_CTA != c) continue;
            st->Pi[t] = (int32_t)map_row(rowmap, r, q);
        }
        for (int e = tid; e < kk * w; e += WIN_THREADS) {
            const int t = e / w, j = e - t * w;
            const int q = own[t];
            if (q / WIN_ROWS_CTA != c) continue;
            panelU[(size_t)t * NB_MAX + j] = mont_redc(P[(q - g0) * SW + j], f);
        }
        if (c == 0) {
            for (int t = tid; t < kk; t += WIN_THREADS) st->J[t] = c0 + Jc[t];
            if (tid == 0) {
                st->k = kk;
                st->win_ok = 1;
                atomicAdd(&st->bar.count, (unsigned)w * (unsigned)G);
            }
        }
    } else if (c == 0 && tid == 0) {
        st->win_ok = 0;
    }
    cluster.sync();   // no block leaves while others may still read its shared memory
}

// The same pivot window on one block, for panels of at most WIN1_NB columns
// (small matrices): the window's w + WIN_EXTRA rows fit one block's shared
// memory, and a block barrier per column costs far less than the cluster
// barrier.  Per column one block-wide minimum (two alternating slots, one
// barrier) finds the pivot, and the pass that eliminates the column also
// looks for the next column's lowest candidate.  Outputs as window_kernel.
__global__ void __launch_bounds__(WIN1_THREADS)
window1_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, Field f, DenseState* st,
               uint32_t* __restrict__ panelU, int G, const int32_t* __restrict__ rowmap) {
    constexpr int ROWS = WIN1_NB + WIN_EXTRA, SW = WIN1_NB + 1;
    // thread layout of the elimination: column slot js (column cc + 1 + js)
    // by row group rg (rows rg, rg + RG1, ...): no division per element
    constexpr int RG1 = WIN1_THREADS / WIN1_NB;
    constexpr int U1 = (ROWS + RG1 - 1) / RG1;
    static_assert(WIN1_THREADS % WIN1_NB == 0 && U1 <= 32, "window layout");
    __shared__ __align__(16) uint32_t P[U1 * RG1 * SW];
    __shared__ int red[2][WIN1_THREADS / 32];
    __shared__ int own[WIN1_NB], Jc[WIN1_NB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int js = tid % WIN1_NB, rg = tid / WIN1_NB;
    const int64_t r = st->r;
    const int64_t left = m - r > 0 ? m - r : 0;
    const int rows = (int)(left < w + WIN_EXTRA ? left : w + WIN_EXTRA);
    int buf = 0;
    auto block_min = [&](int v) -> int {   // one barrier; slots alternate so a slot is rewritten after another barrier
        v = __reduce_min_sync(0xffffffffu, v);
        if (lane == 0) red[buf][warp] = v;
        __syncthreads();
        int x = INT_MAX;
#pragma unroll
        for (int i = 0; i < WIN1_THREADS / 32; ++i) x = min(x, red[buf][i]);
        buf ^= 1;
        return x;
    };
    // load in Montgomery form; rows beyond the window hold zeros (they are
    // never updated, because their entries f are zero, and never offer a
    // candidate)
    int cand = INT_MAX;
    for (int e = tid; e < U1 * RG1 * w; e += WIN1_THREADS) {
        const int i = e / w, j = e - i * w;
        const uint32_t v = i < rows ? M[map_row(rowmap, r, i) * ld + c0 + j] : 0u;
        P[i * SW + j] = to_mont(v, f);
        if (j == 0 && v != 0u && i < cand) cand = i;
    }
    int q = block_min(cand);   // also the barrier after the load
    int kk = 0;
    uint32_t pmask = 0u;       // bit u: row rg + u RG1 is a pivot row
    for (int cc = 0; cc < w; ++cc) {
        if (q != INT_MAX) {
            if (tid == 0) {
                own[kk] = q;
                Jc[kk] = cc;
            }
            if (q % RG1 == rg) pmask |= 1u << (q / RG1);
            ++kk;
        }
        // fraction-free elimination of column cc from the other remaining
        // rows (row_i <- h row_i - f_i row_q on the columns right of cc, for
        // the rows with f_i != 0, the recurrence einv_kernel replays), and
        // the next column's candidate from the updated entries.  The products
        // are computed for every row and kept by a select, so the rows'
        // dependent chains interleave; only the stores are conditional.
        const int nc = w - cc - 1;
        cand = INT_MAX;
        if (nc > 0) {
            if (js < nc) {
                const int j = cc + 1 + js;
                const bool has = q != INT_MAX;
                const uint32_t h = has ? P[q * SW + cc] : 0u;
                const uint32_t pv = has ? P[q * SW + j] : 0u;
                uint32_t x[U1], fi[U1];
#pragma unroll
                for (int u = 0; u < U1; ++u) {
                    const int i = rg + u * RG1;
                    x[u] = P[i * SW + j];
                    fi[u] = P[i * SW + cc];
                }
#pragma unroll
                for (int u = 0; u < U1; ++u) {
                    const uint32_t xn = mont_mul2add(h, x[u], f.p - fi[u], pv, f);
                    const bool upd = has && fi[u] != 0u && !((pmask >> u) & 1u);
                    if (upd) P[(rg + u * RG1) * SW + j] = xn;
                    x[u] = upd ? xn : x[u];
                }
                if (js == 0) {
                    uint32_t nz = 0u;
#pragma unroll
                    for (int u = 0; u < U1; ++u) nz |= x[u] != 0u ? (1u << u) : 0u;
                    nz &= ~pmask;
                    if (nz != 0u) cand = rg + (__ffs((int)nz) - 1) * RG1;
                }
            }
            q = block_min(cand);
        }
    }
    __syncthreads();   // the last column's pivot record is visible to every thread
    if (kk == w || rows == left) {
        for (int t = tid; t < kk; t += WIN1_THREADS) {
            st->Pi[t] = (int32_t)map_row(rowmap, r, own[t]);
            st->J[t] = c0 + Jc[t];
        }
        for (int e = tid; e < kk * w; e += WIN1_THREADS) {
            const int t = e / w, j = e - t * w;
            panelU[(size_t)t * NB_MAX + j] = mont_redc(P[own[t] * SW + j], f);
        }
        if (tid == 0) {
            st->k = kk;
            st->win_ok = 1;
            atomicAdd(&st->bar.count, (unsigned)w * (unsigned)G);
        }
    } else if (tid == 0) {
        st->win_ok = 0;
    }
}

__global__ void __launch_bounds__(PANEL_THREADS)
panel_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, int S_max,
             Field f, DenseState* st, uint32_t* cand, uint32_t* panelU, int* status, WaitLimit wl,
             const int32_t* __restrict__ rowmap) {
    extern __shared__ __align__(16) uint32_t sm[];
    const int SW = w + 1;
    uint32_t* P = sm;
    uint32_t* prow = P + (size_t)S_max * SW;
    int* own = (int*)(prow + NB_MAX);
    unsigned char* isp = (unsigned char*)(own + NB_MAX);
    __shared__ int s_red[PANEL_THREADS / 32];
    __shared__ int s_min, s_q, s_ok;

    if (st->win_ok) return;   // window_kernel found this panel's pivots (and advanced the barrier)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    int* cidx = (int*)(cand + (size_t)2 * G * NB_MAX);   // [2][G] candidate row per block
    const int64_t r = st->r;
    const int64_t left = m - r;
    const int S = left > 0 ? (int)((left + G - 1) / G) : 0;
    const int64_t lo = (int64_t)b * S;   // first position of this block's slab
    int nrows = 0;
    if (S > 0 && lo < left) nrows = (int)min((int64_t)S, left - lo);

    // the slab, the published candidate rows and prow hold Montgomery forms
    // x R mod p (R = 2^32): each fraction-free update is two products and one
    // Montgomery reduction, and the pivot rows go back to plain residues when
    // they are written to panelU
    for (int64_t e = tid; e < (int64_t)nrows * w; e += blockDim.x) {
        const int i = (int)(e / w), j = (int)(e % w);
        P[i * SW + j] = to_mont(M[map_row(rowmap, r, lo + i) * ld + c0 + j], f);
    }
    for (int i = tid; i < nrows; i += blockDim.x) isp[i] = 0;
    for (int t = tid; t < NB_MAX; t += blockDim.x) own[t] = -1;
    if (tid == 0) s_ok = 1;
    __syncthreads();

    // Publish this block's candidate (row imin, already fully updated) for
    // column c0 + col and wait for every block.  Warp 0 only.
    auto publish_and_wait = [&](int col, int imin) {
        const int par = col & 1;
        if (imin != INT_MAX) {
            uint32_t* dst = cand + ((size_t)par * G + b) * NB_MAX;
            for (int j = lane; j < w; j += 32) dst[j] = P[imin * SW + j];
        }
        if (lane == 0) cidx[par * G + b] = imin != INT_MAX ? (int)(lo + imin) : INT_MAX;
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            unsigned int* counter = &st->bar.count;
            const unsigned int target = (unsigned)(c0 + col + 1) * (unsigned)G + wl.extra_arrivals;
            asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
            const long long t0 = clock64();
            for (unsigned int it = 0;; ++it) {
                unsigned int v;
                asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
                if ((int)(v - target) >= 0) break;
                if ((it & 255u) == 255u) {
                    if (*(volatile int*)status != 0) { s_ok = 0; break; }
                    if (clock64() - t0 > wl.spin_cycles) {
                        atomicCAS(status, 0, (int)LINAC_ERR_TIMEOUT);
                        s_ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        __syncwarp();
    };
    // After a __syncthreads that follows publish_and_wait: the pivot of
    // column c0 + col (lowest candidate over all blocks), its row in prow.
    int kk = 0;
    auto take_winner = [&](int col) -> int {
        const int par = col & 1;
        if (warp == 0) {
            int v = INT_MAX;
            for (int g = lane; g < G; g += 32) v = min(v, __ldcg(&cidx[par * G + g]));
            v = __reduce_min_sync(0xffffffffu, v);
            if (lane == 0) s_q = v;
        }
        __syncthreads();
        const int q = s_q;
        if (q != INT_MAX) {
            const int owner = q / S;
            const uint32_t* src = cand + ((size_t)par * G + owner) * NB_MAX;
            for (int j = tid; j < w; j += blockDim.x) prow[j] = __ldcg(src + j);
            if (tid == 0) {
                if (b == owner) { isp[q - lo] = 1; own[kk] = (int)(q - lo); }
                if (b == 0) { st->Pi[kk] = (int32_t)map_row(rowmap, r, q); st->J[kk] = c0 + col; }
            }
            ++kk;
            __syncthreads();
        }
        return q;
    };

    // column 0: search, publish, take the pivot
    int ci = INT_MAX;
    for (int i = tid; i < nrows; i += blockDim.x)
        if (P[i * SW] != 0) { ci = i; break; }
    int imin = panel_block_min(ci, s_red, &s_min);
    if (warp == 0) publish_and_wait(0, imin);
    __syncthreads();
    if (!s_ok) return;
    int q = take_winner(0);

    for (int cc = 0; cc + 1 < w; ++cc) {
        const uint32_t h = q != INT_MAX ? prow[cc] : 0u;
        // narrow update: column cc+1 only, with the search for its candidate
        ci = INT_MAX;
        for (int i = tid; i < nrows; i += blockDim.x) {
            if (isp[i]) continue;
            uint32_t* row = P + i * SW;
            if (q != INT_MAX) {
                const uint32_t fi = row[cc];
                if (fi != 0) row[cc + 1] = mont_mul2add(h, row[cc + 1], f.p - fi, prow[cc + 1], f);
            }
            if (row[cc + 1] != 0 && i < ci) ci = i;
        }
        imin = panel_block_min(ci, s_red, &s_min);
        if (warp == 0) {
            // finish the candidate row, publish it and wait at the barrier
            if (imin != INT_MAX && q != INT_MAX) {
                uint32_t* row = P + imin * SW;
                const uint32_t fi = row[cc];
                if (fi != 0)
                    for (int j = cc + 2 + lane; j < w; j += 32) row[j] = mont_mul2add(h, row[j], f.p - fi, prow[j], f);
                __syncwarp();
            }
            publish_and_wait(cc + 1, imin);
        } else if (q != INT_MAX) {
            // bulk update of the other rows while warp 0 waits
            for (int i = warp - 1; i < nrows; i += nwarps - 1) {
                if (isp[i] || i == imin) continue;
                uint32_t* row = P + i * SW;
                const uint32_t fi = row[cc];
                if (fi == 0) continue;
                const uint32_t nf = f.p - fi;
                for (int j = cc + 2 + lane; j < w; j += 32) row[j] = mont_mul2add(h, row[j], nf, prow[j], f);
            }
        }
        __syncthreads();
        if (!s_ok) return;
        q = take_winner(cc + 1);
    }
    for (int t = 0; t < kk; ++t) {
        const int i = own[t];
        if (i < 0) continue;
        for (int j = tid; j < w; j += blockDim.x) panelU[(size_t)t * NB_MAX + j] = mont_redc(P[i * SW + j], f);
    }
    if (b == 0 && tid == 0) st->k = kk;
}

// ---------------------------------------------------------------------------
// 2. Gathers

// Ft[t][i] = balanced(M[i][J_t]) for every row i, zero for t in [k, kpad).
// A block stages 64 rows' panel segments in shared memory, then writes the
// transposed multipliers with coalesced stores.
__global__ void __launch_bounds__(256)
gather_f_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, Field f,
                const DenseState* __restrict__ st, int32_t* __restrict__ Ft, int64_t ldF,
                const int32_t* __restrict__ rowmap) {
    __shared__ uint32_t seg[64][NB_MAX + 1];
    __shared__ int Jl[NB_MAX];
    const int k = st->k;
    if (k == 0) return;
    const int kpad = (k + UPD_BK - 1) / UPD_BK * UPD_BK;
    const int64_t row0 = (int64_t)blockIdx.x * 64;
    // with a row map, the rows are those left after this panel's pivots
    if (rowmap) m = min(m, (int64_t)(m - st->r - k));
    if (row0 >= m) return;
    for (int t = threadIdx.x; t < k; t += blockDim.x) Jl[t] = st->J[t] - c0;
    for (int e = threadIdx.x; e < 64 * w; e += blockDim.x) {
        const int i = e / w, j = e % w;
        const int64_t row = row0 + i;
        seg[i][j] = row < m ? M[map_row(rowmap, 0, row) * ld + c0 + j] : 0u;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kpad * 64; e += blockDim.x) {
        const int t = e >> 6, i = e & 63;
        const int64_t row = row0 + i;
        if (row < m) Ft[(int64_t)t * ldF + row] = t < k ? to_balanced(seg[i][Jl[t]], f) : 0;
    }
}

// W[t][j] = balanced(M[Pi_t][c0 + j]) for t < k, zero for t in [k, kpad); j < n - c0.
__global__ void gather_w_kernel(const uint32_t* __restrict__ M, int64_t ld, int64_t ncols, int c0, Field f,
                                const DenseState* __restrict__ st, int32_t* __restrict__ W, int64_t ldW) {
    const int t = blockIdx.y;
    const int k = st->k;
    const int kpad = (k + UPD_BK - 1) / UPD_BK * UPD_BK;
    if (t >= kpad) return;
    int32_t* dst = W + (int64_t)t * ldW;
    if (t >= k) {
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ncols;
             j += (int64_t)gridDim.x * blockDim.x)
            dst[j] = 0;
        return;
    }
    const uint32_t* src = M + (int64_t)st->Pi[t] * ld + c0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ncols;
         j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = to_balanced(src[j], f);
}

// ---------------------------------------------------------------------------
// 3. Batched inverses of the pivot heads h_t = panelU[t][J_t - c0].

__global__ void heads_inverse_kernel(DenseState* st, const uint32_t* __restrict__ panelU, int c0,
                                     uint32_t p, int* status) {
    const int k = st->k;
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        const uint32_t h = panelU[(size_t)t * NB_MAX + (st->J[t] - c0)];
        if (h == 0) atomicCAS(status, 0, (int)LINAC_ERR_RANGE);   // cannot happen for p prime
        st->hinv[t] = inverse_mod(h, p);
    }
}

// ---------------------------------------------------------------------------
// 4. TRSM-style reduction of the pivot rows.  The panel left the pivot rows
// related to the original rows W = M[Pi, c0:n] by a fixed k x k transform:
// forward, for s = 0..k-2 and every t > s whose multiplier f_ts = panelU[t][J_s]
// is nonzero, V_t <- h_s V_t - f_ts V_s (the panel's own fraction-free
// recurrence); scaling V_t <- V_t / h_t; backward, for s = k-1..1 and t < s,
// V_t <- V_t - c_ts V_s with c_ts = panelU[t][J_s] / h_t (V_t's entry at J_s
// after the forward pass and the scaling).  The composite is E = G^{-1}, with
// G = M[Pi, J].  Columns of E are independent (column j is the transform of
// the unit vector e_j), so each block builds EINV_COLS columns; E is stored
// transposed and balanced, and the reduced pivot rows are R = E W, a small
// product on the same lazy-accumulation kernel as the trailing update.
__global__ void __launch_bounds__(256)
einv_kernel(const DenseState* __restrict__ st, const uint32_t* __restrict__ panelU, int c0, Field f,
            int32_t* __restrict__ Et) {
    extern __shared__ __align__(16) uint32_t sm[];
    constexpr int S = NB_MAX + 1;
    constexpr int C = EINV_COLS;
    uint32_t* Co = sm;                 // Co[t][s]: f_ts (s < t) or c_ts (s > t)
    uint32_t* Ec = sm + NB_MAX * S;    // Ec[t][c] = E[t][j0 + c]
    __shared__ uint32_t hs[NB_MAX], hinv[NB_MAX];
    __shared__ int Jl[NB_MAX];
    const int k = st->k;
    if (k == 0) return;
    const int kpad = (k + UPD_BK - 1) / UPD_BK * UPD_BK;
    const int j0 = blockIdx.x * C;
    if (j0 >= kpad) return;
    const int tid = threadIdx.x;
    if (j0 >= k) {   // padding rows of Et
        for (int e = tid; e < C * NB_MAX; e += blockDim.x) Et[(size_t)(j0 + e / NB_MAX) * NB_MAX + e % NB_MAX] = 0;
        return;
    }
    for (int t = tid; t < k; t += blockDim.x) {
        Jl[t] = st->J[t] - c0;
        hinv[t] = st->hinv[t];
    }
    __syncthreads();
    // the recurrence runs on Montgomery forms x R mod p (R = 2^32): each step
    // is two products and one Montgomery reduction; E leaves in plain form
    for (int t = tid; t < k; t += blockDim.x) hs[t] = to_mont(panelU[(size_t)t * NB_MAX + Jl[t]], f);
    for (int e = tid; e < k * k; e += blockDim.x) {
        const int t = e / k, s = e % k;
        const uint32_t v = panelU[(size_t)t * NB_MAX + Jl[s]];
        Co[t * S + s] = to_mont(s > t ? mulmod(v, hinv[t], f) : v, f);
    }
    for (int e = tid; e < k * C; e += blockDim.x) {
        const int t = e / C, c = e % C;
        Ec[t * C + c] = (t == j0 + c) ? f.c32 : 0u;   // the held form of 1 is R mod p
    }
    __syncthreads();
    for (int t = tid; t < k; t += blockDim.x) hinv[t] = to_mont(hinv[t], f);
    __syncthreads();
    // Each step updates rows of the block's C columns; thread tid owns column
    // c = tid % C and the rows RGE apart from its row group tg = tid / C, a
    // fixed layout with no division per element.  Every product is computed
    // and the store is skipped where the coefficient is zero, as the
    // recurrence prescribes, so a thread's rows are independent chains.
    constexpr int RGE = 256 / C;                      // row groups
    constexpr int UE = (NB_MAX + RGE - 1) / RGE;      // rows per thread and step
    static_assert(256 % C == 0, "einv layout");
    const int cc = tid % C, tg = tid / C;
    // forward (all stages: row j itself is rescaled by h_s at every earlier
    // stage s whose multiplier f_js is nonzero, so E[j][j] changes before s = j)
    for (int s = 0; s + 1 < k; ++s) {
        const uint32_t h = hs[s];
        const uint32_t es = Ec[s * C + cc];
        uint32_t x[UE], ft[UE];
#pragma unroll
        for (int u = 0; u < UE; ++u) {
            const int t = s + 1 + tg + u * RGE;
            ft[u] = t < k ? Co[t * S + s] : 0u;
            x[u] = t < k ? Ec[t * C + cc] : 0u;
        }
#pragma unroll
        for (int u = 0; u < UE; ++u) {
            const uint32_t xn = mont_mul2add(h, x[u], f.p - ft[u], es, f);
            if (ft[u] != 0u) Ec[(s + 1 + tg + u * RGE) * C + cc] = xn;
        }
        __syncthreads();
    }
    for (int e = tid; e < k * C; e += blockDim.x) Ec[e] = mont_mul(Ec[e], hinv[e / C], f);
    __syncthreads();
    for (int s = k - 1; s >= 1; --s) {
        const uint32_t es = Ec[s * C + cc];
        uint32_t x[UE], ct[UE];
#pragma unroll
        for (int u = 0; u < UE; ++u) {
            const int t = tg + u * RGE;
            ct[u] = t < s ? Co[t * S + s] : 0u;
            x[u] = t < s ? Ec[t * C + cc] : 0u;
        }
#pragma unroll
        for (int u = 0; u < UE; ++u) {
            const uint32_t xn = submod(x[u], mont_mul(ct[u], es, f), f);
            if (ct[u] != 0u) Ec[(tg + u * RGE) * C + cc] = xn;
        }
        __syncthreads();
    }
    // Et[j][t] = balanced E[t][j] for the block's columns j; zero for t >= k
    for (int e = tid; e < C * NB_MAX; e += blockDim.x) {
        const int c = e / NB_MAX, t = e % NB_MAX;
        const int j = j0 + c;
        Et[(size_t)j * NB_MAX + t] = (j < k && t < k) ? to_balanced(mont_redc(Ec[t * C + c], f), f) : 0;
    }
}

// ---------------------------------------------------------------------------
// 5. Row moves: positions of [r, r+k) that do not hold a pivot row send their
// row (and multipliers) to the pivot rows' old positions outside [r, r+k).
// Block a handles pair a; every block derives the same pairing.

__global__ void __launch_bounds__(256)
move_kernel(uint32_t* __restrict__ M, int64_t ld, int64_t n, int c0, const DenseState* __restrict__ st,
            int32_t* __restrict__ Ft, int64_t ldF) {
    __shared__ int srcs[NB_MAX], dsts[NB_MAX];
    __shared__ unsigned char occ[NB_MAX];
    __shared__ int npairs;
    const int k = st->k;
    if (k == 0) return;
    const int r = st->r;
    if (threadIdx.x == 0) {
        for (int d = 0; d < k; ++d) occ[d] = 0;
        for (int t = 0; t < k; ++t) {
            const int q = st->Pi[t];
            if (q >= r && q < r + k) occ[q - r] = 1;
        }
        int a = 0;
        for (int d = 0; d < k; ++d)
            if (!occ[d]) srcs[a++] = r + d;
        int bcount = 0;
        for (int t = 0; t < k; ++t) {
            const int q = st->Pi[t];
            if (q < r || q >= r + k) dsts[bcount++] = q;
        }
        npairs = a;   // equals bcount: |D \ S| = |S \ D|
    }
    __syncthreads();
    const int a = blockIdx.x;
    if (a >= npairs) return;
    const int64_t src = srcs[a], dst = dsts[a];
    for (int64_t j = c0 + threadIdx.x; j < n; j += blockDim.x) M[dst * ld + j] = M[src * ld + j];
    const int kpad = (k + UPD_BK - 1) / UPD_BK * UPD_BK;
    for (int t = threadIdx.x; t < kpad; t += blockDim.x)
        Ft[(int64_t)t * ldF + dst] = Ft[(int64_t)t * ldF + src];
}

// ---------------------------------------------------------------------------
// Solve helpers and validation

__global__ void pack_kernel(const uint32_t* __restrict__ A, int64_t m, int64_t nA, int64_t ldA,
                            const uint32_t* __restrict__ B, int64_t k, int64_t ldB,
                            uint32_t* __restrict__ Mx, int64_t ldM) {
    const int64_t ncols = nA + k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * ldM;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ldM, j = e % ldM;
        uint32_t v = 0;
        if (j < nA) v = A[i * ldA + j];
        else if (j < ncols) v = B[i * ldB + (j - nA)];
        Mx[e] = v;
    }
}

// One block per right-hand side j: consistent iff the reduced column vanishes
// at and below the rank (section 5.2); X column from the pivot rows, free
// variables zero.
__global__ void __launch_bounds__(256)
extract_kernel(const uint32_t* __restrict__ Mx, int64_t m, int64_t nA, int64_t ldM,
               const int32_t* __restrict__ d_rank, const int32_t* __restrict__ d_pivots,
               uint32_t* __restrict__ X, int64_t ldX, uint8_t* __restrict__ cons) {
    __shared__ int s_bad;
    const int64_t j = blockIdx.x;
    const int rank = *d_rank;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    int bad = 0;
    for (int64_t i = rank + threadIdx.x; i < m; i += blockDim.x)
        if (Mx[i * ldM + nA + j] != 0) bad = 1;
    if (bad) atomicOr(&s_bad, 1);
    __syncthreads();
    const int ok = !s_bad;
    if (threadIdx.x == 0) cons[j] = (uint8_t)ok;
    for (int64_t i = threadIdx.x; i < nA; i += blockDim.x) X[i * ldX + j] = 0;
    __syncthreads();
    if (!ok) return;
    for (int t = threadIdx.x; t < rank; t += blockDim.x)
        X[(int64_t)d_pivots[t] * ldX + j] = Mx[(int64_t)t * ldM + nA + j];
}

__global__ void validate_kernel(const uint32_t* __restrict__ A, int64_t m, int64_t n, int64_t ld,
                                uint32_t p, int* status) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e % n;
        if (A[i * ld + j] >= p) { atomicCAS(status, 0, (int)LINAC_ERR_RANGE); return; }
    }
}

// ---------------------------------------------------------------------------
// Host driver

namespace {

struct DenseLayout {
    size_t off_state, off_cand, off_panel, off_e, off_ft, off_w, off_r, total;
    int64_t ldF, ldW;
};

DenseLayout dense_layout(int64_t m, int64_t n, int G) {
    DenseLayout L;
    size_t o = 0;
    L.off_state = o; o = align_up(o + sizeof(DenseState), 256);
    L.off_cand = o;  o = align_up(o + (size_t)2 * G * (NB_MAX + 1) * 4, 256);
    L.off_panel = o; o = align_up(o + (size_t)NB_MAX * NB_MAX * 4, 256);
    L.off_e = o;     o = align_up(o + (size_t)NB_MAX * NB_MAX * 4, 256);
    L.ldF = (int64_t)align_up((size_t)std::max<int64_t>(m, 1), 4);
    L.off_ft = o;    o = align_up(o + (size_t)NB_MAX * L.ldF * 4, 256);
    L.ldW = (int64_t)align_up((size_t)std::max<int64_t>(n, 1), 4);
    L.off_w = o;     o = align_up(o + (size_t)NB_MAX * L.ldW * 4, 256);
    L.off_r = o;     o = align_up(o + (size_t)NB_MAX * L.ldW * 4, 256);
    L.total = o;
    return L;
}

}  // namespace

int panel_grid(int64_t m) {
    const int nsm = sm_count();
    int64_t g = (m + 127) / 128;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, nsm));
}

size_t panel_smem(int S_max, int w) {
    return (size_t)S_max * (w + 1) * 4 + NB_MAX * 4 + NB_MAX * 4 + (size_t)S_max + 16;
}

int dense_default_nb(int64_t m, int64_t n) {
    (void)n;
    return m >= 2048 ? 128 : 64;
}

size_t dense_workspace_bytes(int64_t m, int64_t n, int nb) {
    (void)nb;
    return dense_layout(m, n, panel_grid(m)).total;
}

linac_status dense_rref(uint32_t* dA, int64_t m, int64_t n, int64_t ld, const Field& f,
                        int64_t nsearch, int32_t* d_rank, int32_t* d_pivots, int path, int nb,
                        cudaStream_t stream) {
    int* status = status_word(stream);
    if (!status) return LINAC_ERR_NOMEM;
    const int64_t npiv = std::min(m, nsearch);
    if (nb <= 0) nb = dense_default_nb(m, n);
    if (nb % UPD_BK != 0 || nb > NB_MAX) return LINAC_ERR_ARG;

    const int G = panel_grid(m);
    const int S_max = (int)((m + G - 1) / G);
    size_t psmem = panel_smem(S_max, nb);
    int max_smem = 0;
    max_smem = max_smem_optin();
    if (max_smem <= 0) return LINAC_ERR_CUDA;
    while (psmem > (size_t)max_smem - 1024 && nb > UPD_BK) {   // very tall matrices: narrower panels
        nb -= UPD_BK;
        psmem = panel_smem(S_max, nb);
    }
    if (psmem > (size_t)max_smem - 1024) return LINAC_ERR_UNSUPPORTED;
    if ((m + UPD_BM - 1) / UPD_BM > 65535) return LINAC_ERR_UNSUPPORTED;

    DenseLayout L = dense_layout(m, n, G);
    void* base = nullptr;
    linac_status st_ = scratch_get(stream, L.total, &base);
    if (st_ != LINAC_OK) return st_;
    char* ws = (char*)base;
    DenseState* st = (DenseState*)(ws + L.off_state);
    uint32_t* cand = (uint32_t*)(ws + L.off_cand);
    uint32_t* panelU = (uint32_t*)(ws + L.off_panel);
    int32_t* Ft = (int32_t*)(ws + L.off_ft);
    int32_t* Et = (int32_t*)(ws + L.off_e);
    int32_t* W = (int32_t*)(ws + L.off_w);
    int32_t* R = (int32_t*)(ws + L.off_r);

    if ((st_ = ensure_dynamic_smem((const void*)panel_kernel, (int)psmem)) != LINAC_OK) return st_;
    if ((st_ = ensure_dynamic_smem((const void*)einv_kernel, (int)EINV_SMEM)) != LINAC_OK) return st_;
    int occ = 0;
    LINAC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, panel_kernel, PANEL_THREADS, psmem));
    if (occ < 1 || G > occ * sm_count()) return LINAC_ERR_UNSUPPORTED;

    LimbScratch limb{};
    bool limb_ok = false;
    if (path == LINAC_PATH_LIMB) {
        limb.m_pad = (int64_t)align_up((size_t)std::max<int64_t>(m, 1), UPD_BM);
        limb.n_pad = (int64_t)align_up((size_t)std::max<int64_t>(n, 1), UPD_BN);
        const size_t fbytes = (size_t)4 * limb.m_pad * NB_MAX, rbytes = (size_t)4 * limb.n_pad * NB_MAX;
        void* lb = nullptr;
        st_ = scratch_get_slot(stream, 3, fbytes + rbytes, &lb);
        if (st_ != LINAC_OK) return st_;
        limb.Fl = (uint8_t*)lb;
        limb.Rl = (uint8_t*)lb + fbytes;
        limb_ok = true;
    }
    CrtScratch crt{};
    bool crt_ok = false;
    if (path == LINAC_PATH_CRT || path == LINAC_PATH_HYBRID) {
        void* cb = nullptr;
        st_ = scratch_get_slot(stream, 8, crt_scratch_bytes(m, n), &cb);
        if (st_ != LINAC_OK) return st_;
        crt_scratch_layout(cb, m, n, &crt);
        crt_ok = true;
    }
    {
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((npiv + 255) / 256, 1024));
        ProfScope ps(stream, PROF_INIT);
        init_kernel<<<(unsigned)blocks, 256, 0, stream>>>(st, d_pivots, npiv, d_rank);
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    if (m == 0 || n == 0) return LINAC_OK;

    for (int64_t c0 = 0; c0 < nsearch; c0 += nb) {
        const int w = (int)std::min<int64_t>(nb, nsearch - c0);
        const int64_t ncols = n - c0;
        {
            ProfScope ps(stream, PROF_PANEL);
            launch_window(dA, m, ld, (int)c0, w, f, st, panelU, G, nullptr, stream);
        }
        {
            const uint32_t* Mc = dA;
            int64_t m_ = m, ld_ = ld;
            int c0_ = (int)c0, w_ = w, S_ = S_max;
            Field f_ = f;
            WaitLimit wl = wait_limit();
            const int32_t* rowmap = nullptr;
            void* args[] = {(void*)&Mc, &m_, &ld_, &c0_, &w_, &S_, &f_, &st, &cand, &panelU, &status, &wl, &rowmap};
            ProfScope ps(stream, PROF_PANEL);
            LINAC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)panel_kernel, dim3(G), dim3(PANEL_THREADS),
                                                       args, psmem, stream));
        }
        {
            ProfScope ps(stream, PROF_GATHER_F);
            gather_f_kernel<<<(unsigned)((m + 63) / 64), 256, 0, stream>>>(dA, m, ld, (int)c0, w, f, st, Ft, L.ldF,
                                                                           nullptr);
        }
        {
            const unsigned gx = (unsigned)std::min<int64_t>((ncols + 1023) / 1024, 64);
            ProfScope ps(stream, PROF_GATHER_W);
            gather_w_kernel<<<dim3(std::max(1u, gx), NB_MAX), 256, 0, stream>>>(dA, ld, ncols, (int)c0, f, st, W,
                                                                                 L.ldW);
        }
        {
            ProfScope ps(stream, PROF_INVERSE);
            heads_inverse_kernel<<<1, NB_MAX, 0, stream>>>(st, panelU, (int)c0, f.p, status);
        }
        {
            ProfScope ps(stream, PROF_TRSM);
            einv_kernel<<<NB_MAX / EINV_COLS, 256, EINV_SMEM, stream>>>(st, panelU, (int)c0, f, Et);
        }
        {
            linac_status gs = launch_gemm_assign(f, st, Et, NB_MAX, W, L.ldW, ncols, R, L.ldW, stream);
            if (gs != LINAC_OK) return gs;
        }
        {
            ProfScope ps(stream, PROF_MOVE);
            move_kernel<<<NB_MAX, 256, 0, stream>>>(dA, ld, n, (int)c0, st, Ft, L.ldF);
        }
        linac_status us = launch_update(path, dA, m, n, ld, (int)c0, f, st, Ft, L.ldF, R, L.ldW,
                                       limb_ok ? &limb : nullptr, crt_ok ? &crt : nullptr, status, &st->next_area,
                                       stream);
        if (us != LINAC_OK) return us;
        {
            ProfScope ps(stream, PROF_FINISH);
            finish_kernel<<<1, NB_MAX, 0, stream>>>(st, d_pivots, d_rank);
        }
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    return LINAC_OK;
}

linac_status solve_pack(const uint32_t* dA, int64_t m, int64_t nA, int64_t ldA, const uint32_t* dB,
                        int64_t k, int64_t ldB, uint32_t* dM, int64_t ldM, cudaStream_t stream) {
    if (m == 0) return LINAC_OK;
    const int64_t total = m * ldM;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096));
    ProfScope ps(stream, PROF_SOLVE_PACK);
    pack_kernel<<<blocks, 256, 0, stream>>>(dA, m, nA, ldA, dB, k, ldB, dM, ldM);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

linac_status solve_extract(const uint32_t* dM, int64_t m, int64_t nA, int64_t k, int64_t ldM,
                           const int32_t* d_rank, const int32_t* d_pivots, uint32_t* dX, int64_t ldX,
                           uint8_t* d_consistent, cudaStream_t stream) {
    if (k == 0) return LINAC_OK;
    ProfScope ps(stream, PROF_SOLVE_EXTRACT);
    extract_kernel<<<(unsigned)k, 256, 0, stream>>>(dM, m, nA, ldM, d_rank, d_pivots, dX, ldX, d_consistent);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

linac_status validate_range(const uint32_t* dA, int64_t m, int64_t n, int64_t ld, uint32_t p,
                            int* d_status, cudaStream_t stream) {
    if (m == 0 || n == 0) return LINAC_OK;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m * n + 255) / 256, 4096));
    ProfScope ps(stream, PROF_VALIDATE);
    validate_kernel<<<blocks, 256, 0, stream>>>(dA, m, n, ld, p, d_status);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

}  // namespace linac
