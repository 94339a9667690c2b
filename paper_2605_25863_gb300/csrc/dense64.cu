// dense64.cu -- Gauss-Jordan elimination to RREF over Z/pZ for primes p < 2^64
// with uint64 residues (section 2.3, "Basic Usage": the uint64 backend for
// primes that do not fit 32 bits; section 3.2 for the elimination itself).
//
// Blocked, right-looking, like the 32-bit driver, with panels of NB64 = 32
// columns.  Per panel:
//   1. panel64_kernel (one block): fraction-free Gauss-Jordan of the panel
//      columns on a window of the first NB64 + 16 remaining rows, in
//      Montgomery form, tracking each row's combination of original rows.
//      If every panel column finds a pivot in the window, or the window
//      holds every remaining row, its pivots are the panel's.  Otherwise a
//      full-height search over all remaining rows picks the pivot rows and
//      the window elimination is repeated on exactly those rows.  Output:
//      k pivots (columns J, rows P) and E = G^(-1) for the k x k block
//      G = A[P, J], scaled by 2^128 for the update's reduction.
//   2. gather64_kernel: F = A[:, J] (every row), scaled by 2^128.
//   3. gemm64_kernel<assign>: R = E A[P, c0:n] (the pivot rows in RREF).
//   4. gemm64_kernel<update>: A[:, c0:n] -= F R for every row; the pivot
//      rows become zero (G E = I), every other row loses its J entries.
//   5. move64_kernel: the non-pivot rows in [r, r+k) go to the pivot rows'
//      old places at or after r+k, R goes to rows r..r+k-1.
//   6. advance64_kernel: pivot list, r += k.
// Steps 4 and 5 run twice: on the panel's first 64 columns (its own and the
// next panel's), then, after step 6, on the rest.  Steps 1 and 2 of the next
// panel run on a second stream meanwhile (see dense64_rref).  No block ever
// waits on another block; all state is device-resident, so the host issues a
// fixed sequence of launches per panel.
#include <algorithm>
#include <climits>
#include <map>
#include <mutex>
#include <utility>

#include "field64.cuh"
#include "linac_host.h"
#include "profile.h"

namespace linac {

constexpr int NB64 = 32;                    // panel width
constexpr int W64_ROWS = NB64 + 16;         // window rows
constexpr int P64_THREADS = 512;
constexpr int P64_WARPS = P64_THREADS / 32;
constexpr int P64_ROWS_PER_WARP = (W64_ROWS + P64_WARPS - 1) / P64_WARPS;
constexpr int G64_BM = 64, G64_BN = 64, G64_THREADS = 256;

// What one panel found.  Two of these alternate, so a panel kernel can run
// while the previous panel's update still reads its own.
struct Panel64Out {
    int32_t k;                 // pivots of the panel
    int32_t r0;                // rank before the panel = first row the pivot rows move to
    int32_t nmove;             // rows displaced by the move
    int32_t pad;
    int32_t pc[NB64];          // pivot columns (absolute), increasing
    int32_t pr[NB64];          // pivot rows (absolute, before the move), same order
    int32_t mv_src[NB64];      // displaced rows (in [r0, r0+k))
    int32_t mv_dst[NB64];      // their new places (old pivot rows at or after r0+k)
    uint64_t Et[NB64 * NB64];  // Et[s * NB64 + t] = E[t][s] * 2^128 mod p
};

struct Dense64State {
    int32_t r;                 // rank so far (advanced once a panel's first 64 columns are final)
    int32_t tall_panels;       // panels that needed the full-height search
    int32_t pad[2];
    Panel64Out out[2];
};

// ---------------------------------------------------------------------------
// Panel: window Gauss-Jordan with tracking, full-height search fallback

struct Panel64Smem {
    uint64_t X[W64_ROWS][NB64];        // window rows x panel columns (Montgomery)
    uint64_t T[W64_ROWS][NB64];        // row combinations: T[i][t] = coefficient of pivot t's original row
    uint64_t self[W64_ROWS];           // coefficient of the row's own original row (non-pivot rows)
    uint64_t dh[W64_ROWS];             // current head of each pivot row (Montgomery)
    uint64_t dinv[NB64];               // head^-1 * 2^128 mod p (times T R, one Montgomery product gives T head^-1 2^128)
    int32_t rowid[W64_ROWS];           // absolute row of each slot
    int32_t slot_piv[W64_ROWS];        // pivot index of the slot, -1
    int32_t pslot[NB64], pcl[NB64];    // slot and panel column of pivot t
    int32_t cand[2][P64_WARPS];        // per warp: its lowest candidate row for the next column
    int32_t red[P64_WARPS];
    int32_t q[2];
    int32_t ispos[NB64];               // move plan: position r + u already holds a pivot row
};

// Fraction-free Gauss-Jordan over the panel's w columns on the nrows rows
// listed in rowid: for each column, the lowest non-pivot slot with a nonzero
// entry becomes pivot number kk (slot q, head h), and every other slot i with
// entry f != 0 becomes h * row_i - f * row_q over the later panel columns.
// Each row also carries its combination of original rows: the coefficient of
// its own row (self) and of each pivot row chosen so far (T, indexed by pivot
// order, so only kk + 1 columns are live at step kk).  When q becomes pivot
// kk its own coefficient moves to T[q][kk].  Pivot heads are tracked in dh (a
// pivot row scaled by h has its head scaled by h).  Non-pivot rows never
// eliminate, so a pivot row's combination involves pivot rows only.
// Warp w owns rows w, w + P64_WARPS, ...; lanes take columns.  While a warp
// updates its rows it also finds its lowest candidate for the next column,
// so each column costs one block barrier.  Returns the number of pivots.
__device__ int gj_window64(const uint64_t* __restrict__ A, int64_t ld, int c0, int w, int nrows,
                           const Field64& f, Panel64Smem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t v[P64_ROWS_PER_WARP];
#pragma unroll
    for (int u = 0; u < P64_ROWS_PER_WARP; ++u) {
        const int i = warp + u * P64_WARPS;
        v[u] = (i < nrows && lane < w) ? A[(int64_t)sm.rowid[i] * ld + c0 + lane] : 0ull;
    }
    int cand = INT_MAX;
#pragma unroll
    for (int u = 0; u < P64_ROWS_PER_WARP; ++u) {
        const int i = warp + u * P64_WARPS;
        if (i < nrows) {
            sm.X[i][lane] = m64_to_mont(v[u], f);
            sm.T[i][lane] = 0ull;
            if (lane == 0) {
                sm.self[i] = f.r1;
                sm.slot_piv[i] = -1;
            }
            if (cand == INT_MAX && __shfl_sync(0xffffffffu, v[u], 0) != 0) cand = i;
        }
    }
    if (lane == 0) sm.cand[0][warp] = cand;
    __syncthreads();
    int kk = 0;
    for (int j = 0; j < w; ++j) {
        int q = lane < P64_WARPS ? sm.cand[j & 1][lane] : INT_MAX;
        q = __reduce_min_sync(0xffffffffu, q);
        const int jn = j + 1;
        int next = INT_MAX;
        if (q == INT_MAX) {
#pragma unroll
            for (int u = 0; u < P64_ROWS_PER_WARP; ++u) {
                const int i = warp + u * P64_WARPS;
                if (jn < w && i < nrows && next == INT_MAX && sm.slot_piv[i] < 0 && sm.X[i][jn] != 0) next = i;
            }
        } else {
            const uint64_t h = sm.X[q][j];
            const uint64_t self_q = sm.self[q];
            const int npan = w - j - 1;
            const int nwork = npan + kk + 1;
#pragma unroll
            for (int u = 0; u < P64_ROWS_PER_WARP; ++u) {
                const int i = warp + u * P64_WARPS;
                if (i >= nrows || i == q) continue;
                const uint64_t fi = sm.X[i][j];
                const bool piv_i = sm.slot_piv[i] >= 0;
                if (fi != 0) {
                    for (int cc = lane; cc < nwork; cc += 32) {
                        if (cc < npan) {
                            const int c = j + 1 + cc;
                            sm.X[i][c] = m64_sub(m64_mul(h, sm.X[i][c], f), m64_mul(fi, sm.X[q][c], f), f);
                        } else {
                            const int t = cc - npan;
                            const uint64_t yq = t == kk ? self_q : sm.T[q][t];
                            sm.T[i][t] = m64_sub(m64_mul(h, sm.T[i][t], f), m64_mul(fi, yq, f), f);
                        }
                    }
                    if (lane == 0) {
                        if (piv_i) sm.dh[i] = m64_mul(h, sm.dh[i], f);
                        else sm.self[i] = m64_mul(h, sm.self[i], f);
                    }
                }
                if (jn < w && !piv_i && next == INT_MAX) {
                    __syncwarp();   // lane 0 wrote X[i][jn] above
                    if (sm.X[i][jn] != 0) next = i;
                }
            }
            if (threadIdx.x == 0) {
                sm.T[q][kk] = self_q;
                sm.slot_piv[q] = kk;
                sm.pslot[kk] = q;
                sm.pcl[kk] = j;
                sm.dh[q] = h;
            }
            ++kk;
        }
        if (lane == 0) sm.cand[jn & 1][warp] = next;
        __syncthreads();
    }
    return kk;
}

// Full-height search: the pivot rows of the panel among all rows r..m-1.
// The panel columns are copied to `tall` (m - r rows of NB64 words) and
// reduced to row-echelon form column by column with the same fraction-free
// step, on raw residues: a product reduced by m64_mul carries an extra factor
// 2^-64, which scales a row without changing which of its entries are zero,
// and only that pattern decides the pivots.  A chosen row is cleared so it is
// never chosen again.  Writes the pivot rows to sm.rowid[0..kt), returns kt.
__device__ int tall_search64(const uint64_t* __restrict__ A, int64_t m, int64_t ld, int c0, int w, int r,
                             const Field64& f, uint64_t* __restrict__ tall, Panel64Smem& sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NWARP = P64_WARPS;
    const int64_t mrem = m - r;
    for (int64_t i = warp; i < mrem; i += NWARP)
        if (lane < w) tall[i * NB64 + lane] = A[(r + i) * ld + c0 + lane];
    __syncthreads();
    int kt = 0;
    for (int j = 0; j < w; ++j) {
        int best = INT_MAX;
        for (int64_t i = tid; i < mrem; i += P64_THREADS)
            if (tall[i * NB64 + j] != 0) { best = (int)i; break; }
        best = __reduce_min_sync(0xffffffffu, best);
        if (lane == 0) sm.red[warp] = best;
        __syncthreads();
        if (warp == 0) {
            int v = lane < NWARP ? sm.red[lane] : INT_MAX;
            v = __reduce_min_sync(0xffffffffu, v);
            if (lane == 0) sm.q[j & 1] = v;
        }
        __syncthreads();
        const int q = sm.q[j & 1];
        if (q == INT_MAX) continue;
        const uint64_t h = tall[(int64_t)q * NB64 + j];
        const int c = j + 1 + lane;
        const uint64_t yq = c < w ? tall[(int64_t)q * NB64 + c] : 0ull;
        for (int64_t i = warp; i < mrem; i += NWARP) {
            if (i == q) continue;
            const uint64_t fi = tall[i * NB64 + j];
            if (fi == 0 || c >= w) continue;
            tall[i * NB64 + c] = m64_sub(m64_mul(h, tall[i * NB64 + c], f), m64_mul(fi, yq, f), f);
        }
        __syncthreads();
        if (tid > j && tid < w) tall[(int64_t)q * NB64 + tid] = 0;
        if (tid == 0) sm.rowid[kt] = r + q;
        ++kt;
        __syncthreads();
    }
    return kt;
}

__global__ void __launch_bounds__(P64_THREADS)
panel64_kernel(const uint64_t* __restrict__ A, int64_t m, int64_t ld, int c0, int w, Field64 f,
               Dense64State* __restrict__ st, Panel64Out* __restrict__ po, uint64_t* __restrict__ tall) {
    __shared__ Panel64Smem sm;
    const int tid = threadIdx.x;
    const int r = st->r;
    const int64_t mrem = m - r;
    if (mrem <= 0 || w <= 0) {
        if (tid == 0) { po->k = 0; po->nmove = 0; po->r0 = r; }
        return;
    }
    int nrows = mrem < W64_ROWS ? (int)mrem : W64_ROWS;
    for (int i = tid; i < nrows; i += P64_THREADS) sm.rowid[i] = r + i;
    __syncthreads();
    int kk = gj_window64(A, ld, c0, w, nrows, f, sm);
    if (kk < w && mrem > W64_ROWS) {
        // the window may lack a pivot that a lower row holds
        __syncthreads();
        nrows = tall_search64(A, m, ld, c0, w, r, f, tall, sm);
        __syncthreads();
        kk = gj_window64(A, ld, c0, w, nrows, f, sm);
        if (tid == 0) st->tall_panels += 1;
    }
    __syncthreads();
    // E[t][s] = T_t[slot of pivot s] / head_t, scaled by 2^128: with the
    // tracking entry held as T R and dinv = head^-1 R^2, one Montgomery
    // product gives T head^-1 R^2.
    if (tid < kk) {
        const uint64_t inv = m64_pow(sm.dh[sm.pslot[tid]], f.p - 2, f);   // head^-1 R
        sm.dinv[tid] = m64_mul(inv, f.r2, f);                             // head^-1 R^2
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    for (int s = warp; s < kk; s += P64_WARPS)
        if (lane < kk) po->Et[s * NB64 + lane] = m64_mul(sm.T[sm.pslot[lane]][s], sm.dinv[lane], f);
    if (warp == 0) {
        // rows r..r+kk-1 receive the pivot rows (lane t: pivot t, position
        // r+t); the non-pivot rows there go to the places the pivot rows leave
        // at or after r+kk, paired in order by two ballots
        const int prow = lane < kk ? sm.rowid[sm.pslot[lane]] : -1;
        if (lane < kk) {
            po->pc[lane] = c0 + sm.pcl[lane];
            po->pr[lane] = prow;
        }
        sm.ispos[lane] = 0;
        __syncwarp();
        if (lane < kk && prow < r + kk) sm.ispos[prow - r] = 1;
        __syncwarp();
        const bool displaced = lane < kk && !sm.ispos[lane];
        const bool vacated = lane < kk && prow >= r + kk;
        const unsigned bd = __ballot_sync(0xffffffffu, displaced), bv = __ballot_sync(0xffffffffu, vacated);
        const unsigned below = (1u << lane) - 1u;
        if (displaced) po->mv_src[__popc(bd & below)] = r + lane;
        if (vacated) po->mv_dst[__popc(bv & below)] = prow;
        if (lane == 0) {
            po->nmove = __popc(bd);   // equal to __popc(bv): both count the pivot rows outside [r, r+kk)
            po->r0 = r;
            po->k = kk;
        }
    }
}

// ---------------------------------------------------------------------------
// F = A[:, J] * 2^128 mod p, stored transposed: Ft[s * ldF + i]; rows m..ldF-1
// are zero.

__global__ void __launch_bounds__(256)
gather64_kernel(const uint64_t* __restrict__ A, int64_t m, int64_t ld, const Panel64Out* __restrict__ po,
                Field64 f, uint64_t* __restrict__ Ft, int64_t ldF) {
    __shared__ int32_t pcs[NB64];
    const int k = po->k;
    if (k == 0) return;
    if (threadIdx.x < k) pcs[threadIdx.x] = po->pc[threadIdx.x];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ldF; i += (int64_t)gridDim.x * blockDim.x) {
        for (int s = 0; s < k; ++s) {
            const uint64_t v = i < m ? m64_mul(A[i * ld + pcs[s]], f.r3, f) : 0ull;
            Ft[(int64_t)s * ldF + i] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// C (rows x ncols) = sum_s At[s][i] B[s][j] / 2^128 mod p (ASSIGN), or
// C -= that (update).  k = po->k <= NB64 products per output, accumulated
// exactly in 160 bits.  Rows of B are B + brow[s] * ldB (brow = null: s).
// ASSIGN takes rows = k (the pivot rows).  64 x 64 tile per 256-thread
// block; each thread owns 4 rows x (2 + 2) columns, the columns split so
// that a warp's 16-byte shared-memory reads of B are conflict free.

template <bool ASSIGN>
__global__ void __launch_bounds__(G64_THREADS, 2)
gemm64_kernel(const uint64_t* __restrict__ At, int64_t ldAt, const uint64_t* __restrict__ B, int64_t ldB,
              const int32_t* __restrict__ brow, uint64_t* __restrict__ C, int64_t ldC, int64_t nrows,
              int64_t ncols, const Panel64Out* __restrict__ po, Field64 f) {
    __shared__ __align__(16) uint64_t As[NB64][G64_BM];
    __shared__ __align__(16) uint64_t Bs[NB64][G64_BN];
    const int k = po->k;
    if (k == 0) return;
    const int64_t rows = ASSIGN ? (int64_t)k : nrows;
    const int64_t i0 = (int64_t)blockIdx.y * G64_BM, j0 = (int64_t)blockIdx.x * G64_BN;
    if (i0 >= rows) return;
    const int tid = threadIdx.x;
    for (int e = tid; e < k * G64_BM; e += G64_THREADS) {
        const int s = e / G64_BM, ii = e % G64_BM;
        As[s][ii] = i0 + ii < rows ? At[(int64_t)s * ldAt + i0 + ii] : 0ull;
    }
    for (int e = tid; e < k * (G64_BN / 2); e += G64_THREADS) {
        const int s = e / (G64_BN / 2), jj = 2 * (e % (G64_BN / 2));
        const int64_t j = j0 + jj;
        const uint64_t* src = B + (int64_t)(brow ? brow[s] : s) * ldB + j;
        ulonglong2 v = make_ulonglong2(0ull, 0ull);
        if (j + 1 < ncols) v = *reinterpret_cast<const ulonglong2*>(src);
        else if (j < ncols) v.x = src[0];
        *reinterpret_cast<ulonglong2*>(&Bs[s][jj]) = v;
    }
    __syncthreads();

    const int ty = tid >> 4, tx = tid & 15;
    uint32_t acc[4][4][5];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int l = 0; l < 5; ++l) acc[u][v][l] = 0u;
    for (int s = 0; s < k; ++s) {
        const ulonglong2 a01 = *reinterpret_cast<const ulonglong2*>(&As[s][ty * 4]);
        const ulonglong2 a23 = *reinterpret_cast<const ulonglong2*>(&As[s][ty * 4 + 2]);
        const ulonglong2 b01 = *reinterpret_cast<const ulonglong2*>(&Bs[s][tx * 2]);
        const ulonglong2 b23 = *reinterpret_cast<const ulonglong2*>(&Bs[s][32 + tx * 2]);
        const uint64_t a[4] = {a01.x, a01.y, a23.x, a23.y};
        const uint64_t b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) mac160(acc[u][v], a[u], b[v]);
    }

#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + ty * 4 + u;
        if (i >= rows) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int64_t j = j0 + half * 32 + tx * 2;
            if (j >= ncols) continue;
            uint64_t* dst = C + i * ldC + j;
            const uint64_t v0 = reduce160(acc[u][half * 2], f);
            if (j + 1 < ncols) {
                const uint64_t v1 = reduce160(acc[u][half * 2 + 1], f);
                ulonglong2 o;
                if (ASSIGN) {
                    o = make_ulonglong2(v0, v1);
                } else {
                    const ulonglong2 c = *reinterpret_cast<const ulonglong2*>(dst);
                    o = make_ulonglong2(m64_sub(c.x, v0, f), m64_sub(c.y, v1, f));
                }
                *reinterpret_cast<ulonglong2*>(dst) = o;
            } else {
                dst[0] = ASSIGN ? v0 : m64_sub(dst[0], v0, f);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Move, advance, init

// Columns [c0 + j0, c0 + j1): the displaced rows go to the pivot rows' old
// places, then R (columns relative to c0) fills rows r0..r0+k-1.
__global__ void __launch_bounds__(256)
move64_kernel(uint64_t* __restrict__ A, int64_t ld, int c0, int64_t j0, int64_t j1,
              const Panel64Out* __restrict__ po, const uint64_t* __restrict__ R, int64_t ldR) {
    __shared__ int32_t src[NB64], dst[NB64];
    const int k = po->k;
    if (k == 0) return;
    const int r = po->r0, nm = po->nmove;
    if (threadIdx.x < nm) {
        src[threadIdx.x] = po->mv_src[threadIdx.x];
        dst[threadIdx.x] = po->mv_dst[threadIdx.x];
    }
    __syncthreads();
    for (int64_t j = j0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < j1; j += (int64_t)gridDim.x * blockDim.x) {
        uint64_t* col = A + c0 + j;
        for (int u = 0; u < nm; ++u) col[(int64_t)dst[u] * ld] = col[(int64_t)src[u] * ld];
        for (int t = 0; t < k; ++t) col[(int64_t)(r + t) * ld] = R[(int64_t)t * ldR + j];
    }
}

// Pivot list and rank; the panel's record stays for its remaining columns.
__global__ void advance64_kernel(Dense64State* __restrict__ st, const Panel64Out* __restrict__ po,
                                 int32_t* __restrict__ pivots, int32_t* __restrict__ d_rank) {
    const int k = po->k, r = po->r0;
    if ((int)threadIdx.x < k) pivots[r + threadIdx.x] = po->pc[threadIdx.x];
    if (threadIdx.x == 0) {
        st->r = r + k;
        *d_rank = r + k;
    }
}

__global__ void init64_kernel(Dense64State* __restrict__ st, int32_t* __restrict__ pivots, int64_t npiv,
                              int32_t* __restrict__ d_rank) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npiv; i += (int64_t)gridDim.x * blockDim.x)
        pivots[i] = -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->r = 0;
        st->tall_panels = 0;
        for (int b = 0; b < 2; ++b) {
            st->out[b].k = 0;
            st->out[b].nmove = 0;
            st->out[b].r0 = 0;
        }
        *d_rank = 0;
    }
}

// ---------------------------------------------------------------------------
// Solve helpers and range validation (uint64)

__global__ void pack64_kernel(const uint64_t* __restrict__ A, int64_t m, int64_t nA, int64_t ldA,
                              const uint64_t* __restrict__ B, int64_t k, int64_t ldB, uint64_t* __restrict__ Mx,
                              int64_t ldM) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * ldM; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ldM, j = e % ldM;
        uint64_t v = 0;
        if (j < nA) v = A[i * ldA + j];
        else if (j < nA + k) v = B[i * ldB + (j - nA)];
        Mx[e] = v;
    }
}

// One block per right-hand side j (section 5.2): consistent iff its reduced
// column vanishes at and below the rank; X from the pivot rows, free
// variables zero.
__global__ void __launch_bounds__(256)
extract64_kernel(const uint64_t* __restrict__ Mx, int64_t m, int64_t nA, int64_t ldM,
                 const int32_t* __restrict__ d_rank, const int32_t* __restrict__ d_pivots,
                 uint64_t* __restrict__ X, int64_t ldX, uint8_t* __restrict__ cons) {
    __shared__ int s_bad;
    const int64_t j = blockIdx.x;
    const int rank = *d_rank;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    bool bad = false;
    for (int64_t i = rank + threadIdx.x; i < m; i += blockDim.x) bad |= Mx[i * ldM + nA + j] != 0;
    if (bad) atomicOr(&s_bad, 1);
    __syncthreads();
    const bool ok = s_bad == 0;
    if (threadIdx.x == 0) cons[j] = ok ? 1 : 0;
    for (int64_t i = threadIdx.x; i < nA; i += blockDim.x) X[i * ldX + j] = 0;
    __syncthreads();
    if (!ok) return;
    for (int t = threadIdx.x; t < rank; t += blockDim.x)
        X[(int64_t)d_pivots[t] * ldX + j] = Mx[(int64_t)t * ldM + nA + j];
}

__global__ void validate64_kernel(const uint64_t* __restrict__ A, int64_t m, int64_t n, int64_t ld, uint64_t p,
                                  int* status) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * n; e += (int64_t)gridDim.x * blockDim.x) {
        if (A[(e / n) * ld + e % n] >= p) {
            atomicCAS(status, 0, (int)LINAC_ERR_RANGE);
            return;
        }
    }
}

// ---------------------------------------------------------------------------
// Host driver

namespace {

struct Dense64Layout {
    size_t off_state, off_ft, off_r, off_tall, total;
    int64_t ldF, ldR;
};

Dense64Layout dense64_layout(int64_t m, int64_t n) {
    Dense64Layout L;
    size_t o = 0;
    L.off_state = o; o = align_up(o + sizeof(Dense64State), 256);
    L.ldF = (int64_t)align_up((size_t)std::max<int64_t>(m, 1), G64_BM);
    L.off_ft = o;    o = align_up(o + (size_t)2 * NB64 * L.ldF * 8, 256);   // two F buffers
    L.ldR = (int64_t)align_up((size_t)std::max<int64_t>(n, 1), G64_BN);
    L.off_r = o;     o = align_up(o + (size_t)NB64 * L.ldR * 8, 256);
    L.off_tall = o;  o = align_up(o + (size_t)std::max<int64_t>(m, 1) * NB64 * 8, 256);
    L.total = o;
    return L;
}

// Second stream (highest priority) and events of one caller stream: the
// panel kernels run on `side` so that each overlaps the previous panel's
// update.  Created on first
// use per (device, stream) and kept for the life of the process.
struct Side64 {
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, panel = nullptr, narrow = nullptr;
};
std::mutex g_side_mu;
std::map<std::pair<int, cudaStream_t>, Side64> g_side;

linac_status side64_get(cudaStream_t stream, Side64* out) {
    int dev = 0;
    LINAC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_side_mu);
    Side64& sd = g_side[std::make_pair(dev, stream)];
    if (!sd.side) {
        // highest priority: when an update block retires, the block scheduler
        // places the waiting panel block first instead of another update block
        int least = 0, greatest = 0;
        LINAC_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        LINAC_CUDA_TRY(cudaStreamCreateWithPriority(&sd.side, cudaStreamNonBlocking, greatest));
        LINAC_CUDA_TRY(cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming));
        LINAC_CUDA_TRY(cudaEventCreateWithFlags(&sd.panel, cudaEventDisableTiming));
        LINAC_CUDA_TRY(cudaEventCreateWithFlags(&sd.narrow, cudaEventDisableTiming));
    }
    *out = sd;
    return LINAC_OK;
}

}  // namespace

size_t dense64_workspace_bytes(int64_t m, int64_t n) { return dense64_layout(m, n).total; }

// Per panel t (record out[t & 1], F buffer t & 1):
//   side:   [wait: panel t-1's first 64 columns final] panel kernel, gather F
//   stream: [wait: panel t] R = E W; update and move of the panel's first 64
//           columns (its own 32 and the next panel's 32); advance the rank
//           [signal]; update and move of the remaining columns.
// So panel t+1 runs while panel t's remaining columns are updated.  The next
// R = E W waits for that update (stream order), the next gather writes the
// other F buffer, and the next panel writes the other record; each buffer's
// previous reader finished before the signal the writer waits for.
linac_status dense64_rref(uint64_t* dA, int64_t m, int64_t n, int64_t ld, const Field64& f, int64_t nsearch,
                          int32_t* d_rank, int32_t* d_pivots, cudaStream_t stream) {
    const int64_t npiv = std::min(m, nsearch);
    if ((m + G64_BM - 1) / G64_BM > 65535) return LINAC_ERR_UNSUPPORTED;
    const Dense64Layout L = dense64_layout(m, n);
    void* base = nullptr;
    linac_status s = scratch_get_slot(stream, 6, L.total, &base);
    if (s != LINAC_OK) return s;
    Side64 sd;
    if ((s = side64_get(stream, &sd)) != LINAC_OK) return s;
    char* ws = (char*)base;
    Dense64State* st = (Dense64State*)(ws + L.off_state);
    uint64_t* Ft2[2] = {(uint64_t*)(ws + L.off_ft), (uint64_t*)(ws + L.off_ft) + (size_t)NB64 * L.ldF};
    uint64_t* R = (uint64_t*)(ws + L.off_r);
    uint64_t* tall = (uint64_t*)(ws + L.off_tall);
    {
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((npiv + 255) / 256, 1024));
        ProfScope ps(stream, PROF_INIT);
        init64_kernel<<<blocks, 256, 0, stream>>>(st, d_pivots, npiv, d_rank);
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    if (m == 0 || n == 0 || nsearch == 0) return LINAC_OK;   // no panel: nothing forks to the side stream
    const unsigned gather_blocks = (unsigned)std::min<int64_t>((L.ldF + 255) / 256, 1024);
    const unsigned gy = (unsigned)((m + G64_BM - 1) / G64_BM);
    LINAC_CUDA_TRY(cudaEventRecord(sd.fork, stream));
    LINAC_CUDA_TRY(cudaStreamWaitEvent(sd.side, sd.fork, 0));
    int t = 0;
    for (int64_t c0 = 0; c0 < nsearch; c0 += NB64, ++t) {
        const int w = (int)std::min<int64_t>(NB64, nsearch - c0);
        const int64_t ncols = n - c0;
        const int64_t nnarrow = std::min<int64_t>(ncols, G64_BN);
        Panel64Out* po = &st->out[t & 1];
        uint64_t* Ft = Ft2[t & 1];
        if (t > 0) LINAC_CUDA_TRY(cudaStreamWaitEvent(sd.side, sd.narrow, 0));
        {
            ProfScope ps(sd.side, PROF_U64_PANEL);
            panel64_kernel<<<1, P64_THREADS, 0, sd.side>>>(dA, m, ld, (int)c0, w, f, st, po, tall);
        }
        {
            ProfScope ps(sd.side, PROF_GATHER_F);
            gather64_kernel<<<gather_blocks, 256, 0, sd.side>>>(dA, m, ld, po, f, Ft, L.ldF);
        }
        LINAC_CUDA_TRY(cudaEventRecord(sd.panel, sd.side));
        LINAC_CUDA_TRY(cudaStreamWaitEvent(stream, sd.panel, 0));
        {
            ProfScope ps(stream, PROF_TRSM);
            const unsigned gx = (unsigned)((ncols + G64_BN - 1) / G64_BN);
            gemm64_kernel<true><<<dim3(gx, 1), G64_THREADS, 0, stream>>>(po->Et, NB64, dA + c0, ld, po->pr, R,
                                                                         L.ldR, NB64, ncols, po, f);
        }
        {
            ProfScope ps(stream, PROF_U64_UPDATE);
            gemm64_kernel<false><<<dim3(1, gy), G64_THREADS, 0, stream>>>(Ft, L.ldF, R, L.ldR, nullptr, dA + c0, ld,
                                                                          m, nnarrow, po, f);
        }
        {
            ProfScope ps(stream, PROF_MOVE);
            move64_kernel<<<1, 256, 0, stream>>>(dA, ld, (int)c0, 0, nnarrow, po, R, L.ldR);
        }
        {
            ProfScope ps(stream, PROF_FINISH);
            advance64_kernel<<<1, NB64, 0, stream>>>(st, po, d_pivots, d_rank);
        }
        LINAC_CUDA_TRY(cudaEventRecord(sd.narrow, stream));
        if (ncols > nnarrow) {
            const int64_t nrest = ncols - nnarrow;
            {
                ProfScope ps(stream, PROF_U64_UPDATE);
                const unsigned gx = (unsigned)((nrest + G64_BN - 1) / G64_BN);
                gemm64_kernel<false><<<dim3(gx, gy), G64_THREADS, 0, stream>>>(
                    Ft, L.ldF, R + nnarrow, L.ldR, nullptr, dA + c0 + nnarrow, ld, m, nrest, po, f);
            }
            {
                ProfScope ps(stream, PROF_MOVE);
                const unsigned mb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nrest + 255) / 256, 1024));
                move64_kernel<<<mb, 256, 0, stream>>>(dA, ld, (int)c0, nnarrow, ncols, po, R, L.ldR);
            }
        }
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    return LINAC_OK;
}

linac_status solve64_pack(const uint64_t* dA, int64_t m, int64_t nA, int64_t ldA, const uint64_t* dB, int64_t k,
                          int64_t ldB, uint64_t* dM, int64_t ldM, cudaStream_t stream) {
    if (m == 0) return LINAC_OK;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m * ldM + 255) / 256, 4096));
    ProfScope ps(stream, PROF_SOLVE_PACK);
    pack64_kernel<<<blocks, 256, 0, stream>>>(dA, m, nA, ldA, dB, k, ldB, dM, ldM);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

linac_status solve64_extract(const uint64_t* dM, int64_t m, int64_t nA, int64_t k, int64_t ldM,
                             const int32_t* d_rank, const int32_t* d_pivots, uint64_t* dX, int64_t ldX,
                             uint8_t* d_consistent, cudaStream_t stream) {
    if (k == 0) return LINAC_OK;
    ProfScope ps(stream, PROF_SOLVE_EXTRACT);
    extract64_kernel<<<(unsigned)k, 256, 0, stream>>>(dM, m, nA, ldM, d_rank, d_pivots, dX, ldX, d_consistent);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

linac_status validate64_range(const uint64_t* dA, int64_t m, int64_t n, int64_t ld, uint64_t p, int* d_status,
                              cudaStream_t stream) {
    if (m == 0 || n == 0) return LINAC_OK;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m * n + 255) / 256, 4096));
    ProfScope ps(stream, PROF_VALIDATE);
    validate64_kernel<<<blocks, 256, 0, stream>>>(dA, m, n, ld, p, d_status);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

}  // namespace linac
