// lup.cu -- LUP factorisation P A = L U over Z/pZ (linac_lup).
//
// Paper section 6 ("Conclusions and Outlook") names an LUP factorisation as
// the option to add beside the rank decomposition.  The reading implemented
// (and pinned in the oracle): the elimination is the column loop of section
// 3.2, but only the rows that are not yet pivots are reduced, pivot rows are
// not rescaled, and each column's pivot is the lowest-index row, in the
// ORIGINAL order, among the rows not yet used whose entry is nonzero.  P lists
// the pivot rows in pivot order, then the other rows in increasing order; L
// holds the multipliers; U is the row-echelon form.
//
// Blocked like the RREF driver (dense.cu), but rows never move: the rows that
// are not pivots yet are kept in a device list in increasing order, and the
// pivot search and the updates address rows through it.  Per panel of nb
// columns [c0, c1):
//   1. window_kernel / panel_kernel (shared with the RREF) find the k pivots
//      among the listed rows: J (columns), Pi (rows, in pivot order);
//   2. gather_w: W = M[Pi, c0:n] (balanced);
//   3. lu_panel_kernel: the unscaled LU of W's panel block, W_p = L11 U11 (k
//      inverse heads, one per stage), E = L11^-1 and T = U11[:, J]^-1;
//   4. U_p = E W (the panel's U rows), R = T U_p = G^-1 W with G = W[:, J]
//      (so R[:, J] = I), on the assign GEMM of the trailing update;
//   5. the list drops the pivot rows; F = M[list, J]; L21 = F T (stored
//      transposed), again on the assign GEMM;
//   6. every listed row: M[row, c0:n] -= F[row] R (the Schur complement,
//      F G^-1 W = L21 U_p; the RREF's update kernel, row-mapped mode);
//   7. write-back: pivot row t gets U_p[t] and L11[t][s] at J_s (s < t);
//      listed rows get L21 at J (their entries there are now zero);
//   8. perm[r + t] = Pi[t], pivots[r + t] = J[t], r += k.
// The work matrix then holds L and U packed in the original row positions;
// a final gather writes L (m x min(m, n), unit lower) and U (m x n) in P's
// order.
#include <algorithm>
#include <climits>

#include "dense_kernels.cuh"
#include "linac_host.h"
#include "profile.h"
#include "update.cuh"

namespace linac {

namespace {

constexpr int LU_THREADS = 512;
constexpr int LU_S = NB_MAX + 1;
constexpr size_t LU_SMEM = (size_t)3 * NB_MAX * LU_S * 4;

// Step 3.  One block.  W is k x ldW (balanced; columns 0..w-1 are the panel).
// Outputs (NB_MAX x NB_MAX, zero outside k x k): L11c[t][s] = L11 (canonical),
// EtE[s][t] = E[t][s], EtT[s][t] = T[t][s], TL[s][t] = T[s][t] (balanced; the
// first two are the transposed left operands of R = E W and R = T U_p, the
// third that of L21^T = T^T F^T).
__global__ void __launch_bounds__(LU_THREADS)
lu_panel_kernel(const DenseState* __restrict__ st, const int32_t* __restrict__ W, int64_t ldW, int c0, int w,
                Field f, uint32_t* __restrict__ L11c, int32_t* __restrict__ EtE, int32_t* __restrict__ EtT,
                int32_t* __restrict__ TL) {
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t* U = sm;                         // U[t][j]: the panel block, reduced in place
    uint32_t* Lm = sm + NB_MAX * LU_S;        // L11, then Tu
    uint32_t* Ei = sm + 2 * NB_MAX * LU_S;    // E = L11^-1
    __shared__ uint32_t hinv[NB_MAX];
    __shared__ int Jl[NB_MAX];
    const int k = st->k;
    const int tid = threadIdx.x;
    for (int e = tid; e < NB_MAX * NB_MAX; e += blockDim.x) {
        L11c[e] = 0;
        EtE[e] = 0;
        EtT[e] = 0;
        TL[e] = 0;
    }
    if (k == 0) return;
    for (int t = tid; t < k; t += blockDim.x) Jl[t] = st->J[t] - c0;
    for (int e = tid; e < k * w; e += blockDim.x) {
        const int t = e / w, j = e - t * w;
        U[t * LU_S + j] = from_balanced(W[(int64_t)t * ldW + j], f);
    }
    for (int e = tid; e < k * k; e += blockDim.x) {
        const int t = e / k, s = e - t * k;
        Lm[t * LU_S + s] = t == s ? 1u : 0u;
        Ei[t * LU_S + s] = t == s ? 1u : 0u;
    }
    __syncthreads();
    // forward elimination of the pivot rows in pivot order (unscaled):
    // row t <- row t - l_ts row s with l_ts = U[t][J_s] / U[s][J_s]
    for (int s = 0; s < k; ++s) {
        const int js = Jl[s];
        if (tid == 0) hinv[s] = inverse_mod(U[s * LU_S + js], f.p);
        __syncthreads();
        const uint32_t hi = hinv[s];
        for (int t = s + 1 + tid; t < k; t += blockDim.x) Lm[t * LU_S + s] = mulmod(U[t * LU_S + js], hi, f);
        __syncthreads();
        const int nc = w - js;
        for (int e = tid; e < (k - s - 1) * nc; e += blockDim.x) {
            const int t = s + 1 + e / nc, j = js + e % nc;
            const uint32_t l = Lm[t * LU_S + s];
            if (l) U[t * LU_S + j] = submod(U[t * LU_S + j], mulmod(l, U[s * LU_S + j], f), f);
        }
        __syncthreads();
    }
    // E = L11^-1 by forward substitution, stage s: rows t > s, columns <= s
    for (int s = 0; s + 1 < k; ++s) {
        for (int e = tid; e < (k - s - 1) * (s + 1); e += blockDim.x) {
            const int t = s + 1 + e / (s + 1), c = e % (s + 1);
            const uint32_t l = Lm[t * LU_S + s];
            if (l) Ei[t * LU_S + c] = submod(Ei[t * LU_S + c], mulmod(l, Ei[s * LU_S + c], f), f);
        }
        __syncthreads();
    }
    for (int e = tid; e < k * k; e += blockDim.x) {
        const int t = e / k, s = e - t * k;
        if (s < t) L11c[t * NB_MAX + s] = Lm[t * LU_S + s];
        EtE[s * NB_MAX + t] = to_balanced(Ei[t * LU_S + s], f);
    }
    __syncthreads();
    // T = U11[:, J]^-1 = Uh^-1 D^-1 with D = diag(heads), Uh = D^-1 U11[:, J]
    // unit upper: Tu = Uh^-1 by back substitution (stage s: rows t < s,
    // columns >= s), reusing Lm for Tu and Ei for Uh
    for (int e = tid; e < k * k; e += blockDim.x) {
        const int t = e / k, u = e - t * k;
        Ei[t * LU_S + u] = u > t ? mulmod(U[t * LU_S + Jl[u]], hinv[t], f) : 0u;
        Lm[t * LU_S + u] = t == u ? 1u : 0u;
    }
    __syncthreads();
    for (int s = k - 1; s >= 1; --s) {
        for (int e = tid; e < s * (k - s); e += blockDim.x) {
            const int t = e / (k - s), c = s + e % (k - s);
            const uint32_t u = Ei[t * LU_S + s];
            if (u) Lm[t * LU_S + c] = submod(Lm[t * LU_S + c], mulmod(u, Lm[s * LU_S + c], f), f);
        }
        __syncthreads();
    }
    for (int e = tid; e < k * k; e += blockDim.x) {
        const int t = e / k, u = e - t * k;
        const int32_t T = to_balanced(mulmod(Lm[t * LU_S + u], hinv[u], f), f);
        EtT[u * NB_MAX + t] = T;
        TL[t * NB_MAX + u] = T;
    }
}

// Step 5: drop this panel's pivot rows from the list (stable).  One block;
// mark holds one byte per row of M.
__global__ void __launch_bounds__(1024)
lu_compact_kernel(const DenseState* __restrict__ st, int64_t m, const int32_t* __restrict__ cur,
                  int32_t* __restrict__ next, uint8_t* __restrict__ mark) {
    __shared__ int wsum[32];
    __shared__ int carry;
    const int k = st->k, r = st->r;
    const int64_t len = m - r;
    for (int t = threadIdx.x; t < k; t += blockDim.x) mark[st->Pi[t]] = 1;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < len; base += blockDim.x) {
        const int64_t x = base + threadIdx.x;
        const int row = x < len ? cur[x] : -1;
        const int keep = row >= 0 && !mark[row];
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int before = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            wsum[lane] = v;   // inclusive prefix over warps
        }
        __syncthreads();
        const int off = carry + (warp ? wsum[warp - 1] : 0);
        if (keep) next[off + before] = row;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    for (int t = threadIdx.x; t < k; t += blockDim.x) mark[st->Pi[t]] = 0;
}

// Step 7.  Block t < k: pivot row Pi[t] receives U_p[t] (columns c0..n) and
// L11[t][s] at J_s (s < t).  Blocks k.. : listed rows receive L21 at J.
__global__ void __launch_bounds__(256)
lu_writeback_kernel(uint32_t* __restrict__ M, int64_t m, int64_t ld, int64_t ncols, int c0, Field f,
                    const DenseState* __restrict__ st, const int32_t* __restrict__ Up, int64_t ldU,
                    const uint32_t* __restrict__ L11c, const int32_t* __restrict__ L21t, int64_t ldL,
                    const int32_t* __restrict__ list) {
    const int k = st->k;
    if (k == 0) return;
    const int b = blockIdx.x;
    if (b < NB_MAX) {
        if (b >= k) return;
        uint32_t* row = M + (int64_t)st->Pi[b] * ld + c0;
        const int32_t* up = Up + (int64_t)b * ldU;
        for (int64_t j = threadIdx.x; j < ncols; j += blockDim.x) row[j] = from_balanced(up[j], f);
        __syncthreads();
        for (int s = threadIdx.x; s < b; s += blockDim.x) row[st->J[s] - c0] = L11c[b * NB_MAX + s];
        return;
    }
    const int64_t left = m - st->r - k;
    for (int64_t i = (int64_t)(b - NB_MAX) * blockDim.x + threadIdx.x; i < left;
         i += (int64_t)(gridDim.x - NB_MAX) * blockDim.x) {
        uint32_t* row = M + (int64_t)list[i] * ld;
        for (int t = 0; t < k; ++t) row[st->J[t]] = from_balanced(L21t[(int64_t)t * ldL + i], f);
    }
}

// Step 8 (perm part): perm[r + t] = Pi[t].
__global__ void lu_perm_kernel(const DenseState* __restrict__ st, int32_t* __restrict__ perm) {
    const int k = st->k, r = st->r;
    for (int t = threadIdx.x; t < k; t += blockDim.x) perm[r + t] = st->Pi[t];
}

// The list of rows left at the end completes P: perm[rank + x] = list[x].
__global__ void lu_perm_tail_kernel(const int32_t* __restrict__ d_rank, int64_t m, const int32_t* __restrict__ list,
                                    int32_t* __restrict__ perm) {
    const int r = *d_rank;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < m - r; x += (int64_t)gridDim.x * blockDim.x)
        perm[r + x] = list[x];
}

__global__ void lu_list_init_kernel(int32_t* __restrict__ a, int32_t* __restrict__ b, uint8_t* __restrict__ mark,
                                    int64_t m) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < m; x += (int64_t)gridDim.x * blockDim.x) {
        a[x] = (int32_t)x;
        b[x] = (int32_t)x;
        mark[x] = 0;
    }
}

// Output: row i of L and U from the packed work matrix, in P's order.  One
// block per row.
__global__ void __launch_bounds__(256)
lu_output_kernel(const uint32_t* __restrict__ Wm, int64_t m, int64_t n, int64_t ldw,
                 const int32_t* __restrict__ perm, const int32_t* __restrict__ d_rank,
                 const int32_t* __restrict__ piv, uint32_t* __restrict__ L, int64_t ldL, uint32_t* __restrict__ U,
                 int64_t ldU) {
    const int64_t i = blockIdx.x;
    const int r = *d_rank;
    const int64_t mn = m < n ? m : n;
    const uint32_t* src = Wm + (int64_t)perm[i] * ldw;
    const int64_t head = i < r ? piv[i] : n;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) U[i * ldU + j] = j >= head ? src[j] : 0u;
    for (int64_t s = threadIdx.x; s < mn; s += blockDim.x) {
        uint32_t v = 0;
        if (s == i) v = 1;
        else if (s < i && s < r) v = src[piv[s]];
        L[i * ldL + s] = v;
    }
}

struct LupLayout {
    size_t off_w, off_state, off_cand, off_panel, off_l11, off_ete, off_ett, off_tl, off_ft, off_wt, off_up, off_r,
        off_l21, off_lista, off_listb, off_mark, total;
    int64_t ldw, ldF, ldW;
};

LupLayout lup_layout(int64_t m, int64_t n, int G) {
    LupLayout L;
    size_t o = 0;
    L.ldw = (int64_t)align_up((size_t)std::max<int64_t>(n, 1), 4);
    L.ldF = (int64_t)align_up((size_t)std::max<int64_t>(m, 1), 4);
    L.ldW = L.ldw;
    const size_t nb2 = (size_t)NB_MAX * NB_MAX * 4;
    L.off_w = o;      o = align_up(o + (size_t)std::max<int64_t>(m, 1) * L.ldw * 4, 256);
    L.off_state = o;  o = align_up(o + sizeof(DenseState), 256);
    L.off_cand = o;   o = align_up(o + (size_t)2 * G * (NB_MAX + 1) * 4, 256);
    L.off_panel = o;  o = align_up(o + nb2, 256);
    L.off_l11 = o;    o = align_up(o + nb2, 256);
    L.off_ete = o;    o = align_up(o + nb2, 256);
    L.off_ett = o;    o = align_up(o + nb2, 256);
    L.off_tl = o;     o = align_up(o + nb2, 256);
    L.off_ft = o;     o = align_up(o + (size_t)NB_MAX * L.ldF * 4, 256);
    L.off_wt = o;     o = align_up(o + (size_t)NB_MAX * L.ldW * 4, 256);
    L.off_up = o;     o = align_up(o + (size_t)NB_MAX * L.ldW * 4, 256);
    L.off_r = o;      o = align_up(o + (size_t)NB_MAX * L.ldW * 4, 256);
    L.off_l21 = o;    o = align_up(o + (size_t)NB_MAX * L.ldF * 4, 256);
    L.off_lista = o;  o = align_up(o + (size_t)std::max<int64_t>(m, 1) * 4, 256);
    L.off_listb = o;  o = align_up(o + (size_t)std::max<int64_t>(m, 1) * 4, 256);
    L.off_mark = o;   o = align_up(o + (size_t)std::max<int64_t>(m, 1), 256);
    L.total = o;
    return L;
}

}  // namespace

linac_status lup_factor(const uint32_t* dA, int64_t m, int64_t n, int64_t ldA, const Field& f, uint32_t* dL,
                        int64_t ldL, uint32_t* dU, int64_t ldU, int32_t* d_perm, int32_t* d_rank,
                        int32_t* d_pivots, cudaStream_t stream) {
    int* status = status_word(stream);
    if (!status) return LINAC_ERR_NOMEM;
    const int64_t mn = std::min(m, n);
    int nb = dense_default_nb(m, n);
    const int G = panel_grid(m);
    const int S_max = (int)((std::max<int64_t>(m, 1) + G - 1) / G);
    size_t psmem = panel_smem(S_max, nb);
    const int max_smem = max_smem_optin();
    if (max_smem <= 0) return LINAC_ERR_CUDA;
    while (psmem > (size_t)max_smem - 1024 && nb > UPD_BK) {
        nb -= UPD_BK;
        psmem = panel_smem(S_max, nb);
    }
    if (psmem > (size_t)max_smem - 1024 || LU_SMEM > (size_t)max_smem) return LINAC_ERR_UNSUPPORTED;
    if ((m + UPD_BM - 1) / UPD_BM > 65535 || m > INT32_MAX / 2) return LINAC_ERR_UNSUPPORTED;

    const LupLayout L = lup_layout(m, n, G);
    void* base = nullptr;
    linac_status s = scratch_get_slot(stream, 10, L.total, &base);
    if (s != LINAC_OK) return s;
    char* ws = (char*)base;
    uint32_t* Wm = (uint32_t*)(ws + L.off_w);
    DenseState* st = (DenseState*)(ws + L.off_state);
    uint32_t* cand = (uint32_t*)(ws + L.off_cand);
    uint32_t* panelU = (uint32_t*)(ws + L.off_panel);
    uint32_t* L11c = (uint32_t*)(ws + L.off_l11);
    int32_t* EtE = (int32_t*)(ws + L.off_ete);
    int32_t* EtT = (int32_t*)(ws + L.off_ett);
    int32_t* TL = (int32_t*)(ws + L.off_tl);
    int32_t* Ft = (int32_t*)(ws + L.off_ft);
    int32_t* Wt = (int32_t*)(ws + L.off_wt);
    int32_t* Up = (int32_t*)(ws + L.off_up);
    int32_t* R = (int32_t*)(ws + L.off_r);
    int32_t* L21t = (int32_t*)(ws + L.off_l21);
    int32_t* list_cur = (int32_t*)(ws + L.off_lista);
    int32_t* list_next = (int32_t*)(ws + L.off_listb);
    uint8_t* mark = (uint8_t*)(ws + L.off_mark);

    if ((s = ensure_dynamic_smem((const void*)panel_kernel, (int)psmem)) != LINAC_OK) return s;
    if ((s = ensure_dynamic_smem((const void*)lu_panel_kernel, (int)LU_SMEM)) != LINAC_OK) return s;
    int occ = 0;
    LINAC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, panel_kernel, PANEL_THREADS, psmem));
    if (occ < 1 || G > occ * sm_count()) return LINAC_ERR_UNSUPPORTED;

    {
        ProfScope ps(stream, PROF_INIT);
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((mn + 255) / 256, 1024));
        init_kernel<<<(unsigned)blocks, 256, 0, stream>>>(st, d_pivots, mn, d_rank);
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    if (m == 0) return LINAC_OK;
    {
        ProfScope ps(stream, PROF_LUP);
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 4096));
        lu_list_init_kernel<<<blocks, 256, 0, stream>>>(list_cur, list_next, mark, m);
        LINAC_CUDA_TRY(cudaGetLastError());
        if (n > 0) {
            LINAC_CUDA_TRY(cudaMemcpy2DAsync(Wm, (size_t)L.ldw * 4, dA, (size_t)ldA * 4, (size_t)n * 4, (size_t)m,
                                             cudaMemcpyDeviceToDevice, stream));
        }
    }
    const WaitLimit wl0 = wait_limit();
    for (int64_t c0 = 0; c0 < n; c0 += nb) {
        const int w = (int)std::min<int64_t>(nb, n - c0);
        const int64_t ncols = n - c0;
        {
            ProfScope ps(stream, PROF_PANEL);
            launch_window(Wm, m, L.ldw, (int)c0, w, f, st, panelU, G, list_cur, stream);
        }
        {
            const uint32_t* Mc = Wm;
            int64_t m_ = m, ld_ = L.ldw;
            int c0_ = (int)c0, w_ = w, S_ = S_max;
            Field f_ = f;
            WaitLimit wl = wl0;
            const int32_t* rowmap = list_cur;
            void* args[] = {(void*)&Mc, &m_, &ld_, &c0_, &w_, &S_, &f_, &st, &cand, &panelU, &status, &wl, &rowmap};
            ProfScope ps(stream, PROF_PANEL);
            LINAC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)panel_kernel, dim3(G), dim3(PANEL_THREADS), args,
                                                       psmem, stream));
        }
        {
            const unsigned gx = (unsigned)std::min<int64_t>((ncols + 1023) / 1024, 64);
            ProfScope ps(stream, PROF_GATHER_W);
            gather_w_kernel<<<dim3(std::max(1u, gx), NB_MAX), 256, 0, stream>>>(Wm, L.ldw, ncols, (int)c0, f, st, Wt,
                                                                                 L.ldW);
        }
        {
            ProfScope ps(stream, PROF_LUP);
            lu_panel_kernel<<<1, LU_THREADS, LU_SMEM, stream>>>(st, Wt, L.ldW, (int)c0, w, f, L11c, EtE, EtT, TL);
            LINAC_CUDA_TRY(cudaGetLastError());
        }
        if ((s = launch_gemm_assign(f, st, EtE, NB_MAX, Wt, L.ldW, ncols, Up, L.ldW, stream)) != LINAC_OK) return s;
        if ((s = launch_gemm_assign(f, st, EtT, NB_MAX, Up, L.ldW, ncols, R, L.ldW, stream)) != LINAC_OK) return s;
        {
            ProfScope ps(stream, PROF_LUP);
            lu_compact_kernel<<<1, 1024, 0, stream>>>(st, m, list_cur, list_next, mark);
            LINAC_CUDA_TRY(cudaGetLastError());
        }
        {
            ProfScope ps(stream, PROF_GATHER_F);
            gather_f_kernel<<<(unsigned)((m + 63) / 64), 256, 0, stream>>>(Wm, m, L.ldw, (int)c0, w, f, st, Ft, L.ldF,
                                                                           list_next);
        }
        if ((s = launch_gemm_assign(f, st, TL, NB_MAX, Ft, L.ldF, m, L21t, L.ldF, stream)) != LINAC_OK) return s;
        if ((s = launch_update_rows(Wm, m, n, L.ldw, (int)c0, f, st, Ft, L.ldF, R, L.ldW, list_next, stream)) !=
            LINAC_OK)
            return s;
        {
            ProfScope ps(stream, PROF_LUP);
            const unsigned rb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 1024));
            lu_writeback_kernel<<<NB_MAX + rb, 256, 0, stream>>>(Wm, m, L.ldw, ncols, (int)c0, f, st, Up, L.ldW, L11c,
                                                                 L21t, L.ldF, list_next);
            lu_perm_kernel<<<1, NB_MAX, 0, stream>>>(st, d_perm);
            LINAC_CUDA_TRY(cudaGetLastError());
        }
        {
            ProfScope ps(stream, PROF_FINISH);
            finish_kernel<<<1, NB_MAX, 0, stream>>>(st, d_pivots, d_rank);
            LINAC_CUDA_TRY(cudaGetLastError());
        }
        std::swap(list_cur, list_next);
    }
    {
        ProfScope ps(stream, PROF_LUP);
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 1024));
        lu_perm_tail_kernel<<<blocks, 256, 0, stream>>>(d_rank, m, list_cur, d_perm);
        lu_output_kernel<<<(unsigned)m, 256, 0, stream>>>(Wm, m, n, L.ldw, d_perm, d_rank, d_pivots, dL, ldL, dU, ldU);
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    return LINAC_OK;
}

}  // namespace linac
