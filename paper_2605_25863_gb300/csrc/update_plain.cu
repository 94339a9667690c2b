// update_plain.cu -- trailing update on the CUDA cores (the paper's "Row
// reduce" of section 3.2, blocked to rank k): C <- C - F R mod p.
//
// Arithmetic: F and R hold balanced residues |x| <= (p-1)/2, so every product
// satisfies |x y| <= ((p-1)/2)^2 < 2^60.  Each output accumulates its products
// exactly in a signed 64-bit register (one IMAD.WIDE per field multiply-add);
// after every FOLD products the accumulator H*2^32 + L is folded to
// H*(2^32 mod p) + L, which keeps |acc| < 2^62 + 2^32 so that FOLD more
// products stay below 2^63 (the host derives FOLD >= 4 from p; FOLD = 8 for
// the pseudo-Mersenne primes 2^31 - 1 and 2^31 - 19).  One reduction per
// output and panel finishes the job: two more folds and conditional
// subtractions when 2^32 mod p is sparse (reduce_alu), Barrett otherwise.
// No floating point anywhere.
#include <algorithm>

#include "linac_host.h"
#include "profile.h"
#include "update.cuh"

namespace linac {

// MODE 0: trailing update of M (rows [r, r+k) receive R).  MODE 1: plain
// product written as balanced residues to Out (k_pad x ldOut); M, m, c0 unused
// except that m bounds the A rows read.  MODE 2: trailing update of the rows
// rowmap[0..m) of M (the rows of the LUP factorisation that are not pivots
// yet); A row i is the multiplier row of M's row rowmap[i].
//
// Tiling: 128 x 64 outputs per 256-thread block, 8 x 4 per thread (two 4-row
// groups, one 4-column group), 128 registers so two blocks share an SM; K in
// chunks of 16 staged by cp.async double buffering.  The products occupy the
// integer multiply pipe (one mad.wide.s32 each, about four pipe cycles per
// warp instruction on this GPU), which bounds the kernel.
template <int FOLD, int SHIFTS, int MODE>
__global__ void __launch_bounds__(256, 2)
update_plain_kernel(uint32_t* __restrict__ M, int64_t m, int64_t n, int64_t ld, int c0, Field f,
                    FoldShifts fs, const DenseState* __restrict__ st, const int32_t* __restrict__ Ft,
                    int64_t ldF, const int32_t* __restrict__ R, int64_t ldR, int32_t* __restrict__ Out,
                    int64_t ldOut, const int32_t* __restrict__ rowmap) {
    static_assert(UPD_BK % FOLD == 0, "fold cadence must divide the K chunk");
    __shared__ __align__(16) int32_t As[2][UPD_BK][UPD_BM];
    __shared__ __align__(16) int32_t Bs[2][UPD_BK][UPD_BN2];
    const int k = st->k;
    if (k == 0) return;
    const int r = st->r;
    const int kpad = (k + UPD_BK - 1) / UPD_BK * UPD_BK;
    const int64_t row0 = (int64_t)blockIdx.y * UPD_BM;
    if (MODE == 2) {   // the rows left after this panel's pivots
        m = min(m, (int64_t)(m - r - k));
        if (row0 >= m) return;
    }
    const int64_t col0 = (int64_t)blockIdx.x * UPD_BN2;   // relative to c0
    const int64_t ncols = n - c0;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

    auto load = [&](int stage, int k0) {
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const int c = tid + it * 256;
            const int kk = c >> 5, x4 = (c & 31) * 4;
            const int64_t row = row0 + x4;
            const int bytes = row + 4 <= m ? 16 : (row < m ? (int)(m - row) * 4 : 0);
            const int32_t* src = bytes ? Ft + (int64_t)(k0 + kk) * ldF + row : Ft;
            cp_async16(&As[stage][kk][x4], src, bytes);
        }
        {
            const int kk = tid >> 4, x4 = (tid & 15) * 4;
            const int64_t col = col0 + x4;
            const int bytes = col + 4 <= ncols ? 16 : (col < ncols ? (int)(ncols - col) * 4 : 0);
            const int32_t* src = bytes ? R + (int64_t)(k0 + kk) * ldR + col : R;
            cp_async16(&Bs[stage][kk][x4], src, bytes);
        }
        cp_async_commit();
    };

    int64_t acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;

    const int nk = kpad / UPD_BK;
    load(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        if (kt + 1 < nk) {
            load((kt + 1) & 1, (kt + 1) * UPD_BK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int s = kt & 1;
#pragma unroll
        for (int kk = 0; kk < UPD_BK; ++kk) {
            const int4 a0 = *reinterpret_cast<const int4*>(&As[s][kk][ty * 4]);
            const int4 a1 = *reinterpret_cast<const int4*>(&As[s][kk][64 + ty * 4]);
            const int4 b0 = *reinterpret_cast<const int4*>(&Bs[s][kk][tx * 4]);
            const int a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const int b[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += (int64_t)a[i] * (int64_t)b[j];
            if ((kk + 1) % FOLD == 0) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fold_any<SHIFTS>(acc[i][j], f, fs);
            }
        }
        __syncthreads();
    }

    if (MODE == 1) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t row = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (row >= kpad) continue;
            const int64_t col = col0 + tx * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (col + q < ncols) Out[row * ldOut + col + q] = to_balanced(reduce_acc<SHIFTS>(acc[i][q], f, fs), f);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t row = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (row >= m) continue;
        const bool pivot_row = MODE == 0 && row >= r && row < r + k;
        const int64_t col = col0 + tx * 4;
        if (col >= ncols) continue;
        uint32_t* dst = M + (MODE == 2 ? (int64_t)rowmap[row] : row) * ld + c0 + col;
        uint32_t out[4];
        if (pivot_row) {
            const int32_t* rr = R + (int64_t)(row - r) * ldR + col;
#pragma unroll
            for (int q = 0; q < 4; ++q) out[q] = col + q < ncols ? from_balanced(rr[q], f) : 0u;
        } else if (col + 4 <= ncols) {
            const uint4 cv = *reinterpret_cast<const uint4*>(dst);
            const uint32_t c4[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) out[q] = submod(c4[q], reduce_acc<SHIFTS>(acc[i][q], f, fs), f);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                out[q] = col + q < ncols ? submod(dst[q], reduce_acc<SHIFTS>(acc[i][q], f, fs), f) : 0u;
        }
        if (col + 4 <= ncols) {
            *reinterpret_cast<uint4*>(dst) = make_uint4(out[0], out[1], out[2], out[3]);
        } else {
            for (int q = 0; q < 4 && col + q < ncols; ++q) dst[q] = out[q];
        }
    }
}

namespace {
template <int MODE>
void launch_plain(dim3 grid, cudaStream_t stream, uint32_t* M, int64_t m, int64_t n, int64_t ld, int c0,
                  const Field& f, const DenseState* st, const int32_t* Ft, int64_t ldF, const int32_t* R,
                  int64_t ldR, int32_t* Out, int64_t ldOut, const int32_t* rowmap = nullptr) {
    FoldShifts fs;
    const int sh = fold_shifts(f, &fs);
    const int fold = f.fold >= 16 ? 16 : (f.fold >= 8 ? 8 : 4);
#define LINAC_UPD(FO, SH) \
    update_plain_kernel<FO, SH, MODE><<<grid, 256, 0, stream>>>(M, m, n, ld, c0, f, fs, st, Ft, ldF, R, ldR, Out, ldOut, \
                                                                 rowmap)
#define LINAC_UPD_SH(FO)                    \
    switch (sh) {                           \
        case 1: LINAC_UPD(FO, 1); break;    \
        case 2: LINAC_UPD(FO, 2); break;    \
        case 3: LINAC_UPD(FO, 3); break;    \
        default: LINAC_UPD(FO, 0); break;   \
    }
    if (fold == 16) { LINAC_UPD_SH(16) }
    else if (fold == 8) { LINAC_UPD_SH(8) }
    else { LINAC_UPD_SH(4) }
#undef LINAC_UPD_SH
#undef LINAC_UPD
}
}  // namespace

linac_status launch_update_rows(uint32_t* M, int64_t mrows, int64_t n, int64_t ld, int c0, const Field& f,
                                const DenseState* st, const int32_t* Ft, int64_t ldF, const int32_t* R,
                                int64_t ldR, const int32_t* rowmap, cudaStream_t stream) {
    const int64_t ncols = n - c0;
    if (ncols <= 0 || mrows <= 0) return LINAC_OK;
    if ((mrows + UPD_BM - 1) / UPD_BM > 65535) return LINAC_ERR_UNSUPPORTED;
    dim3 grid((unsigned)((ncols + UPD_BN2 - 1) / UPD_BN2), (unsigned)((mrows + UPD_BM - 1) / UPD_BM));
    ProfScope ps(stream, PROF_UPDATE_PLAIN);
    launch_plain<2>(grid, stream, M, mrows, n, ld, c0, f, st, Ft, ldF, R, ldR, nullptr, 0, rowmap);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

linac_status launch_update_limb(uint32_t* M, int64_t m, int64_t n, int64_t ld, int c0, const Field& f,
                                const DenseState* st, const int32_t* Ft, int64_t ldF, const int32_t* R,
                                int64_t ldR, const LimbScratch* limb, cudaStream_t stream);

linac_status launch_update_crt(uint32_t* M, int64_t m, int64_t n, int64_t ld, int c0, const Field& f,
                               const DenseState* st, const int32_t* Ft, int64_t ldF, const int32_t* R,
                               int64_t ldR, const CrtScratch* crt, int* status, cudaStream_t stream);

linac_status launch_update(int path, uint32_t* M, int64_t m, int64_t n, int64_t ld, int c0,
                           const Field& f, const DenseState* st, const int32_t* Ft, int64_t ldF,
                           const int32_t* R, int64_t ldR, const LimbScratch* limb,
                           const CrtScratch* crt, int* status, cudaStream_t stream) {
    if (path == LINAC_PATH_LIMB)
        return launch_update_limb(M, m, n, ld, c0, f, st, Ft, ldF, R, ldR, limb, stream);
    if (path == LINAC_PATH_CRT)
        return launch_update_crt(M, m, n, ld, c0, f, st, Ft, ldF, R, ldR, crt, status, stream);
    const int64_t ncols = n - c0;
    if (ncols <= 0 || m <= 0) return LINAC_OK;
    dim3 grid((unsigned)((ncols + UPD_BN2 - 1) / UPD_BN2), (unsigned)((m + UPD_BM - 1) / UPD_BM));
    ProfScope ps(stream, PROF_UPDATE_PLAIN);
    launch_plain<0>(grid, stream, M, m, n, ld, c0, f, st, Ft, ldF, R, ldR, nullptr, 0);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

linac_status launch_gemm_assign(const Field& f, const DenseState* st, const int32_t* Et, int64_t ldE,
                                const int32_t* W, int64_t ldW, int64_t ncols, int32_t* R, int64_t ldR,
                                cudaStream_t stream) {
    if (ncols <= 0) return LINAC_OK;
    dim3 grid((unsigned)((ncols + UPD_BN2 - 1) / UPD_BN2), 1);
    ProfScope ps(stream, PROF_TRSM);
    // A rows are the NB_MAX columns of Et (zero beyond k); K runs to kpad(k)
    launch_plain<1>(grid, stream, nullptr, NB_MAX, ncols, 0, 0, f, st, Et, ldE, W, ldW, R, ldR);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

}  // namespace linac
