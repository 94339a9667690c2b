// update_plain.cu -- trailing update on the CUDA cores (the paper's "Row
// reduce" of section 3.2, blocked to rank k): C <- C - F R mod p.
//
// Arithmetic (plain_tile, update_tiles.cuh): F and R hold balanced residues
// |x| <= (p-1)/2, every product is accumulated exactly in a signed 64-bit
// register, folded every FOLD products (the host derives FOLD >= 4 from p;
// FOLD = 8 for the pseudo-Mersenne primes 2^31 - 1 and 2^31 - 19) and
// reduced once per output and panel.  No floating point anywhere.
#include <algorithm>

#include "linac_host.h"
#include "profile.h"
#include "update.cuh"
#include "update_tiles.cuh"

namespace linac {

// Standalone plain update: one 128 x 64 output tile (plain_tile in
// update_tiles.cuh, MODE 0, 1 or 2) per 256-thread block.  8 x 4 outputs per
// thread, 128 registers so two blocks share an SM.  The products occupy the
// integer multiply pipe (one mad.wide.s32 each, about four pipe cycles per
// warp instruction on this GPU), which bounds the kernel.
template <int FOLD, int SHIFTS, int MODE>
__global__ void __launch_bounds__(256, 2)
update_plain_kernel(uint32_t* __restrict__ M, int64_t m, int64_t n, int64_t ld, int c0, Field f,
                    FoldShifts fs, const DenseState* __restrict__ st, const int32_t* __restrict__ Ft,
                    int64_t ldF, const int32_t* __restrict__ R, int64_t ldR, int32_t* __restrict__ Out,
                    int64_t ldOut, const int32_t* __restrict__ rowmap) {
    const int k = st->k;
    if (k == 0) return;
    const int r = st->r;
    const int64_t row0 = (int64_t)blockIdx.y * UPD_BM;
    if (MODE == 2) {   // the rows left after this panel's pivots
        m = min(m, (int64_t)(m - r - k));
        if (row0 >= m) return;
    }
    const int64_t col0 = (int64_t)blockIdx.x * UPD_BN2;   // relative to c0
    plain_tile<FOLD, SHIFTS, MODE>(M, m, n, ld, c0, f, fs, k, r, Ft, ldF, R, ldR, Out, ldOut, rowmap, row0, col0,
                                   (int)threadIdx.x, BlockBarrier{});
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

linac_status launch_update_hybrid(uint32_t* M, int64_t m, int64_t n, int64_t ld, int c0, const Field& f,
                                  const DenseState* st, const int32_t* Ft, int64_t ldF, const int32_t* R,
                                  int64_t ldR, const CrtScratch* crt, unsigned int* counter, int* status,
                                  cudaStream_t stream);

linac_status launch_update(int path, uint32_t* M, int64_t m, int64_t n, int64_t ld, int c0,
                           const Field& f, const DenseState* st, const int32_t* Ft, int64_t ldF,
                           const int32_t* R, int64_t ldR, const LimbScratch* limb,
                           const CrtScratch* crt, int* status, unsigned int* counter, cudaStream_t stream) {
    if (path == LINAC_PATH_HYBRID)
        return launch_update_hybrid(M, m, n, ld, c0, f, st, Ft, ldF, R, ldR, crt, counter, status, stream);
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
