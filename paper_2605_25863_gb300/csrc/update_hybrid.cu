// update_hybrid.cu -- trailing update C <- C - F R (mod p) on the CUDA cores
// and the integer tensor pipe at the same time (LINAC_PATH_HYBRID).
//
// The plain update keeps the integer multiply pipe busy and leaves the tensor
// pipe idle; the multi-modular update does the opposite (update_crt.cu).  The
// two pipes overlap in part: one block whose first 8 warps issue mad.wide.s32
// and whose last 8 warps issue mma.sync did the work of both in 0.339 ms
// against 0.428 ms for the two one after the other (probes/int_rates.cu).
// This kernel runs both updates in one persistent block per SM:
//   warps 0-7   (group 0)  plain tiles, 128 x 64 outputs each (plain_tile);
//   warps 8-15  (group 1)  the same 128 x 64 output area as two 64 x 64
//                          multi-modular tiles (crt_tile).
// Each group takes the next 128 x 64 area from one atomic counter when it is
// free, so the split between the two adapts to their speeds on the device.
// Each group synchronises only itself, on its own named barrier (1 and 2);
// the plain group stages its operands with cp.async, the multi-modular group
// with bulk copies completing on its three mbarriers.  Both write their own
// rows only, so the result is the same as either standalone update.
#include <algorithm>

#include "linac_host.h"
#include "profile.h"
#include "update.cuh"
#include "update_tiles.cuh"

namespace linac {

CrtConsts make_crt(uint32_t p);
linac_status launch_crt_split(const int32_t* Ft, int64_t ldF, int64_t m, const int32_t* R, int64_t ldR,
                              int64_t ncols, const DenseState* st, const CrtConsts& cc, const CrtScratch* crt,
                              cudaStream_t stream);

namespace {

constexpr int HY_THREADS = 512;
constexpr int HY_GROUP = 256;
constexpr size_t HY_SMEM = CRT_SMEM;   // the multi-modular group's ring (plain_tile's arrays are static)

template <int FOLD, int SHIFTS>
__global__ void __launch_bounds__(HY_THREADS, 1)
update_hybrid_kernel(uint32_t* __restrict__ M, int64_t m, int64_t n, int64_t ld, int c0, Field f, FoldShifts fs,
                     const DenseState* __restrict__ st, const int32_t* __restrict__ Ft, int64_t ldF,
                     const int32_t* __restrict__ R, int64_t ldR, const uint8_t* __restrict__ Fr,
                     const uint8_t* __restrict__ Rr, int64_t m_pad, int64_t n_pad, CrtConsts cc, int* status,
                     long long spin, unsigned int* __restrict__ next_area) {
    __shared__ int s_area[2];
    extern __shared__ __align__(128) uint8_t smem[];
    const int k = st->k;
    if (k == 0) return;
    const int r = st->r;
    const int64_t ncols = n - c0;
    const int tiles_x = (int)((ncols + UPD_BN2 - 1) / UPD_BN2);
    const int areas = tiles_x * (int)((m + UPD_BM - 1) / UPD_BM);
    const int tid = threadIdx.x % HY_GROUP;
    // takes the next 128 x 64 output area for this group (-1: none left)
    auto next = [&](int group, const NamedBarrier& bar) -> int {
        if (tid == 0) s_area[group] = (int)atomicAdd(next_area, 1u);
        bar.sync();
        const int a = s_area[group];
        bar.sync();   // every thread has read s_area before it is written again
        return a < areas ? a : -1;
    };
    if (threadIdx.x < HY_GROUP) {
        const NamedBarrier bar{1, HY_GROUP};
        for (int a; (a = next(0, bar)) >= 0;) {
            const int64_t row0 = (int64_t)(a / tiles_x) * UPD_BM, col0 = (int64_t)(a % tiles_x) * UPD_BN2;
            plain_tile<FOLD, SHIFTS, 0>(M, m, n, ld, c0, f, fs, k, r, Ft, ldF, R, ldR, nullptr, 0, nullptr, row0,
                                        col0, tid, bar);
        }
    } else {
        const NamedBarrier bar{2, HY_GROUP};
        const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
        const uint32_t bar0 = sbase + CRT_STAGES * CRT_STAGE_BYTES;
        if (tid == 0) {
            for (int s = 0; s < CRT_STAGES; ++s) mbar_init(bar0 + 8 * s, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        int j0 = 0;   // the group's running load sequence
        bool ok = true;
        for (int a; ok && (a = next(1, bar)) >= 0;) {
            const int64_t row0 = (int64_t)(a / tiles_x) * UPD_BM, col0 = (int64_t)(a % tiles_x) * UPD_BN2;
#pragma unroll 1
            for (int64_t rh = row0; ok && rh < row0 + UPD_BM && rh < m; rh += CRT_BM) {
                ok = crt_tile(M, m, n, ld, c0, f, k, r, Fr, Rr, m_pad, n_pad, R, ldR, cc, status, spin, rh, col0, j0,
                              tid, smem, sbase, bar0, bar);
                j0 += CRT_L;
            }
        }
    }
}

}  // namespace

linac_status launch_update_hybrid(uint32_t* M, int64_t m, int64_t n, int64_t ld, int c0, const Field& f,
                                  const DenseState* st, const int32_t* Ft, int64_t ldF, const int32_t* R,
                                  int64_t ldR, const CrtScratch* crt, unsigned int* counter, int* status,
                                  cudaStream_t stream) {
    if (!crt || !counter) return LINAC_ERR_ARG;
    const int64_t ncols = n - c0;
    if (ncols <= 0 || m <= 0) return LINAC_OK;
    const int64_t areas = ((ncols + UPD_BN2 - 1) / UPD_BN2) * ((m + UPD_BM - 1) / UPD_BM);
    if (areas >= INT32_MAX) return LINAC_ERR_UNSUPPORTED;
    const CrtConsts cc = make_crt(f.p);
    linac_status s = launch_crt_split(Ft, ldF, m, R, ldR, ncols, st, cc, crt, stream);
    if (s != LINAC_OK) return s;
    LINAC_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned int), stream));
    FoldShifts fs;
    const int sh = fold_shifts(f, &fs);
    const int fold = f.fold >= 16 ? 16 : (f.fold >= 8 ? 8 : 4);
    const unsigned grid = (unsigned)std::min<int64_t>(areas, sm_count());
    const long long spin = wait_limit().spin_cycles;
    ProfScope ps(stream, PROF_UPDATE_HYBRID);
#define LINAC_HY(FO, SH)                                                                                           \
    do {                                                                                                           \
        if ((s = ensure_dynamic_smem((const void*)update_hybrid_kernel<FO, SH>, (int)HY_SMEM)) != LINAC_OK) return s; \
        update_hybrid_kernel<FO, SH><<<grid, HY_THREADS, HY_SMEM, stream>>>(M, m, n, ld, c0, f, fs, st, Ft, ldF, R,  \
                                                                           ldR, crt->Fr, crt->Rr, crt->m_pad,      \
                                                                           crt->n_pad, cc, status, spin, counter); \
    } while (0)
#define LINAC_HY_SH(FO)                  \
    switch (sh) {                        \
        case 1: LINAC_HY(FO, 1); break;  \
        case 2: LINAC_HY(FO, 2); break;  \
        case 3: LINAC_HY(FO, 3); break;  \
        default: LINAC_HY(FO, 0); break; \
    }
    if (fold == 16) { LINAC_HY_SH(16) }
    else if (fold == 8) { LINAC_HY_SH(8) }
    else { LINAC_HY_SH(4) }
#undef LINAC_HY_SH
#undef LINAC_HY
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

}  // namespace linac
