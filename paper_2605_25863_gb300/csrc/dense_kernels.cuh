// dense_kernels.cuh -- declarations of the dense-elimination kernels defined
// in dense.cu, with the launch constants they were written for.
#pragma once
#include <cstdint>

#include "update.cuh"

namespace linac {

constexpr int PANEL_THREADS = 512;   // block size of panel_kernel
constexpr int WIN_EXTRA = 16;        // window rows beyond the panel width
constexpr int WIN_CTAS = 8;          // thread blocks of window_kernel's cluster
constexpr int WIN_THREADS = 256;     // threads per block of window_kernel
constexpr int WIN_ROWS_CTA = (NB_MAX + WIN_EXTRA + WIN_CTAS - 1) / WIN_CTAS;   // window rows per block
constexpr int EINV_COLS = 8;         // columns of E = G^{-1} per einv_kernel block
constexpr size_t EINV_SMEM = ((size_t)NB_MAX * (NB_MAX + 1) + (size_t)NB_MAX * EINV_COLS) * 4;

__global__ void init_kernel(DenseState* st, int32_t* d_pivots, int64_t npiv, int32_t* d_rank);
__global__ void finish_kernel(DenseState* st, int32_t* d_pivots, int32_t* d_rank);
__global__ void __cluster_dims__(WIN_CTAS, 1, 1) __launch_bounds__(WIN_THREADS)
window_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, Field f, DenseState* st,
              uint32_t* __restrict__ panelU, int G);
__global__ void __launch_bounds__(PANEL_THREADS)
panel_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, int S_max,
             Field f, DenseState* st, uint32_t* cand, uint32_t* panelU, int* status, WaitLimit wl);
__global__ void __launch_bounds__(256)
gather_f_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, Field f,
                const DenseState* __restrict__ st, int32_t* __restrict__ Ft, int64_t ldF);
__global__ void gather_w_kernel(const uint32_t* __restrict__ M, int64_t ld, int64_t ncols, int c0, Field f,
                                const DenseState* __restrict__ st, int32_t* __restrict__ W, int64_t ldW);
__global__ void heads_inverse_kernel(DenseState* st, const uint32_t* __restrict__ panelU, int c0,
                                     uint32_t p, int* status);
__global__ void __launch_bounds__(256)
einv_kernel(const DenseState* __restrict__ st, const uint32_t* __restrict__ panelU, int c0, Field f,
            int32_t* __restrict__ Et);
__global__ void __launch_bounds__(256)
move_kernel(uint32_t* __restrict__ M, int64_t ld, int64_t n, int c0, const DenseState* __restrict__ st,
            int32_t* __restrict__ Ft, int64_t ldF);

}  // namespace linac
