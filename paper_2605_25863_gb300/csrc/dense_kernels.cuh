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
constexpr int WIN1_NB = 64;          // widest panel of the one-block window
constexpr int WIN1_THREADS = 512;    // threads of window1_kernel
constexpr int EINV_COLS = 8;         // columns of E = G^{-1} per einv_kernel block
constexpr size_t EINV_SMEM = ((size_t)NB_MAX * (NB_MAX + 1) + (size_t)NB_MAX * EINV_COLS) * 4;

// Row maps.  The pivot search and the multiplier gather address the
// remaining rows by their position x in [0, m - r): the row is r + x when
// rowmap is null (the RREF keeps the remaining rows contiguous), rowmap[x]
// otherwise (the LUP factorisation keeps them in their original places and
// lists them in increasing order, so the lowest position is the lowest
// original row).  The gather addresses all rows the same way, with x from 0.
__device__ __forceinline__ int64_t map_row(const int32_t* rowmap, int64_t base, int64_t x) {
    return rowmap ? (int64_t)rowmap[x] : base + x;
}

// Blocks of the cooperative panel search for m rows, and its dynamic shared
// memory for slabs of S_max rows and panel width w.
int panel_grid(int64_t m);
size_t panel_smem(int S_max, int w);

__global__ void init_kernel(DenseState* st, int32_t* d_pivots, int64_t npiv, int32_t* d_rank);
__global__ void finish_kernel(DenseState* st, int32_t* d_pivots, int32_t* d_rank);
__global__ void __cluster_dims__(WIN_CTAS, 1, 1) __launch_bounds__(WIN_THREADS)
window_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, Field f, DenseState* st,
              uint32_t* __restrict__ panelU, int G, const int32_t* __restrict__ rowmap);
__global__ void __launch_bounds__(WIN1_THREADS)
window1_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, Field f, DenseState* st,
               uint32_t* __restrict__ panelU, int G, const int32_t* __restrict__ rowmap);

// Pivot window of a panel of w columns: the one-block kernel for w <= WIN1_NB,
// the 8-block cluster otherwise.
inline void launch_window(const uint32_t* M, int64_t m, int64_t ld, int c0, int w, const Field& f,
                          DenseState* st, uint32_t* panelU, int G, const int32_t* rowmap, cudaStream_t stream) {
    if (w <= WIN1_NB)
        window1_kernel<<<1, WIN1_THREADS, 0, stream>>>(M, m, ld, c0, w, f, st, panelU, G, rowmap);
    else
        window_kernel<<<WIN_CTAS, WIN_THREADS, 0, stream>>>(M, m, ld, c0, w, f, st, panelU, G, rowmap);
}

__global__ void __launch_bounds__(PANEL_THREADS)
panel_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, int S_max,
             Field f, DenseState* st, uint32_t* cand, uint32_t* panelU, int* status, WaitLimit wl,
             const int32_t* __restrict__ rowmap);
__global__ void __launch_bounds__(256)
gather_f_kernel(const uint32_t* __restrict__ M, int64_t m, int64_t ld, int c0, int w, Field f,
                const DenseState* __restrict__ st, int32_t* __restrict__ Ft, int64_t ldF,
                const int32_t* __restrict__ rowmap);
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
