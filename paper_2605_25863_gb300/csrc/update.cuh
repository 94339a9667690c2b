// update.cuh -- the trailing update C <- C - F * R (mod p) shared by the dense
// driver and its two arithmetic paths, plus the on-device elimination state.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "linac_device.cuh"

namespace linac {

constexpr int NB_MAX = 128;   // widest panel
constexpr int UPD_BM = 128;   // update tile rows
constexpr int UPD_BN = 128;   // update tile columns (limb path)
constexpr int UPD_BN2 = 64;   // update tile columns (plain path: two blocks per SM)
constexpr int UPD_BK = 16;    // update K chunk; panel widths are multiples of it

// Device-resident state of one dense elimination (lives in scratch memory).
struct DenseState {
    int32_t r;              // rank so far = first row of the current panel's pivots
    int32_t k;              // pivots found in the current panel
    int32_t win_ok;         // the current panel's pivots came from window_kernel (panel_kernel skips)
    int32_t pad1;
    GridBarrier bar;
    int32_t J[NB_MAX];      // pivot columns of the current panel (absolute)
    int32_t Pi[NB_MAX];     // pivot rows of the current panel (absolute, before the move)
    int32_t best[NB_MAX];   // per panel column: lowest candidate row (INT_MAX = none)
    uint32_t hinv[NB_MAX];  // inverses of the pivot heads
    uint32_t next_area;     // work counter of the hybrid update
    uint32_t pad2[3];
};

// Extra scratch used by the limb path (u8 limb planes of F and R).
struct LimbScratch {
    uint8_t* Fl;      // 4 planes x m_pad rows x kpad_max bytes (row-major, K contiguous)
    uint8_t* Rl;      // 4 planes x n_pad cols x kpad_max bytes (column-major, K contiguous)
    int64_t m_pad, n_pad;
};

// Extra scratch used by the multi-modular path (s8 residue planes of F and R
// for nine moduli; update_crt.cu).
struct CrtScratch {
    uint8_t* Fr;      // 9 planes x m_pad rows x 128 bytes
    uint8_t* Rr;      // 9 planes x n_pad columns x 128 bytes
    int64_t m_pad, n_pad;
};
size_t crt_scratch_bytes(int64_t m, int64_t n);
void crt_scratch_layout(void* base, int64_t m, int64_t n, CrtScratch* out);

// M[d, c0:n] <- M[d, c0:n] - F[d] R (rows d outside [r, r+k)) and
// M[r+t, c0:n] <- R[t] (t < k).  F is stored transposed (Ft: k x ldF, balanced
// int32), R row-major (k x ldR, balanced int32, columns relative to c0).
linac_status launch_update(int path, uint32_t* M, int64_t m, int64_t n, int64_t ld, int c0,
                           const Field& f, const DenseState* st, const int32_t* Ft, int64_t ldF,
                           const int32_t* R, int64_t ldR, const LimbScratch* limb,
                           const CrtScratch* crt, int* status, unsigned int* counter, cudaStream_t stream);

// M[rowmap[i], c0:n] <- M[rowmap[i], c0:n] - F[i] R for i < mrows (the LUP
// factorisation's trailing update of the rows that are not pivots yet; Ft is
// k x ldF with column i holding row rowmap[i]'s multipliers).
linac_status launch_update_rows(uint32_t* M, int64_t mrows, int64_t n, int64_t ld, int c0, const Field& f,
                                const DenseState* st, const int32_t* Ft, int64_t ldF, const int32_t* R,
                                int64_t ldR, const int32_t* rowmap, cudaStream_t stream);

// R[t][j] <- balanced(sum_s E[t][s] W[s][j]) for t < kpad(k), j < ncols, with
// Et = E transposed (kpad x ldE) and W (kpad x ldW), both balanced int32.
linac_status launch_gemm_assign(const Field& f, const DenseState* st, const int32_t* Et, int64_t ldE,
                                const int32_t* W, int64_t ldW, int64_t ncols, int32_t* R, int64_t ldR,
                                cudaStream_t stream);

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace linac
