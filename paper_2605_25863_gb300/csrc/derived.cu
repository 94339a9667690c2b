// derived.cu -- building systems on the device and reading results off an
// RREF (extern "C" entry points linac_load_matrix, linac_matmul,
// linac_null_space, linac_rank_factor).
//
//  load_matrix_kernel   A[r][c] = prod_t bases[r][lindices[c][t]] mod p: rows
//                       are sampling points, columns monomials (paper section
//                       3.3, "Building linear systems on GPUs"; section 2.3,
//                       cuda_load_matrix).  As in the paper each block stages
//                       its points' basis values in shared memory and every
//                       thread owns monomials; here a block owns 8 points so
//                       each monomial's indices are read once per 8 rows.
//                       The product runs in Montgomery form: d Montgomery
//                       multiplications give prod * R^(-d), and the running
//                       value starts at R^d mod p instead of 1, so the result
//                       is the plain product.
//  matmul_mod_kernel    C = A B mod p with lazy signed 64-bit accumulation of
//                       balanced residues (same arithmetic as the trailing
//                       update); expands a template of polynomial entries at
//                       many points (monomial values x coefficients) and
//                       states A = C R and A K = 0 on the device.
//  null space           the canonical kernel basis of section 5.1: one column
//                       per free (non-pivot) column f, -1 at f, R[t][f] at
//                       pivot column J[t], 0 elsewhere, so A K = 0.
//  rank factor          C = A[:, J], the pivot columns of the original matrix
//                       (section 5.1: A = C R).
#include <algorithm>
#include <climits>

#include "linac_host.h"
#include "profile.h"

namespace linac {

namespace {

constexpr int LM_THREADS = 256;
constexpr int LM_ROWS = 8;                  // points per block
constexpr int LM_SMEM_BASIS = 1536;         // basis values per point staged in shared memory

// Bounds-checked: an index outside [0, n_basis) yields 0 and sets the status
// word to LINAC_ERR_RANGE instead of reading out of bounds.
template <bool SMEM>
__global__ void __launch_bounds__(LM_THREADS)
load_matrix_kernel(const uint32_t* __restrict__ bases, int64_t n_rows, int n_basis, int64_t ldb,
                   const int32_t* __restrict__ lind, int64_t n_cols, int d, Field f, uint32_t rd,
                   uint32_t* __restrict__ A, int64_t lda, int* status) {
    // SMEM: n_basis x LM_ROWS, basis-major, so the 8 points' values of one
    // basis variable are two 16-byte words (rows beyond the last point are
    // zero and never stored)
    extern __shared__ __align__(16) uint32_t sb[];
    const int64_t r0 = (int64_t)blockIdx.y * LM_ROWS;
    const int nr = (int)(n_rows - r0 < LM_ROWS ? n_rows - r0 : LM_ROWS);
    if (SMEM) {
        for (int e = threadIdx.x; e < LM_ROWS * n_basis; e += LM_THREADS) {
            const int rr = e / n_basis, b = e - rr * n_basis;
            sb[b * LM_ROWS + rr] = rr < nr ? bases[(r0 + rr) * ldb + b] : 0u;
        }
        __syncthreads();
    }
    const int64_t c = (int64_t)blockIdx.x * LM_THREADS + threadIdx.x;
    if (c >= n_cols) return;
    uint32_t acc[LM_ROWS];
#pragma unroll
    for (int rr = 0; rr < LM_ROWS; ++rr) acc[rr] = rd;   // R^d mod p
    bool bad = false;
    for (int t = 0; t < d; ++t) {
        const int idx = lind[c * d + t];
        if (idx < 0 || idx >= n_basis) {
            bad = true;
            continue;
        }
        if (SMEM) {
            const uint4 lo = *reinterpret_cast<const uint4*>(sb + idx * LM_ROWS);
            const uint4 hi = *reinterpret_cast<const uint4*>(sb + idx * LM_ROWS + 4);
            const uint32_t v[LM_ROWS] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
            for (int rr = 0; rr < LM_ROWS; ++rr) acc[rr] = mont_mul(acc[rr], v[rr], f);
        } else {
#pragma unroll
            for (int rr = 0; rr < LM_ROWS; ++rr)
                if (rr < nr) acc[rr] = mont_mul(acc[rr], bases[(r0 + rr) * ldb + idx], f);
        }
    }
    if (bad) atomicCAS(status, 0, (int)LINAC_ERR_RANGE);
#pragma unroll
    for (int rr = 0; rr < LM_ROWS; ++rr)
        if (rr < nr) A[(r0 + rr) * lda + c] = bad ? 0u : acc[rr];
}

constexpr int MM_BM = 128, MM_BN = 64, MM_BK = 16;

// C = A B mod p.  128 x 64 output tile per 256-thread block, 8 x 4 outputs per
// thread; operands converted to balanced residues (|x| <= (p-1)/2) while they
// are staged, each product accumulated exactly with one signed 32 x 32 -> 64
// multiply-add, the accumulator folded (H*2^32 + L -> H*(2^32 mod p) + L)
// every FOLD products (on the ALU pipe when 2^32 mod p is sparse), one
// reduction per output at the end.
template <int FOLD, int SHIFTS>
__global__ void __launch_bounds__(256, 2)
matmul_mod_kernel(const uint32_t* __restrict__ A, int64_t m, int64_t K, int64_t lda, const uint32_t* __restrict__ B,
                  int64_t n, int64_t ldb, Field f, FoldShifts fs, uint32_t* __restrict__ C, int64_t ldc) {
    static_assert(MM_BK % FOLD == 0, "fold cadence must divide the K chunk");
    __shared__ __align__(16) int32_t As[MM_BK][MM_BM];
    __shared__ __align__(16) int32_t Bs[MM_BK][MM_BN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.y * MM_BM, col0 = (int64_t)blockIdx.x * MM_BN;
    int64_t acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    for (int64_t k0 = 0; k0 < K; k0 += MM_BK) {
        {
            const int r = tid >> 1, kb = (tid & 1) * 8;
            const int64_t row = row0 + r;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int64_t kk = k0 + kb + q;
                const uint32_t v = (row < m && kk < K) ? A[row * lda + kk] : 0u;
                As[kb + q][r] = to_balanced(v, f);
            }
        }
        {
            const int kk = tid >> 4, cb = (tid & 15) * 4;
            const int64_t k = k0 + kk;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t col = col0 + cb + q;
                const uint32_t v = (k < K && col < n) ? B[k * ldb + col] : 0u;
                Bs[kk][cb + q] = to_balanced(v, f);
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < MM_BK; ++kk) {
            const int4 a0 = *reinterpret_cast<const int4*>(&As[kk][ty * 4]);
            const int4 a1 = *reinterpret_cast<const int4*>(&As[kk][64 + ty * 4]);
            const int4 b0 = *reinterpret_cast<const int4*>(&Bs[kk][tx * 4]);
            const int a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const int b[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mac_s64(acc[i][j], a[i], b[j]);
            if ((kk + 1) % FOLD == 0) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fold_any<SHIFTS>(acc[i][j], f, fs);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t row = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (row >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t col = col0 + tx * 4 + j;
            if (col < n) C[row * ldc + col] = reduce_acc<SHIFTS>(acc[i][j], f, fs);
        }
    }
}

// pos[c] = t for pivot column c = J[t] (t < rank), -1 otherwise; free[q] =
// the q-th non-pivot column in increasing order, -1 after the nullity; one
// block, a running prefix count over chunks of the columns.
__global__ void __launch_bounds__(1024)
free_columns_kernel(const int32_t* __restrict__ rank_p, const int32_t* __restrict__ piv, int64_t n,
                    int64_t npiv_cap, int32_t* __restrict__ pos, int32_t* __restrict__ free_out,
                    int32_t* __restrict__ nullity_out, int64_t kcols, int* status) {
    __shared__ int warp_sums[32];
    __shared__ int s_base;
    const int rank = max(0, min(*rank_p, (int)(npiv_cap < n ? npiv_cap : n)));
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) pos[c] = -1;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < rank; t += blockDim.x) {
        const int c = piv[t];
        if (c >= 0 && c < n) pos[c] = t;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c0 = 0; c0 < n; c0 += blockDim.x) {
        const int64_t c = c0 + threadIdx.x;
        const int isfree = c < n && pos[c] < 0;
        const unsigned ball = __ballot_sync(0xffffffffu, isfree);
        const int before_in_warp = __popc(ball & ((1u << lane) - 1u));
        if (lane == 0) warp_sums[warp] = __popc(ball);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += warp_sums[w];
        const int q = s_base + before + before_in_warp;
        if (isfree) free_out[q] = (int32_t)c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += warp_sums[w];
            s_base += tot;
        }
        __syncthreads();
    }
    const int nullity = s_base;
    for (int64_t q = nullity + threadIdx.x; q < n; q += blockDim.x) free_out[q] = -1;
    if (threadIdx.x == 0) {
        *nullity_out = nullity;
        if (nullity > kcols) atomicCAS(status, 0, (int)LINAC_ERR_RANGE);
    }
}

// K[i][q] for q < kcols: -1 (= p - 1) at i = free[q], R[t][free[q]] at the
// pivot column i = J[t], 0 elsewhere and in columns q >= nullity.
template <typename T>
__global__ void null_space_kernel(const T* __restrict__ R, int64_t ldr, int64_t n, const int32_t* __restrict__ pos,
                                  const int32_t* __restrict__ free_c, const int32_t* __restrict__ nullity_p, T p,
                                  T* __restrict__ K, int64_t kcols, int64_t ldk, int64_t i0) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = i0 + blockIdx.y;
    if (q >= kcols) return;
    const int nullity = *nullity_p;
    T v = 0;
    if (q < nullity) {
        const int fc = free_c[q];
        if (i == fc) v = p - 1;
        else {
            const int t = pos[i];
            if (t >= 0) v = R[(int64_t)t * ldr + fc];
        }
    }
    K[i * ldk + q] = v;
}

// C[i][t] = A[i][J[t]] for t < rank, 0 for rank <= t < ccols.
template <typename T>
__global__ void rank_factor_kernel(const T* __restrict__ A, int64_t lda, int64_t n, const int32_t* __restrict__ rank_p,
                                   const int32_t* __restrict__ piv, int64_t npiv_cap, T* __restrict__ C,
                                   int64_t ccols, int64_t ldc, int64_t i0) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = i0 + blockIdx.y;
    if (t >= ccols) return;
    const int rank = max(0, min(*rank_p, (int)(npiv_cap < n ? npiv_cap : n)));
    T v = 0;
    if (t < rank) {
        const int c = piv[t];
        if (c >= 0 && c < n) v = A[i * lda + c];
    }
    C[i * ldc + t] = v;
}

int reset_status_word(cudaStream_t stream, int** out) {
    int* s = status_word(stream);
    if (!s) return LINAC_ERR_NOMEM;
    if (cudaMemsetAsync(s, 0, sizeof(int), stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return LINAC_ERR_CUDA;
    }
    *out = s;
    return LINAC_OK;
}

}  // namespace

linac_status launch_matmul(const uint32_t* A, int64_t m, int64_t K, int64_t lda, const uint32_t* B, int64_t n,
                           int64_t ldb, const Field& f, uint32_t* C, int64_t ldc, cudaStream_t stream) {
    if (m == 0 || n == 0) return LINAC_OK;
    const int64_t gy = (m + MM_BM - 1) / MM_BM, gx = (n + MM_BN - 1) / MM_BN;
    if (gy > 65535 || gx > INT_MAX) return LINAC_ERR_UNSUPPORTED;
    dim3 grid((unsigned)gx, (unsigned)gy);
    ProfScope ps(stream, PROF_MATMUL);
    FoldShifts fs;
    const int sh = fold_shifts(f, &fs);
#define LINAC_MM(FO, SH) matmul_mod_kernel<FO, SH><<<grid, 256, 0, stream>>>(A, m, K, lda, B, n, ldb, f, fs, C, ldc)
    if (f.fold >= 8) {
        switch (sh) {
            case 1: LINAC_MM(8, 1); break;
            case 2: LINAC_MM(8, 2); break;
            case 3: LINAC_MM(8, 3); break;
            default: LINAC_MM(8, 0); break;
        }
    } else {
        switch (sh) {
            case 1: LINAC_MM(4, 1); break;
            case 2: LINAC_MM(4, 2); break;
            case 3: LINAC_MM(4, 3); break;
            default: LINAC_MM(4, 0); break;
        }
    }
#undef LINAC_MM
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

}  // namespace linac

using namespace linac;

extern "C" {

linac_status linac_load_matrix(const uint32_t* d_bases, int64_t n_rows, int64_t n_basis, int64_t ld_bases,
                               const int32_t* d_lindices, int64_t n_cols, int32_t d, uint32_t p, uint32_t* d_A,
                               int64_t ldA, cudaStream_t stream) {
    if (n_rows < 0 || n_basis < 0 || n_cols < 0 || d < 0 || ld_bases < n_basis || ldA < n_cols) return LINAC_ERR_ARG;
    if (n_basis > INT_MAX || n_cols > INT32_MAX) return LINAC_ERR_ARG;
    if (n_rows > 0 && n_cols > 0 && (!d_A || (d > 0 && (!d_bases || !d_lindices)))) return LINAC_ERR_ARG;
    if (d > 0 && n_basis == 0 && n_rows > 0 && n_cols > 0) return LINAC_ERR_ARG;
    if (!prime_ok(p)) return LINAC_ERR_PRIME;
    const Field f = make_field(p);
    int* status = nullptr;
    linac_status s = (linac_status)reset_status_word(stream, &status);
    if (s != LINAC_OK) return s;
    if (n_rows == 0 || n_cols == 0) return LINAC_OK;
    // R^d mod p (R = 2^32 = c32 mod p): the start value that cancels the d
    // factors R^(-1) of the Montgomery products
    uint64_t rd = 1 % p;
    for (int t = 0; t < d; ++t) rd = rd * f.c32 % p;
    const int64_t gy = (n_rows + LM_ROWS - 1) / LM_ROWS;
    if (gy > 65535) return LINAC_ERR_UNSUPPORTED;
    dim3 grid((unsigned)((n_cols + LM_THREADS - 1) / LM_THREADS), (unsigned)gy);
    ProfScope ps(stream, PROF_LOAD_MATRIX);
    if (n_basis <= LM_SMEM_BASIS) {
        const size_t smem = (size_t)LM_ROWS * n_basis * 4;
        load_matrix_kernel<true><<<grid, LM_THREADS, smem, stream>>>(d_bases, n_rows, (int)n_basis, ld_bases, d_lindices,
                                                                     n_cols, d, f, (uint32_t)rd, d_A, ldA, status);
    } else {
        load_matrix_kernel<false><<<grid, LM_THREADS, 0, stream>>>(d_bases, n_rows, (int)n_basis, ld_bases, d_lindices,
                                                                   n_cols, d, f, (uint32_t)rd, d_A, ldA, status);
    }
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

linac_status linac_matmul(const uint32_t* d_A, int64_t m, int64_t K, int64_t ldA, const uint32_t* d_B, int64_t n,
                          int64_t ldB, uint32_t p, uint32_t* d_C, int64_t ldC, cudaStream_t stream) {
    if (m < 0 || K < 0 || n < 0 || ldA < K || ldB < n || ldC < n) return LINAC_ERR_ARG;
    if (m > 0 && n > 0 && (!d_C || (K > 0 && (!d_A || !d_B)))) return LINAC_ERR_ARG;
    if (!prime_ok(p)) return LINAC_ERR_PRIME;
    return launch_matmul(d_A, m, K, ldA, d_B, n, ldB, make_field(p), d_C, ldC, stream);
}

}  // extern "C"

namespace {

// Shared by the uint32 and uint64 entry points (the prime is checked there).
template <typename T>
linac_status null_space_impl(const T* d_R, int64_t m, int64_t n, int64_t ld, const int32_t* d_rank,
                             const int32_t* d_pivots, T p, T* d_K, int64_t kcols, int64_t ldK, int32_t* d_free,
                             int32_t* d_nullity, cudaStream_t stream) {
    int* status = nullptr;
    linac_status s = (linac_status)reset_status_word(stream, &status);
    if (s != LINAC_OK) return s;
    if (n == 0) {
        LINAC_CUDA_TRY(cudaMemsetAsync(d_nullity, 0, sizeof(int32_t), stream));
        return LINAC_OK;
    }
    void* buf = nullptr;
    if ((s = scratch_get_slot(stream, 4, (size_t)n * 4, &buf)) != LINAC_OK) return s;
    int32_t* pos = (int32_t*)buf;
    const int64_t npiv = std::min(m, n);
    {
        ProfScope ps(stream, PROF_DERIVED);
        free_columns_kernel<<<1, 1024, 0, stream>>>(d_rank, d_pivots, n, npiv, pos, d_free, d_nullity, kcols, status);
        LINAC_CUDA_TRY(cudaGetLastError());
        // one launch per 65535 rows of K (the grid's y limit)
        for (int64_t i0 = 0; kcols > 0 && i0 < n; i0 += 65535) {
            const int64_t rows = std::min<int64_t>(65535, n - i0);
            dim3 grid((unsigned)((kcols + 255) / 256), (unsigned)rows);
            null_space_kernel<T><<<grid, 256, 0, stream>>>(d_R, ld, n, pos, d_free, d_nullity, p, d_K, kcols, ldK, i0);
            LINAC_CUDA_TRY(cudaGetLastError());
        }
    }
    return LINAC_OK;
}

template <typename T>
linac_status rank_factor_impl(const T* d_A, int64_t m, int64_t n, int64_t ld, const int32_t* d_rank,
                              const int32_t* d_pivots, T* d_C, int64_t ccols, int64_t ldC, cudaStream_t stream) {
    if (m == 0 || ccols == 0) return LINAC_OK;
    ProfScope ps(stream, PROF_DERIVED);
    for (int64_t i0 = 0; i0 < m; i0 += 65535) {   // one launch per 65535 rows (the grid's y limit)
        const int64_t rows = std::min<int64_t>(65535, m - i0);
        dim3 grid((unsigned)((ccols + 255) / 256), (unsigned)rows);
        rank_factor_kernel<T><<<grid, 256, 0, stream>>>(d_A, ld, n, d_rank, d_pivots, std::min(m, n), d_C, ccols, ldC,
                                                        i0);
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    return LINAC_OK;
}

linac_status null_space_args(const void* d_R, int64_t m, int64_t n, int64_t ld, const int32_t* d_rank,
                             const int32_t* d_pivots, const void* d_K, int64_t kcols, int64_t ldK,
                             const int32_t* d_free, const int32_t* d_nullity) {
    if (m < 0 || n < 0 || ld < n || kcols < 0 || ldK < kcols || n > INT32_MAX) return LINAC_ERR_ARG;
    if (!d_rank || !d_nullity || (n > 0 && !d_free) || (n > 0 && kcols > 0 && !d_K)) return LINAC_ERR_ARG;
    if (m > 0 && n > 0 && (!d_R || !d_pivots)) return LINAC_ERR_ARG;
    return LINAC_OK;
}

linac_status rank_factor_args(const void* d_A, int64_t m, int64_t n, int64_t ld, const int32_t* d_rank,
                              const int32_t* d_pivots, const void* d_C, int64_t ccols, int64_t ldC) {
    if (m < 0 || n < 0 || ld < n || ccols < 0 || ldC < ccols) return LINAC_ERR_ARG;
    if (!d_rank || (m > 0 && ccols > 0 && (!d_C || !d_pivots || (n > 0 && !d_A)))) return LINAC_ERR_ARG;
    return LINAC_OK;
}

}  // namespace

extern "C" {

linac_status linac_null_space(const uint32_t* d_R, int64_t m, int64_t n, int64_t ld, const int32_t* d_rank,
                              const int32_t* d_pivots, uint32_t p, uint32_t* d_K, int64_t kcols, int64_t ldK,
                              int32_t* d_free, int32_t* d_nullity, cudaStream_t stream) {
    linac_status s = null_space_args(d_R, m, n, ld, d_rank, d_pivots, d_K, kcols, ldK, d_free, d_nullity);
    if (s != LINAC_OK) return s;
    if (!prime_ok(p)) return LINAC_ERR_PRIME;
    return null_space_impl<uint32_t>(d_R, m, n, ld, d_rank, d_pivots, p, d_K, kcols, ldK, d_free, d_nullity, stream);
}

linac_status linac_null_space64(const uint64_t* d_R, int64_t m, int64_t n, int64_t ld, const int32_t* d_rank,
                                const int32_t* d_pivots, uint64_t p, uint64_t* d_K, int64_t kcols, int64_t ldK,
                                int32_t* d_free, int32_t* d_nullity, cudaStream_t stream) {
    linac_status s = null_space_args(d_R, m, n, ld, d_rank, d_pivots, d_K, kcols, ldK, d_free, d_nullity);
    if (s != LINAC_OK) return s;
    if (!prime64_ok(p)) return LINAC_ERR_PRIME;
    return null_space_impl<uint64_t>(d_R, m, n, ld, d_rank, d_pivots, p, d_K, kcols, ldK, d_free, d_nullity, stream);
}

linac_status linac_rank_factor(const uint32_t* d_A, int64_t m, int64_t n, int64_t ld, const int32_t* d_rank,
                               const int32_t* d_pivots, uint32_t* d_C, int64_t ccols, int64_t ldC,
                               cudaStream_t stream) {
    linac_status s = rank_factor_args(d_A, m, n, ld, d_rank, d_pivots, d_C, ccols, ldC);
    if (s != LINAC_OK) return s;
    return rank_factor_impl<uint32_t>(d_A, m, n, ld, d_rank, d_pivots, d_C, ccols, ldC, stream);
}

linac_status linac_rank_factor64(const uint64_t* d_A, int64_t m, int64_t n, int64_t ld, const int32_t* d_rank,
                                 const int32_t* d_pivots, uint64_t* d_C, int64_t ccols, int64_t ldC,
                                 cudaStream_t stream) {
    linac_status s = rank_factor_args(d_A, m, n, ld, d_rank, d_pivots, d_C, ccols, ldC);
    if (s != LINAC_OK) return s;
    return rank_factor_impl<uint64_t>(d_A, m, n, ld, d_rank, d_pivots, d_C, ccols, ldC, stream);
}

}  // extern "C"
