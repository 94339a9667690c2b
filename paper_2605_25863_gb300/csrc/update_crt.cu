// update_crt.cu -- trailing update C <- C - F R (mod p) on the integer tensor
// pipe by multi-modular (residue number system) arithmetic.
//
// F (m x k) and R (k x N) hold balanced residues, |x| <= h = (p - 1)/2, so the
// exact integer product D = F R satisfies |D| <= k h^2 < 2^67 for k <= 128
// and p < 2^31.  Nine pairwise coprime moduli m_i <= 256 (CRT_MODULI below)
// have product M > 2^71.4 > 2 * 2^67, so D is fixed by its residues D mod m_i
// (Chinese remainder theorem) and recovered exactly:
//
//   1. Split (per panel): F_i = F mod m_i and R'_i = (R mod m_i) y_i mod m_i,
//      both balanced, |x| <= 128, stored as s8; y_i = (M/m_i)^(-1) mod m_i.
//   2. For each i, D'_i = F_i R'_i on mma.sync m16n8k32 s8 x s8 -> s32 (the
//      integer MMA of sm_103a; tcgen05 kind::i8 does not exist there).
//      Exact: |D'_i| <= k * 128^2 <= 2^21.
//   3. D'_i = D y_i (mod m_i) and y_i (M/m_i) = 1 (mod m_i), so
//      sum_i D'_i (M/m_i) = D (mod M), and D = sum_i D'_i (M/m_i) - beta M
//      for the integer beta that puts D in (-M/2, M/2).  Since |D|/M < 2^-4.4,
//      beta is the integer nearest to sum_i D'_i / m_i (|beta| < 2^17).  It is
//      found in fixed point: S = sum_i D'_i floor(2^38 / m_i) differs from
//      2^38 sum_i D'_i / m_i by less than sum_i |D'_i| <= 9 * 2^21 < 2^25,
//      and 2^38 |D|/M < 2^34, so beta = floor((S + 2^37) / 2^38) exactly.
//      No residue is reduced on the way: per modulus and output the step is
//      two signed 32 x 32 -> 64 multiply-adds (S and X below).
//   4. D mod p = (X + beta ((-M) mod p)) mod p with X = sum_i D'_i
//      ((M/m_i) mod p), all exact in signed 64 bits (|X| < 2^56,
//      |beta ((-M) mod p)| < 2^48) and reduced once.
// No floating point anywhere.
//
// Data: per panel the split kernels write the residue planes Fr[i][row][.]
// (the k <= 128 residues of one row of F, 128 bytes) and Rr[i][col][.] (one
// column of R').  Within every 128-byte row the 16-byte chunk c is stored at
// chunk c ^ (row & 7), so a 64-row tile copied contiguously into shared
// memory is already swizzled and the fragment loads are free of bank
// conflicts.  Update: one 256-thread block per 64 x 64 output tile, two
// blocks per SM; the tile's nine (A_i, B_i) pairs (8 KB + 8 KB each) stream
// through a three-stage ring of shared-memory buffers filled by bulk
// asynchronous copies (cp.async.bulk, the Blackwell TMA engine) that
// complete on mbarriers.  Each of the 8 warps computes 32 x 16 outputs, and
// issues the GEMM of modulus i + 1 before folding modulus i into S and X.
// (Measured and not kept: persistent blocks looping over tiles, and one
// packed 64-bit accumulator with a per-modulus reduction of D'_i; both were
// slower.)
#include <algorithm>

#include "linac_host.h"
#include "profile.h"
#include "update.cuh"
#include "update_tiles.cuh"

namespace linac {

namespace {
constexpr uint32_t CRT_MODULI[CRT_L] = {256, 255, 253, 251, 247, 241, 239, 233, 229};
constexpr int CRT_THREADS = 256;
}  // namespace

CrtConsts make_crt(uint32_t p) {
    CrtConsts c{};
    unsigned __int128 M = 1;
    for (int i = 0; i < CRT_L; ++i) M *= CRT_MODULI[i];
    for (int i = 0; i < CRT_L; ++i) {
        const uint32_t mi = CRT_MODULI[i];
        c.m[i] = mi;
        uint64_t Mi_mod = 1, Mi_p = 1;
        for (int j = 0; j < CRT_L; ++j)
            if (j != i) {
                Mi_mod = Mi_mod * CRT_MODULI[j] % mi;
                Mi_p = Mi_p * CRT_MODULI[j] % p;
            }
        uint32_t y = 0;
        for (uint32_t t = 1; t < mi; ++t)
            if (Mi_mod * t % mi == 1) { y = t; break; }
        c.y[i] = y;
        c.off30[i] = (uint32_t)(((1ull << 30) + mi - 1) / mi * mi);
        c.mgf[i] = (uint32_t)((1ull << 32) / mi);
        c.mgc[i] = (uint32_t)(((1ull << 32) + mi - 1) / mi);
        c.c38[i] = (uint32_t)((1ull << 38) / mi);
        c.wp[i] = (uint32_t)Mi_p;
    }
    const uint64_t Mp = (uint64_t)(M % p);
    c.negMp = (uint32_t)((p - Mp) % p);
    return c;
}

// ---------------------------------------------------------------------------
// Residue planes

// Balanced residue of a balanced x (|x| <= 2^30) modulo m (m <= 256):
// u = x + off30 lies in [0, 2^31 + 256); the quotient estimate
// floor(u floor(2^32/m) / 2^32) is floor(u/m) or one less, so one conditional
// subtraction gives r = u mod m.
__device__ __forceinline__ uint32_t small_mod30(int32_t x, uint32_t m, uint32_t off30, uint32_t mgf) {
    const uint32_t u = (uint32_t)x + off30;   // exact: the true sum lies in [0, 2^32)
    uint32_t r = u - __umulhi(u, mgf) * m;
    if (r >= m) r -= m;
    return r;
}

// u mod m for u < 2^24: floor(u ceil(2^32/m) / 2^32) = floor(u/m) exactly
// (the rounding error u (ceil(2^32/m) m - 2^32) / (m 2^32) < u / 2^32 < 1/m).
__device__ __forceinline__ uint32_t small_mod24(uint32_t u, uint32_t m, uint32_t mgc) {
    return u - __umulhi(u, mgc) * m;
}

__device__ __forceinline__ int32_t small_balanced(uint32_t r, uint32_t m) {
    return r > (m - 1) / 2 ? (int32_t)r - (int32_t)m : (int32_t)r;
}

// Planes of a k x ncols operand T stored t-major (T[t][x], leading dimension
// ldT, balanced int32; rows t >= k read as zero): out[i][x][.] holds the 128
// residues T[0..127][x] mod m_i (times y_i when SCALE), balanced s8, chunk c
// of row x at chunk c ^ (x & 7).  One block per 64 values of x.
template <bool SCALE>
__global__ void __launch_bounds__(256)
crt_split_kernel(const int32_t* __restrict__ T, int64_t ldT, int64_t nx, const DenseState* __restrict__ st,
                 CrtConsts cc, uint8_t* __restrict__ out, int64_t x_pad) {
    __shared__ int32_t tile[CRT_KB][65];
    const int k = st->k;
    if (k == 0) return;
    const int64_t x0 = (int64_t)blockIdx.x * 64;
    for (int e = threadIdx.x; e < CRT_KB * 64; e += blockDim.x) {
        const int t = e >> 6, i = e & 63;
        const int64_t x = x0 + i;
        tile[t][i] = (t < k && x < nx) ? T[(int64_t)t * ldT + x] : 0;
    }
    __syncthreads();
    // item = (row i of the tile, stored chunk s): consecutive threads write
    // consecutive 16-byte chunks of one plane
    for (int item = threadIdx.x; item < 64 * 8; item += blockDim.x) {
        const int i = item >> 3, s = item & 7;
        const int c = s ^ (i & 7);            // logical chunk: residues of t = 16c .. 16c + 15
        int32_t v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = tile[16 * c + j][i];
#pragma unroll 1
        for (int q = 0; q < CRT_L; ++q) {
            const uint32_t mq = cc.m[q];
            uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                uint32_t r = small_mod30(v[j], mq, cc.off30[q], cc.mgf[q]);
                if (SCALE) r = small_mod24(r * cc.y[q], mq, cc.mgc[q]);
                w[j >> 2] |= ((uint32_t)small_balanced(r, mq) & 255u) << (8 * (j & 3));
            }
            *reinterpret_cast<uint4*>(out + ((int64_t)q * x_pad + x0 + i) * CRT_KB + 16 * s) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// ---------------------------------------------------------------------------
// The tensor-core update: one 64 x 64 output tile (crt_tile in
// update_tiles.cuh) per 256-thread block, two blocks per SM.

__global__ void __launch_bounds__(CRT_THREADS, 2)
update_crt_kernel(uint32_t* __restrict__ M, int64_t m, int64_t n, int64_t ld, int c0, Field f,
                  const DenseState* __restrict__ st, const uint8_t* __restrict__ Fr,
                  const uint8_t* __restrict__ Rr, int64_t m_pad, int64_t n_pad,
                  const int32_t* __restrict__ R, int64_t ldR, CrtConsts cc, int* status, long long spin) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int k = st->k;
    if (k == 0) return;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t bar0 = sbase + CRT_STAGES * CRT_STAGE_BYTES;
    if (threadIdx.x == 0) {
        for (int s = 0; s < CRT_STAGES; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    (void)crt_tile(M, m, n, ld, c0, f, k, st->r, Fr, Rr, m_pad, n_pad, R, ldR, cc, status, spin,
                   (int64_t)blockIdx.y * CRT_BM, (int64_t)blockIdx.x * CRT_BN, 0, (int)threadIdx.x, smem, sbase, bar0,
                   BlockBarrier{});
}

// The residue planes of F (m rows) and R' (ncols columns) for one panel.
linac_status launch_crt_split(const int32_t* Ft, int64_t ldF, int64_t m, const int32_t* R, int64_t ldR,
                              int64_t ncols, const DenseState* st, const CrtConsts& cc, const CrtScratch* crt,
                              cudaStream_t stream) {
    ProfScope ps(stream, PROF_CRT_SPLIT);
    crt_split_kernel<false><<<(unsigned)(crt->m_pad / 64), 256, 0, stream>>>(Ft, ldF, m, st, cc, crt->Fr, crt->m_pad);
    crt_split_kernel<true><<<(unsigned)((ncols + 63) / 64), 256, 0, stream>>>(R, ldR, ncols, st, cc, crt->Rr,
                                                                             crt->n_pad);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

linac_status launch_update_crt(uint32_t* M, int64_t m, int64_t n, int64_t ld, int c0, const Field& f,
                               const DenseState* st, const int32_t* Ft, int64_t ldF, const int32_t* R,
                               int64_t ldR, const CrtScratch* crt, int* status, cudaStream_t stream) {
    if (!crt) return LINAC_ERR_ARG;
    const int64_t ncols = n - c0;
    if (ncols <= 0 || m <= 0) return LINAC_OK;
    const CrtConsts cc = make_crt(f.p);
    linac_status as = launch_crt_split(Ft, ldF, m, R, ldR, ncols, st, cc, crt, stream);
    if (as != LINAC_OK) return as;
    as = ensure_dynamic_smem((const void*)update_crt_kernel, (int)CRT_SMEM);
    if (as != LINAC_OK) return as;
    dim3 grid((unsigned)((ncols + CRT_BN - 1) / CRT_BN), (unsigned)((m + CRT_BM - 1) / CRT_BM));
    {
        ProfScope ps(stream, PROF_UPDATE_CRT);
        update_crt_kernel<<<grid, CRT_THREADS, CRT_SMEM, stream>>>(M, m, n, ld, c0, f, st, crt->Fr, crt->Rr,
                                                                   crt->m_pad, crt->n_pad, R, ldR, cc, status,
                                                                   wait_limit().spin_cycles);
    }
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

size_t crt_scratch_bytes(int64_t m, int64_t n) {
    const int64_t m_pad = (std::max<int64_t>(m, 1) + CRT_BM - 1) / CRT_BM * CRT_BM;
    const int64_t n_pad = (std::max<int64_t>(n, 1) + CRT_BN - 1) / CRT_BN * CRT_BN;
    return (size_t)CRT_L * (size_t)(m_pad + n_pad) * CRT_KB;
}

void crt_scratch_layout(void* base, int64_t m, int64_t n, CrtScratch* out) {
    out->m_pad = (std::max<int64_t>(m, 1) + CRT_BM - 1) / CRT_BM * CRT_BM;
    out->n_pad = (std::max<int64_t>(n, 1) + CRT_BN - 1) / CRT_BN * CRT_BN;
    out->Fr = (uint8_t*)base;
    out->Rr = (uint8_t*)base + (size_t)CRT_L * out->m_pad * CRT_KB;
}

}  // namespace linac
