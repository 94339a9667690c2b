// update_limb.cu -- trailing update C <- C - F R (mod p) on the integer tensor
// pipe with four u8 limbs per residue.
//
// Every residue x < p < 2^31 is split as x = sum_{i<4} x_i 2^{8i} with bytes
// x_i (x_3 < 2^7).  Then
//     (F R)[a][b] = sum_{s=0..6} 2^{8s} P_s[a][b],  P_s = sum_{i+j=s} F_i R_j,
// where every F_i R_j is an exact u8 x u8 -> s32 matrix product on the tensor
// cores (mma.sync m16n8k32, the integer MMA that sm_103a provides; the
// tcgen05 kind::i8 form does not exist on this architecture).  Exactness: a
// u8 product is at most 255^2 = 65025 and at most 4 pairs share a shift, so
// P_s <= 4 * K * 65025 < 2^31 for K <= 8256; panels have K <= 128.  Each P_s
// is then weighted by w_s = 2^{8s} mod p and added to the output's running
// residue (P_s w_s + acc < 2^25 * 2^31 + 2^31, one Barrett reduction per
// shift).
//
// Data: per panel the limb planes Fl[l][row][t] (rows of F, K contiguous) and
// Rl[l][col][t] (columns of R, K contiguous) are written by the split
// kernels below.  A 512-thread block owns a 128 x 128 output tile, stages all
// K bytes of its four A and four B limb planes in shared memory (rows padded
// to 144 bytes so the fragment loads are conflict free), and each of its 16
// warps computes a 32 x 32 sub-tile as 2 x 4 m16n8 fragments.
#include <algorithm>

#include "linac_host.h"
#include "profile.h"
#include "update.cuh"

namespace linac {

constexpr int LIMB_BM = 128, LIMB_BN = 128, LIMB_KMAX = NB_MAX, LIMB_ROW = LIMB_KMAX + 16;
constexpr int LIMB_THREADS = 512;
constexpr size_t LIMB_SMEM = (size_t)2 * 4 * 128 * LIMB_ROW;

struct LimbWeights {
    uint32_t w[7];   // 2^(8s) mod p
};

// ---------------------------------------------------------------------------
// Limb planes

// Fl[l][row][t] = byte l of F[row][t] (canonical residue), t < kpad32, rows
// < m_pad (zero beyond m and beyond k).  F comes transposed and balanced.
__global__ void __launch_bounds__(256)
limb_split_f_kernel(const int32_t* __restrict__ Ft, int64_t ldF, int64_t m, const DenseState* __restrict__ st,
                    Field f, uint8_t* __restrict__ Fl, int64_t m_pad) {
    __shared__ uint32_t tile[LIMB_KMAX][65];
    const int k = st->k;
    if (k == 0) return;
    const int kp = (k + 31) / 32 * 32;
    const int64_t row0 = (int64_t)blockIdx.x * 64;
    for (int e = threadIdx.x; e < kp * 64; e += blockDim.x) {
        const int t = e >> 6, i = e & 63;
        const int64_t row = row0 + i;
        uint32_t v = 0;
        if (t < k && row < m) v = from_balanced(Ft[(int64_t)t * ldF + row], f);
        tile[t][i] = v;
    }
    __syncthreads();
    const int quads = kp / 4;
    for (int e = threadIdx.x; e < 64 * quads; e += blockDim.x) {
        const int i = e / quads, q = e % quads;
        const int64_t row = row0 + i;
        if (row >= m_pad) continue;
        const uint32_t x0 = tile[4 * q][i], x1 = tile[4 * q + 1][i], x2 = tile[4 * q + 2][i], x3 = tile[4 * q + 3][i];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const uint32_t sh = 8 * l;
            const uint32_t packed = ((x0 >> sh) & 255u) | (((x1 >> sh) & 255u) << 8) |
                                    (((x2 >> sh) & 255u) << 16) | (((x3 >> sh) & 255u) << 24);
            *reinterpret_cast<uint32_t*>(Fl + ((int64_t)l * m_pad + row) * LIMB_KMAX + 4 * q) = packed;
        }
    }
}

// Rl[l][col][t] = byte l of R[t][col] (canonical), cols < n_pad.
__global__ void __launch_bounds__(256)
limb_split_r_kernel(const int32_t* __restrict__ R, int64_t ldR, int64_t ncols, const DenseState* __restrict__ st,
                    Field f, uint8_t* __restrict__ Rl, int64_t n_pad) {
    __shared__ uint32_t tile[LIMB_KMAX][65];
    const int k = st->k;
    if (k == 0) return;
    const int kp = (k + 31) / 32 * 32;
    const int64_t col0 = (int64_t)blockIdx.x * 64;
    for (int e = threadIdx.x; e < kp * 64; e += blockDim.x) {
        const int t = e >> 6, i = e & 63;
        const int64_t col = col0 + i;
        uint32_t v = 0;
        if (t < k && col < ncols) v = from_balanced(R[(int64_t)t * ldR + col], f);
        tile[t][i] = v;
    }
    __syncthreads();
    const int quads = kp / 4;
    for (int e = threadIdx.x; e < 64 * quads; e += blockDim.x) {
        const int i = e / quads, q = e % quads;
        const int64_t col = col0 + i;
        if (col >= n_pad) continue;
        const uint32_t x0 = tile[4 * q][i], x1 = tile[4 * q + 1][i], x2 = tile[4 * q + 2][i], x3 = tile[4 * q + 3][i];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const uint32_t sh = 8 * l;
            const uint32_t packed = ((x0 >> sh) & 255u) | (((x1 >> sh) & 255u) << 8) |
                                    (((x2 >> sh) & 255u) << 16) | (((x3 >> sh) & 255u) << 24);
            *reinterpret_cast<uint32_t*>(Rl + ((int64_t)l * n_pad + col) * LIMB_KMAX + 4 * q) = packed;
        }
    }
}

// ---------------------------------------------------------------------------
// The tensor-core update

__device__ __forceinline__ void mma_u8(int (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(LIMB_THREADS, 1)
update_limb_kernel(uint32_t* __restrict__ M, int64_t m, int64_t n, int64_t ld, int c0, Field f,
                   const DenseState* __restrict__ st, const uint8_t* __restrict__ Fl,
                   const uint8_t* __restrict__ Rl, int64_t m_pad, int64_t n_pad,
                   const int32_t* __restrict__ R, int64_t ldR, LimbWeights wt) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t* As = smem;                               // [4][128][LIMB_ROW]
    uint8_t* Bs = smem + (size_t)4 * LIMB_BM * LIMB_ROW;   // [4][128][LIMB_ROW]
    const int k = st->k;
    if (k == 0) return;
    const int r = st->r;
    const int kp = (k + 31) / 32 * 32;
    const int64_t row0 = (int64_t)blockIdx.y * LIMB_BM;
    const int64_t col0 = (int64_t)blockIdx.x * LIMB_BN;
    const int64_t ncols = n - c0;
    const int tid = threadIdx.x;

    // stage the four A and four B limb planes (kp bytes per row / column)
    const int chunks = kp / 16;
    for (int e = tid; e < 4 * LIMB_BM * chunks; e += LIMB_THREADS) {
        const int l = e / (LIMB_BM * chunks), rem = e % (LIMB_BM * chunks);
        const int i = rem / chunks, c = rem % chunks;
        cp_async16(As + ((size_t)l * LIMB_BM + i) * LIMB_ROW + 16 * c,
                   Fl + ((int64_t)l * m_pad + row0 + i) * LIMB_KMAX + 16 * c, 16);
        cp_async16(Bs + ((size_t)l * LIMB_BN + i) * LIMB_ROW + 16 * c,
                   Rl + ((int64_t)l * n_pad + col0 + i) * LIMB_KMAX + 16 * c, 16);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    const int wm = warp & 3, wn = warp >> 2;          // 4 x 4 warps, 32 x 32 each
    const int g = lane >> 2, t4 = lane & 3;

    uint32_t acc[2][4][4];   // canonical residues; 32 registers leave room for P and fragments
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][b][q] = 0;

#pragma unroll 1
    for (int s = 0; s <= 6; ++s) {
        int P[2][4][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int q = 0; q < 4; ++q) P[a][b][q] = 0;
        const int ilo = s > 3 ? s - 3 : 0, ihi = s < 3 ? s : 3;
#pragma unroll 1
        for (int i = ilo; i <= ihi; ++i) {
            const int j = s - i;
            const uint8_t* Ai = As + (size_t)i * LIMB_BM * LIMB_ROW;
            const uint8_t* Bj = Bs + (size_t)j * LIMB_BN * LIMB_ROW;
#pragma unroll 1
            for (int kk = 0; kk < kp; kk += 32) {
                uint32_t af[2][4], bf[4][2];
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const uint8_t* base = Ai + (size_t)(wm * 32 + a * 16 + g) * LIMB_ROW + kk + 4 * t4;
                    af[a][0] = *reinterpret_cast<const uint32_t*>(base);
                    af[a][1] = *reinterpret_cast<const uint32_t*>(base + 8 * LIMB_ROW);
                    af[a][2] = *reinterpret_cast<const uint32_t*>(base + 16);
                    af[a][3] = *reinterpret_cast<const uint32_t*>(base + 8 * LIMB_ROW + 16);
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const uint8_t* base = Bj + (size_t)(wn * 32 + b * 8 + g) * LIMB_ROW + kk + 4 * t4;
                    bf[b][0] = *reinterpret_cast<const uint32_t*>(base);
                    bf[b][1] = *reinterpret_cast<const uint32_t*>(base + 16);
                }
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) mma_u8(P[a][b], af[a], bf[b]);
            }
        }
        uint32_t wsel = wt.w[0];
#pragma unroll
        for (int q = 1; q < 7; ++q)
            if (s == q) wsel = wt.w[q];
        const uint64_t w = wsel;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    acc[a][b][q] = reduce64((uint64_t)(uint32_t)P[a][b][q] * w + acc[a][b][q], f);
    }

#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int64_t row = row0 + wm * 32 + a * 16 + g + hh * 8;
            if (row >= m) continue;
            const bool pivot_row = row >= r && row < r + k;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int64_t col = col0 + wn * 32 + b * 8 + t4 * 2;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (col + q >= ncols) continue;
                    uint32_t* dst = M + row * ld + c0 + col + q;
                    if (pivot_row)
                        *dst = from_balanced(R[(int64_t)(row - r) * ldR + col + q], f);
                    else
                        *dst = submod(*dst, acc[a][b][hh * 2 + q], f);
                }
            }
        }
    }
}

linac_status launch_update_limb(uint32_t* M, int64_t m, int64_t n, int64_t ld, int c0, const Field& f,
                                const DenseState* st, const int32_t* Ft, int64_t ldF, const int32_t* R,
                                int64_t ldR, const LimbScratch* limb, cudaStream_t stream) {
    if (!limb) return LINAC_ERR_ARG;
    const int64_t ncols = n - c0;
    if (ncols <= 0 || m <= 0) return LINAC_OK;
    LimbWeights wt;
    uint64_t w = 1 % f.p;
    for (int s = 0; s < 7; ++s) {
        wt.w[s] = (uint32_t)w;
        w = (w << 8) % f.p;
    }
    {
        ProfScope ps(stream, PROF_LIMB_SPLIT);
        limb_split_f_kernel<<<(unsigned)(limb->m_pad / 64), 256, 0, stream>>>(Ft, ldF, m, st, f, limb->Fl,
                                                                               limb->m_pad);
        limb_split_r_kernel<<<(unsigned)((ncols + 127) / 128 * 2), 256, 0, stream>>>(R, ldR, ncols, st, f,
                                                                                      limb->Rl, limb->n_pad);
    }
    linac_status as = ensure_dynamic_smem((const void*)update_limb_kernel, (int)LIMB_SMEM);
    if (as != LINAC_OK) return as;
    dim3 grid((unsigned)((ncols + LIMB_BN - 1) / LIMB_BN), (unsigned)((m + LIMB_BM - 1) / LIMB_BM));
    {
        ProfScope ps(stream, PROF_UPDATE_LIMB);
        update_limb_kernel<<<grid, LIMB_THREADS, LIMB_SMEM, stream>>>(M, m, n, ld, c0, f, st, limb->Fl, limb->Rl,
                                                                      limb->m_pad, limb->n_pad, R, ldR, wt);
    }
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

}  // namespace linac
