// update_tiles.cuh -- the output-tile bodies of the trailing update
// C <- C - F R (mod p), shared by the standalone kernels (update_plain.cu,
// update_crt.cu) and the hybrid kernel (update_hybrid.cu) that runs both at
// once on different warps of one block.
//
// A tile body is executed by one group of 256 threads whose thread index is
// `tid`; it synchronises only that group, through the barrier object it is
// given: the whole block's barrier in the standalone kernels, a named hardware
// barrier in the hybrid kernel, whose two groups must not wait for each other.
#pragma once
#include <cstdint>

#include "update.cuh"

namespace linac {

// Barrier of a whole 256-thread block.
struct BlockBarrier {
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int sync_or(int pred) const { return __syncthreads_or(pred); }
};

// Named barrier `id` (1..15) of `count` threads (a multiple of 32).
struct NamedBarrier {
    int id, count;
    __device__ __forceinline__ void sync() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
    }
    __device__ __forceinline__ int sync_or(int pred) const {
        int out;
        asm volatile(
            "{\n\t.reg .pred p, q;\n\t"
            "setp.ne.s32 q, %1, 0;\n\t"
            "bar.red.or.pred p, %2, %3, q;\n\t"
            "selp.s32 %0, 1, 0, p;\n\t}"
            : "=r"(out)
            : "r"(pred), "r"(id), "r"(count)
            : "memory");
        return out;
    }
};

// ---------------------------------------------------------------------------
// Plain tile (CUDA cores): 128 x 64 outputs, 8 x 4 per thread.
//
// MODE 0: trailing update of M (rows [r, r+k) receive R).  MODE 1: plain
// product written as balanced residues to Out (k_pad x ldOut); M, m, c0 unused
// except that m bounds the A rows read.  MODE 2: trailing update of the rows
// rowmap[0..m) of M; A row i is the multiplier row of M's row rowmap[i].
//
// F and R hold balanced residues |x| <= (p-1)/2, so every product satisfies
// |x y| <= ((p-1)/2)^2 < 2^60.  Each output accumulates its products exactly
// in a signed 64-bit register (one mad.wide.s32 per field multiply-add); after
// every FOLD products the accumulator H*2^32 + L is folded to
// H*(2^32 mod p) + L, which keeps |acc| < 2^62 + 2^32 so that FOLD more
// products stay below 2^63.  One reduction per output and panel finishes:
// two more folds and conditional subtractions when 2^32 mod p is sparse
// (reduce_alu), Barrett otherwise.  K in chunks of 16 staged by cp.async
// double buffering in the function's own shared arrays As (2 x 16 x 128) and
// Bs (2 x 16 x 64).  (Three stages with one barrier per chunk were measured
// and were no faster, alone or beside the multi-modular warps.)
template <int FOLD, int SHIFTS, int MODE, class Bar>
__device__ __forceinline__ void plain_tile(uint32_t* __restrict__ M, int64_t m, int64_t n, int64_t ld, int c0,
                                           const Field& f, const FoldShifts& fs, int k, int r,
                                           const int32_t* __restrict__ Ft, int64_t ldF,
                                           const int32_t* __restrict__ R, int64_t ldR, int32_t* __restrict__ Out,
                                           int64_t ldOut, const int32_t* __restrict__ rowmap, int64_t row0,
                                           int64_t col0, int tid, Bar bar) {
    static_assert(UPD_BK % FOLD == 0, "fold cadence must divide the K chunk");
    __shared__ __align__(16) int32_t As[2][UPD_BK][UPD_BM];
    __shared__ __align__(16) int32_t Bs[2][UPD_BK][UPD_BN2];
    const int kpad = (k + UPD_BK - 1) / UPD_BK * UPD_BK;
    const int64_t ncols = n - c0;
    const int tx = tid & 15, ty = tid >> 4;

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
        bar.sync();
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
        bar.sync();
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

// ---------------------------------------------------------------------------
// Multi-modular tile (integer tensor pipe): 64 x 64 outputs, 32 x 16 per warp.
// The arithmetic and its bounds are described in update_crt.cu.

constexpr int CRT_L = 9;                            // moduli 256, 255, 253, 251, 247, 241, 239, 233, 229
constexpr int CRT_BM = 64, CRT_BN = 64;
constexpr int CRT_KB = NB_MAX;                      // bytes per residue row (k <= 128)
constexpr int CRT_STAGES = 3;
constexpr int CRT_A_BYTES = CRT_BM * CRT_KB;        // 8 KB
constexpr int CRT_B_BYTES = CRT_BN * CRT_KB;        // 8 KB
constexpr int CRT_STAGE_BYTES = CRT_A_BYTES + CRT_B_BYTES;
constexpr size_t CRT_SMEM = (size_t)CRT_STAGES * CRT_STAGE_BYTES + 64;   // the ring, then 3 mbarriers

// Per-prime constants of the reconstruction (computed on the host, make_crt).
struct CrtConsts {
    uint32_t m[CRT_L];      // the moduli
    uint32_t y[CRT_L];      // (M / m_i)^(-1) mod m_i
    uint32_t off30[CRT_L];  // m_i ceil(2^30 / m_i): makes a balanced residue of p non-negative
    uint32_t mgf[CRT_L];    // floor(2^32 / m_i)
    uint32_t mgc[CRT_L];    // ceil(2^32 / m_i)
    uint32_t c38[CRT_L];    // floor(2^38 / m_i) (below 2^31)
    uint32_t wp[CRT_L];     // (M / m_i) mod p
    uint32_t negMp;         // (-M) mod p
};

__device__ __forceinline__ void mma_s8(int (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                       uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done;
}

// Wait for phase `parity` of an mbarrier, giving up (false) after about
// `limit` SM clock cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (clock64() - t0 < limit)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// The residue GEMM of one modulus for this thread's 2 x 2 fragments (32 x 16
// outputs per warp): D += A_q B_q over ksteps k-steps of 32, from one stage.
__device__ __forceinline__ void crt_mma_stage(int (&D)[2][2][4], const uint8_t* As, const uint8_t* Bs,
                                              int arow, int bcol, int g, int ksteps) {
#pragma unroll 1
    for (int ks = 0; ks < ksteps; ++ks) {
        const int c_lo = ((2 * ks) ^ g) * 16, c_hi = ((2 * ks + 1) ^ g) * 16;
        uint32_t af[2][4], bf[2][2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const uint8_t* p0 = As + arow + a * 16 * CRT_KB;
            af[a][0] = *reinterpret_cast<const uint32_t*>(p0 + c_lo);
            af[a][1] = *reinterpret_cast<const uint32_t*>(p0 + 8 * CRT_KB + c_lo);
            af[a][2] = *reinterpret_cast<const uint32_t*>(p0 + c_hi);
            af[a][3] = *reinterpret_cast<const uint32_t*>(p0 + 8 * CRT_KB + c_hi);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const uint8_t* p0 = Bs + bcol + b * 8 * CRT_KB;
            bf[b][0] = *reinterpret_cast<const uint32_t*>(p0 + c_lo);
            bf[b][1] = *reinterpret_cast<const uint32_t*>(p0 + c_hi);
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) mma_s8(D[a][b], af[a][0], af[a][1], af[a][2], af[a][3], bf[b][0], bf[b][1]);
    }
}

// One 64 x 64 output tile (rows row0.., columns col0.. relative to c0) for a
// group of 256 threads.  The group's three-stage ring starts at shared
// address sbase (CRT_STAGES * CRT_STAGE_BYTES bytes, generic pointer smem)
// with its three mbarriers at bar0; the tile's nine loads are items j0 ..
// j0 + 8 of the group's running sequence (stage j % 3, phase j / 3), so a
// group may reduce many tiles in a row.  Returns false (on every thread of the
// group) if a load never arrived: the status word then holds
// LINAC_ERR_TIMEOUT and the group's copies are no longer in flight.
template <class Bar>
__device__ __forceinline__ bool crt_tile(uint32_t* __restrict__ M, int64_t m, int64_t n, int64_t ld, int c0,
                                         const Field& f, int k, int r, const uint8_t* __restrict__ Fr,
                                         const uint8_t* __restrict__ Rr, int64_t m_pad, int64_t n_pad,
                                         const int32_t* __restrict__ R, int64_t ldR, const CrtConsts& cc,
                                         int* status, long long spin, int64_t row0, int64_t col0, int j0, int tid,
                                         uint8_t* smem, uint32_t sbase, uint32_t bar0, Bar bar) {
    const int ksteps = (k + 31) / 32;
    const int64_t ncols = n - c0;
    const int warp = tid >> 5, lane = tid & 31;
    const int wm = warp & 1, wn = warp >> 1;        // 2 x 4 warps of 32 x 16 outputs
    const int g = lane >> 2, t4 = lane & 3;

    auto issue = [&](int q) {   // residues of modulus q of this tile (item j0 + q)
        const int s = (j0 + q) % CRT_STAGES;
        const uint32_t b = bar0 + 8 * s;
        const uint32_t dst = sbase + s * CRT_STAGE_BYTES;
        mbar_expect_tx(b, CRT_STAGE_BYTES);
        bulk_load(dst, Fr + ((int64_t)q * m_pad + row0) * CRT_KB, CRT_A_BYTES, b);
        bulk_load(dst + CRT_A_BYTES, Rr + ((int64_t)q * n_pad + col0) * CRT_KB, CRT_B_BYTES, b);
    };
    int issued = 0;   // loads of this tile issued so far (thread 0 only)
    if (tid == 0)
        for (; issued < CRT_STAGES; ++issued) issue(issued);

    // byte offsets of this thread's fragments inside a stage (the swizzle
    // uses row & 7 = g for every row and column the thread touches)
    const int arow = (wm * 32 + g) * CRT_KB + 4 * t4;
    const int bcol = (wn * 16 + g) * CRT_KB + 4 * t4;
    int failed = 0;
    int q_fail = CRT_L;   // first modulus whose data never arrived
    // waits for modulus q's stage and runs its GEMM into D (false, on every
    // thread, if the data never arrived)
    auto gemm_modulus = [&](int q, int (&D)[2][2][4]) -> bool {
        const int j = j0 + q, s = j % CRT_STAGES;
        if (!mbar_wait(bar0 + 8 * s, (uint32_t)((j / CRT_STAGES) & 1), spin)) failed = 1;
        if (bar.sync_or(failed)) {
            failed = 1;
            q_fail = q;
            return false;
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int e = 0; e < 4; ++e) D[a][b][e] = 0;
        crt_mma_stage(D, smem + s * CRT_STAGE_BYTES, smem + s * CRT_STAGE_BYTES + CRT_A_BYTES, arow, bcol, g,
                      ksteps);
        return true;
    };

    // S = sum_i D'_i floor(2^38 / m_i) and X = sum_i D'_i ((M / m_i) mod p),
    // exact signed 64-bit sums (|S|, |X| < 9 * 2^21 * 2^31 < 2^56)
    int64_t S[2][2][4], X[2][2][4];
    int Dc[2][2][4], Dn[2][2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                S[a][b][e] = 0;
                X[a][b][e] = 0;
            }
    gemm_modulus(0, Dc);
    // software pipeline over the moduli: the GEMM of modulus q + 1 is issued
    // before the reconstruction step of modulus q, so the tensor pipe works
    // while the integer pipe folds D'_q into S and X
#pragma unroll
    for (int q = 0; q < CRT_L; ++q) {
        if (failed) break;
        if (q + 1 < CRT_L && !gemm_modulus(q + 1, Dn)) break;
        bar.sync();   // every warp has read item j0 + q's stage: it may be refilled
        if (tid == 0 && issued < CRT_L) issue(issued++);
        const int32_t c38 = (int32_t)cc.c38[q], wp = (int32_t)cc.wp[q];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    mac_s64(S[a][b][e], Dc[a][b][e], c38);
                    mac_s64(X[a][b][e], Dc[a][b][e], wp);
                    Dc[a][b][e] = Dn[a][b][e];
                }
    }
    if (failed) {
        // wait (bounded) for the copies still in flight into this group's
        // buffers (loads q_fail .. issued - 1), then report
        if (tid == 0) {
            atomicCAS(status, 0, (int)LINAC_ERR_TIMEOUT);
            for (int q = q_fail; q < issued; ++q) {
                const int j = j0 + q;
                (void)mbar_wait(bar0 + 8 * (j % CRT_STAGES), (uint32_t)((j / CRT_STAGES) & 1), spin);
            }
        }
        bar.sync();
        return false;
    }

    // step 4 and the write-back: rows of the new pivot block receive R,
    // every other row C - D mod p
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int64_t row = row0 + wm * 32 + a * 16 + g + hh * 8;
            if (row >= m) continue;
            const bool pivot_row = row >= r && row < r + k;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int64_t col = col0 + wn * 16 + b * 8 + 2 * t4;
                if (col >= ncols) continue;
                uint32_t out[2];
                uint32_t* dst = M + row * ld + c0 + col;
                const bool pair = col + 1 < ncols;
                if (pivot_row) {
                    const int32_t* rr = R + (int64_t)(row - r) * ldR + col;
                    out[0] = from_balanced(rr[0], f);
                    out[1] = pair ? from_balanced(rr[1], f) : 0u;
                } else {
                    uint32_t cval[2];
                    if (pair) {
                        const uint2 cv = *reinterpret_cast<const uint2*>(dst);
                        cval[0] = cv.x;
                        cval[1] = cv.y;
                    } else {
                        cval[0] = dst[0];
                        cval[1] = 0;
                    }
#pragma unroll
                    for (int qq = 0; qq < 2; ++qq) {
                        const int e = hh * 2 + qq;
                        // beta = nearest integer to S / 2^38 (floor of S / 2^38 + 1/2)
                        const int64_t beta = (S[a][b][e] + (1LL << 37)) >> 38;
                        const int64_t x = X[a][b][e] + beta * (int64_t)cc.negMp;
                        out[qq] = submod(cval[qq], reduce_signed(x, f), f);
                    }
                }
                if (pair) *reinterpret_cast<uint2*>(dst) = make_uint2(out[0], out[1]);
                else dst[0] = out[0];
            }
        }
    return true;
}

}  // namespace linac
