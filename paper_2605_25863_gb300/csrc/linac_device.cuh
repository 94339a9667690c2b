// linac_device.cuh -- device-side building blocks shared by the sm_103a kernels:
// modular arithmetic for odd primes p < 2^31, the pivot inverse, a bounded
// grid barrier for cooperative launches, and the on-device state records.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/linac.h"

namespace linac {

// ---------------------------------------------------------------------------
// Per-prime constants, computed once per call on the host.
//
//  mu   = floor(2^64 / p)            Barrett constant for 64-bit operands.
//  c32  = 2^32 mod p                 folds a signed 64-bit lazy accumulator
//                                    H*2^32 + L into H*c32 + L.
//  half = (p - 1) / 2                residues r > half are stored as r - p
//                                    ("balanced" signed form, |x| <= half).
//  fold = number of balanced products |x*y| <= half^2 that may be added to a
//         folded accumulator without leaving the signed 64-bit range.
//  pinv = -p^(-1) mod 2^32,  r2 = 2^64 mod p   Montgomery constants (R = 2^32).
struct Field {
    uint32_t p;
    uint32_t c32;
    uint64_t mu;
    uint32_t half;
    uint32_t fold;
    uint32_t pinv;
    uint32_t r2;
};

__host__ __device__ inline uint32_t lo32(uint64_t x) { return (uint32_t)x; }

// x mod p for any 64-bit x.  Barrett: q = floor(x * mu / 2^64) satisfies
// x/p - 2 < q <= x/p, so x - q*p lies in [0, 2p) and one conditional
// subtraction finishes (p < 2^31 keeps every intermediate in 64 bits).
__device__ __forceinline__ uint32_t reduce64(uint64_t x, const Field& f) {
    uint64_t q = __umul64hi(x, f.mu);
    uint64_t r = x - q * (uint64_t)f.p;
    if (r >= f.p) r -= f.p;
    return (uint32_t)r;
}

__device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b, const Field& f) {
    return reduce64((uint64_t)a * b, f);
}

// (a*x + b*y) mod p with a, b, x, y in [0, p): the sum of two products is
// below 2^63, so a single reduction suffices.
__device__ __forceinline__ uint32_t mul2add(uint32_t a, uint32_t x, uint32_t b, uint32_t y,
                                            const Field& f) {
    return reduce64((uint64_t)a * x + (uint64_t)b * y, f);
}

__device__ __forceinline__ uint32_t addmod(uint32_t a, uint32_t b, const Field& f) {
    uint32_t s = a + b;                     // < 2^32 since a, b < 2^31
    return s >= f.p ? s - f.p : s;
}

__device__ __forceinline__ uint32_t submod(uint32_t a, uint32_t b, const Field& f) {
    return a >= b ? a - b : a + f.p - b;
}

// Balanced signed representative of a residue, |result| <= (p-1)/2.
__device__ __forceinline__ int32_t to_balanced(uint32_t r, const Field& f) {
    return r > f.half ? (int32_t)(r - f.p) : (int32_t)r;
}

__device__ __forceinline__ uint32_t from_balanced(int32_t v, const Field& f) {
    return v < 0 ? (uint32_t)(v + (int32_t)f.p) : (uint32_t)v;
}

// Signed 64-bit lazy accumulator fold: acc = H*2^32 + L  ->  H*c32 + L, which
// is congruent mod p and has magnitude below 2^31*c32 + 2^32 <= 2^62 + 2^32.
__device__ __forceinline__ int64_t fold64(int64_t acc, const Field& f) {
    int32_t H = (int32_t)(acc >> 32);
    uint32_t L = (uint32_t)acc;
    return (int64_t)H * (int64_t)f.c32 + (int64_t)L;
}

// acc += a * b as one fused signed 32 x 32 -> 64 multiply-add (the
// accumulator is the 64-bit addend of mad.wide.s32).
__device__ __forceinline__ void mac_s64(int64_t& acc, int32_t a, int32_t b) {
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// fold64 as a two-instruction carry chain: low word lo(H*c32) + L with carry
// out, high word hi(H*c32) (signed; c32 < 2^31) plus the carry.
__device__ __forceinline__ int64_t fold64_fast(int64_t acc, const Field& f) {
    int64_t out;
    asm("{\n\t"
        ".reg .u32 lo, hi, rlo, rhi;\n\t"
        "mov.b64 {lo, hi}, %1;\n\t"
        "mad.lo.cc.u32 rlo, hi, %2, lo;\n\t"
        "madc.hi.s32 rhi, hi, %2, 0;\n\t"
        "mov.b64 %0, {rlo, rhi};\n\t"
        "}"
        : "=l"(out)
        : "l"(acc), "r"(f.c32));
    return out;
}

// Canonical residue of a signed 64-bit accumulator with |acc| < 2^63.
__device__ __forceinline__ uint32_t reduce_signed(int64_t acc, const Field& f) {
    int64_t t = fold64(acc, f);            // |t| < 2^31 * c32 + 2^32 <= 2^31 * p + 2^32
    // p * 2^32 is a multiple of p above |t| (2^31 p + 2^32 <= 2^32 p for p >= 2)
    // and t + p * 2^32 < 2^63, so the sum is a non-negative 64-bit value.
    uint64_t off = (uint64_t)f.p << 32;
    return reduce64((uint64_t)(t + (int64_t)off), f);
}

// Fold of a signed lazy accumulator with shifts and adds.  When c32 = 2^32
// mod p has at most three set bits (2^e0 + 2^e1 + 2^e2; 2^31 - 1 gives 2,
// 2^31 - 19 gives 38) H*c32 is formed on the ALU pipe, leaving the integer
// multiply pipe to the products.  SHIFTS = 0 selects the multiply-pipe fold
// (any p).  alu_reduce marks primes for which reduce_alu below is exact.
struct FoldShifts {
    uint32_t e[3];      // shift of each set bit of c32
    uint32_t s[3];      // arithmetic right shift giving the high word of h * 2^e
    int32_t alu_reduce; // reduce_alu is exact for this p
    int32_t pad;
};

template <int SHIFTS>
__device__ __forceinline__ int64_t fold_any(int64_t acc, const Field& f, const FoldShifts& fs) {
    if (SHIFTS == 0) return fold64_fast(acc, f);
    // acc = hi:lo; result = lo + sum_i sext(hi) * 2^e_i as a 64-bit carry chain
    // of 32-bit shifts and adds, written out so it stays on the ALU pipe
    uint32_t lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(acc));
    uint32_t rlo = lo, rhi = 0;
#pragma unroll
    for (int i = 0; i < SHIFTS; ++i) {
        asm("{\n\t.reg .u32 t, u;\n\t"
            "shl.b32 t, %2, %3;\n\t"
            "shr.s32 u, %2, %4;\n\t"
            "add.cc.u32 %0, %0, t;\n\t"
            "addc.u32 %1, %1, u;\n\t}"
            : "+r"(rlo), "+r"(rhi)
            : "r"(hi), "r"(fs.e[i]), "r"(fs.s[i]));
    }
    int64_t out;
    asm("mov.b64 %0, {%1, %2};" : "=l"(out) : "r"(rlo), "r"(rhi));
    return out;
}

// Canonical residue of a signed 64-bit accumulator (|acc| < 2^63) by two
// folds and two conditional subtractions, whenever fs.alu_reduce (without
// any multiply when SHIFTS > 0; SHIFTS = 0 folds on the multiply pipe, which
// computes the same L + sext(H) c32).  Two folds bring acc to
//   t2 = L2 + H2*c32 with H2 in [-(c32+1)/2, c32/2 + 1], so
//   t2 in [-c32 (c32+1)/2, 2^32 - 1 + c32 (c32/2 + 1)];
// the host sets alu_reduce only when c32 (c32+1)/2 <= p and
// 2^32 - 1 + c32 (c32/2 + 1) < 3p, so u = t2 + p lies in [0, 4p) and two
// conditional subtractions (2p, then p) finish.
template <int SHIFTS>
__device__ __forceinline__ uint32_t reduce_alu(int64_t acc, const Field& f, const FoldShifts& fs) {
    const int64_t t2 = fold_any<SHIFTS>(fold_any<SHIFTS>(acc, f, fs), f, fs);
    uint64_t u = (uint64_t)(t2 + (int64_t)f.p);
    const uint64_t p2 = 2ull * f.p;
    if (u >= p2) u -= p2;
    if (u >= f.p) u -= f.p;
    return (uint32_t)u;
}

// Canonical residue of a lazy accumulator: the multiply-free reduction when it
// applies, the Barrett reduction otherwise.
template <int SHIFTS>
__device__ __forceinline__ uint32_t reduce_acc(int64_t acc, const Field& f, const FoldShifts& fs) {
    if (fs.alu_reduce) return reduce_alu<SHIFTS>(acc, f, fs);
    return reduce_signed(acc, f);
}

// Montgomery arithmetic with R = 2^32 (P. L. Montgomery, "Modular
// multiplication without trial division", Math. Comp. 44, 1985).  x is held as
// x R mod p; zero stays zero, negation commutes with the map, and the product
// of two held values reduced by mont_redc is the held value of the product.
// mont_redc(t) = t R^(-1) mod p for t < p R: m = (t mod R) (-p^(-1)) mod R
// makes t + m p divisible by R, and (t + m p) / R < 2p (p < 2^31 keeps
// t + m p below 2^64), so one conditional subtraction finishes.
__device__ __forceinline__ uint32_t mont_redc(uint64_t t, const Field& f) {
    const uint32_t m = (uint32_t)t * f.pinv;
    const uint64_t u = t + (uint64_t)m * f.p;
    const uint32_t r = (uint32_t)(u >> 32);
    return r >= f.p ? r - f.p : r;
}

// (a x + b y) R^(-1) mod p for a, x, b, y in [0, p): 2 p^2 < p R.
__device__ __forceinline__ uint32_t mont_mul2add(uint32_t a, uint32_t x, uint32_t b, uint32_t y, const Field& f) {
    return mont_redc((uint64_t)a * x + (uint64_t)b * y, f);
}

__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, const Field& f) {
    return mont_redc((uint64_t)a * b, f);
}

// x -> x R mod p (x in [0, p)): x R^2 R^(-1).
__device__ __forceinline__ uint32_t to_mont(uint32_t x, const Field& f) { return mont_mul(x, f.r2, f); }

// Modular inverse of a (0 < a < p, p odd) by the binary extended Euclidean
// algorithm (Stein's binary gcd, Knuth TAOCP vol. 2 sec. 4.5.2, carrying
// Bezout coefficients): invariants x1*a = u and x2*a = v (mod p); halving a
// coefficient first adds p when it is odd, which is exact because p is odd.
// Returns 0 for a == 0 (no inverse).
__device__ __forceinline__ uint32_t inverse_mod(uint32_t a, uint32_t p) {
    if (a == 0) return 0;
    uint32_t u = a, v = p, x1 = 1, x2 = 0;
    // each pass removes at least one bit from u or v: <= 62 passes for p < 2^31
    for (int guard = 0; guard < 256 && u != 1 && v != 1; ++guard) {
        while ((u & 1u) == 0) {
            u >>= 1;
            x1 = (x1 & 1u) ? (uint32_t)(((uint64_t)x1 + p) >> 1) : (x1 >> 1);
        }
        while ((v & 1u) == 0) {
            v >>= 1;
            x2 = (x2 & 1u) ? (uint32_t)(((uint64_t)x2 + p) >> 1) : (x2 >> 1);
        }
        if (u >= v) { u -= v; x1 = x1 >= x2 ? x1 - x2 : x1 + p - x2; }
        else        { v -= u; x2 = x2 >= x1 ? x2 - x1 : x2 + p - x1; }
    }
    return u == 1 ? x1 : x2;
}

// Modular inverse of a (0 < a < p, p prime) as a^(p-2) (Fermat's little
// theorem), by left-to-right binary exponentiation.  The exponent is the same
// for every thread, so a warp inverting many values never diverges.  Returns
// 0 for a == 0.
__device__ __forceinline__ uint32_t inverse_fermat(uint32_t a, const Field& f) {
    const uint32_t e = f.p - 2u;
    uint32_t x = a;
    for (int b = 30 - __clz(e); b >= 0; --b) {
        x = mulmod(x, x, f);
        if ((e >> b) & 1u) x = mulmod(x, a, f);
    }
    return x;
}

// ---------------------------------------------------------------------------
// Bounded spin limits.  Every wait on another block gives up after about
// kSpinCycles clocks, records LINAC_ERR_TIMEOUT in the status word and lets
// the kernel return, so a fault elsewhere can never hang the device.
constexpr long long kSpinCycles = 4000000000LL;   // ~2 s at 2 GHz

// Limit of the panel kernel's arrival wait, passed by value at every launch:
// spin_cycles clocks (kSpinCycles unless the caller set another limit with
// linac_set_wait_limit), and extra_arrivals added to the arrival target.
// extra_arrivals is 0 except when a test injects a wait failure
// (linac_debug_inject_wait_failure): the target then exceeds the arrivals
// the grid makes, so every block's wait runs out and returns
// LINAC_ERR_TIMEOUT through the status word.
struct WaitLimit {
    long long spin_cycles;
    unsigned int extra_arrivals;
    unsigned int pad;
};

struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};

// Sense-counting grid barrier for kernels launched cooperatively (all blocks
// co-resident).  Returns false if it gave up (timeout or a status already set).
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned nblocks, int* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = &bar->gen;
        unsigned int my_gen = *vgen;
        __threadfence();
        unsigned int arrived = atomicAdd(&bar->count, 1u);
        int ok = 1;
        if (arrived == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            long long t0 = clock64();
            while (*vgen == my_gen) {
                if (*(volatile int*)status != 0) { ok = 0; break; }
                if (clock64() - t0 > kSpinCycles) {
                    atomicCAS(status, 0, (int)LINAC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Arrival barrier on a monotonically increasing counter: each block adds 1
// once per round and waits until the counter reaches target (= rounds done x
// blocks).  No reset step, so the critical path is one posted reduction and
// the polling reads.  The caller has fenced its published data and passed a
// __syncthreads; on return every thread of the block may read what other
// blocks published before arriving.  Gives up (returns false) after about
// kSpinCycles clocks or when the status word is already set.
__device__ __forceinline__ bool grid_arrive_wait(unsigned int* counter, unsigned int target, int* status) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
        int ok = 1;
        const long long t0 = clock64();
        for (unsigned int it = 0;; ++it) {
            unsigned int v;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
            if ((int)(v - target) >= 0) break;
            if ((it & 255u) == 255u) {
                if (*(volatile int*)status != 0) { ok = 0; break; }
                if (clock64() - t0 > kSpinCycles) {
                    atomicCAS(status, 0, (int)LINAC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace linac
