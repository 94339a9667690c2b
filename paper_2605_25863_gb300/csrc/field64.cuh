// field64.cuh -- arithmetic in Z/pZ for odd primes p < 2^64 held in uint64
// (the paper's uint64 backend for primes that do not fit 32 bits, section
// 2.3 "Basic Usage").
//
// Values inside the elimination kernels are kept in Montgomery form x*R mod p
// with R = 2^64 (Montgomery 1985): a product is one 64 x 64 -> 128-bit
// multiplication followed by one reduction t -> t / R mod p, which needs
// only multiplications by the constant -p^(-1) mod 2^64 and by p.
//
// The trailing update accumulates up to 32 full 128-bit products exactly in a
// 160-bit accumulator (five 32-bit limbs, carry-propagating multiply-adds) and
// reduces once per output with two Montgomery steps; the operand F is scaled
// by R^2 beforehand so the two divisions by R cancel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace linac {

struct Field64 {
    uint64_t p;      // odd prime, 3 <= p < 2^64
    uint64_t pinv;   // -p^(-1) mod 2^64
    uint64_t r1;     // 2^64 mod p   (Montgomery form of 1)
    uint64_t r2;     // 2^128 mod p  (x -> x R: multiply by this and reduce)
    uint64_t r3;     // 2^192 mod p  (x -> x R^2)
};

// t / 2^64 mod p for t = hi * 2^64 + lo < p * 2^64.  With m = lo * pinv, the
// sum t + m p is divisible by 2^64: its low word lo + (m p mod 2^64) is 0 when
// lo = 0 and 2^64 otherwise, so the quotient is hi + floor(m p / 2^64) + [lo != 0],
// which is below 2p and may exceed 2^64 when p > 2^63 (the carry is kept).
__device__ __forceinline__ uint64_t m64_redc(uint64_t lo, uint64_t hi, const Field64& f) {
    const uint64_t m = lo * f.pinv;
    const uint64_t mh = __umul64hi(m, f.p);
    const uint64_t s = hi + mh;
    bool over = s < hi;
    const uint64_t s2 = s + (lo != 0 ? 1ull : 0ull);
    over |= s2 < s;
    return (over || s2 >= f.p) ? s2 - f.p : s2;
}

// a b / 2^64 mod p for a, b < p (so a b < p * 2^64).
__device__ __forceinline__ uint64_t m64_mul(uint64_t a, uint64_t b, const Field64& f) {
    return m64_redc(a * b, __umul64hi(a, b), f);
}

__device__ __forceinline__ uint64_t m64_sub(uint64_t a, uint64_t b, const Field64& f) {
    return a >= b ? a - b : a + (f.p - b);
}

// x R mod p for a canonical residue x.
__device__ __forceinline__ uint64_t m64_to_mont(uint64_t x, const Field64& f) { return m64_mul(x, f.r2, f); }

// (x R)^e in Montgomery form, i.e. x^e R mod p, by square-and-multiply.
__device__ __forceinline__ uint64_t m64_pow(uint64_t xm, uint64_t e, const Field64& f) {
    uint64_t acc = f.r1;
    for (; e; e >>= 1) {
        if (e & 1) acc = m64_mul(acc, xm, f);
        xm = m64_mul(xm, xm, f);
    }
    return acc;
}

// l[0..4] += a * b exactly (a, b < 2^64; the 160-bit sum of up to 2^32
// products cannot overflow).  The product is a0 b0 + (a0 b1 + a1 b0) 2^32 +
// a1 b1 2^64 in 32-bit halves; three carry chains add its pieces.
__device__ __forceinline__ void mac160(uint32_t (&l)[5], uint64_t a, uint64_t b) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    asm("mad.lo.cc.u32 %0, %5, %7, %0;\n\t"
        "madc.hi.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %6, %8, %2;\n\t"
        "madc.hi.cc.u32 %3, %6, %8, %3;\n\t"
        "addc.u32 %4, %4, 0;\n\t"
        "mad.lo.cc.u32 %1, %5, %8, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %8, %2;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.u32 %4, %4, 0;\n\t"
        "mad.lo.cc.u32 %1, %6, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %6, %7, %2;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.u32 %4, %4, 0;"
        : "+r"(l[0]), "+r"(l[1]), "+r"(l[2]), "+r"(l[3]), "+r"(l[4])
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
}

// V / 2^128 mod p for the accumulator V = l4:l3:l2:l1:l0 of at most k <= 32
// products of residues (V < k p^2).  First step: V1 = (V + m1 p) / 2^64 <
// p (k p / 2^64 + 1) < (k + 1) p, held as T:H.  Second step: V2 = (V1 + m2 p)
// / 2^64 < p + k + 1, which may carry past 2^64 when p is near 2^64.  One
// subtraction finishes unless p <= k + 1 (tiny primes), where '%' does.
__device__ __forceinline__ uint64_t reduce160(const uint32_t (&l)[5], const Field64& f) {
    const uint64_t L = ((uint64_t)l[1] << 32) | l[0];
    const uint64_t H = ((uint64_t)l[3] << 32) | l[2];
    uint64_t T = l[4];
    const uint64_t m1 = L * f.pinv;
    const uint64_t h1 = H + __umul64hi(m1, f.p);
    T += h1 < H ? 1ull : 0ull;
    const uint64_t h1b = h1 + (L != 0 ? 1ull : 0ull);
    T += h1b < h1 ? 1ull : 0ull;
    const uint64_t m2 = h1b * f.pinv;
    const uint64_t mh2 = __umul64hi(m2, f.p);
    const uint64_t s = mh2 + T;
    bool over = s < mh2;
    const uint64_t s2 = s + (h1b != 0 ? 1ull : 0ull);
    over |= s2 < s;
    uint64_t v = (over || s2 >= f.p) ? s2 - f.p : s2;
    if (v >= f.p) v %= f.p;
    return v;
}

}  // namespace linac
