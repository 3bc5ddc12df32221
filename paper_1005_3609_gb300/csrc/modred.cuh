// Exact reduction of a gather accumulator modulo a prime, integer arithmetic only.
//
// A destination word accumulates v = sum_e coef_e x_e with |x_e| <= p (inputs
// are residues in [0, p) or signed representatives in [-p, p)), so
// |v| <= p S where S = sum_e |coef_e| over the destination's edges; the table
// build refuses any table with S >= 2^20 (kReduceMaxCoefSum).  Arithmetic is
// modulo primes below 2^31 (Sec. 3.5).
//
// The accumulator starts at the bias p 2^21, a multiple of p larger than |v|,
// so that what is reduced is u = p 2^21 + v with 0 < u < 3 p 2^20.
//
// Quotient estimate (a Barrett reduction, Barrett 1986, with a 32-bit
// reciprocal of the prime's own scale): let b be the bit length of p
// (2^(b-1) <= p < 2^b, b >= 2), s = b - 2 and m = floor(2^(32+s) / p), so
// 2^30 <= m <= 2^31 fits 32 bits.  With h = floor(u / 2^s) (below 2^32, since
// u < 2^(b+22)) and q = floor(h m / 2^32) (one 32-bit high multiply):
//   h m <= (u / 2^s)(2^(32+s) / p) = 2^32 u / p                 so q <= u / p;
//   h m >  (u / 2^s - 1)(2^(32+s) / p - 1)
//       >  2^32 u / p - u / 2^s - 2^(32+s) / p,
//   so h m / 2^32 > u / p - u / 2^(32+s) - 2^s / p > u / p - 2^-8 - 1/2,
// hence q is floor(u / p) or floor(u / p) - 1 and r = u - q p lies in [0, 2p).
// As 2p < 2^32, r is exact in 32-bit arithmetic (taken modulo 2^32), and one
// conditional subtraction gives u mod p = v mod p.
#pragma once

#include <stdint.h>

namespace cp {

constexpr uint32_t kReduceMaxCoefSum = 1u << 20;  // sum |coef| into one state must stay below this

// Per-prime constants of the reduction.
struct ModRed {
    uint32_t p;   // the prime, 2 <= p < 2^31
    uint32_t m;   // floor(2^(32+s) / p)
    uint32_t s;   // bit length of p minus 2
    uint32_t pad;
};

__host__ __device__ __forceinline__ ModRed modred_make(uint32_t p) {
    uint32_t b = 0;
    while (b < 32 && (p >> b) != 0) ++b;  // bit length
    ModRed r;
    r.p = p;
    r.s = b - 2;
    r.m = (uint32_t)((1ull << (32 + r.s)) / p);
    r.pad = 0;
    return r;
}

// The bias every accumulator of prime p starts from: p 2^21.
__host__ __device__ __forceinline__ long long modred_bias(uint32_t p) { return (long long)p << 21; }

// A signed representative of u mod p in [-p, p), as its 32-bit two's
// complement: r - p with r = u - q p in [0, 2p) (one instruction fewer than
// the full reduction).  The gathers read every input word as a signed 32-bit
// value, so inputs in [-p, p) still give |v| < p S and the bias above covers
// them; a gather whose output only feeds further gathers may store this.
__device__ __forceinline__ uint32_t modred_reduce_signed(long long acc, uint32_t p, uint32_t m, uint32_t s) {
    const unsigned long long u = (unsigned long long)acc;
    const uint32_t h = (uint32_t)(u >> s);
    const uint32_t q = __umulhi(h, m);
    return (uint32_t)u - q * p - p;  // r - p, r in [0, 2p); exact modulo 2^32
}

// u mod p for an accumulator u = p 2^21 + v, |v| < p 2^20.
__device__ __forceinline__ uint32_t modred_reduce(long long acc, uint32_t p, uint32_t m, uint32_t s) {
    const unsigned long long u = (unsigned long long)acc;
    const uint32_t h = (uint32_t)(u >> s);
    const uint32_t q = __umulhi(h, m);
    const uint32_t r = (uint32_t)u - q * p;  // in [0, 2p), exact modulo 2^32
    return min(r, r - p);
}

}  // namespace cp
