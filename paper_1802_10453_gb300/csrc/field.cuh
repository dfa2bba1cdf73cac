// field.cuh -- arithmetic in F = Z/pZ (p prime, p < 2^31) for the device.
//
// Residues are canonical uint32 in [0, p).  Reduction of a 64-bit value uses
// Barrett's method (P. Barrett, "Implementing the Rivest Shamir and Adleman
// public key encryption algorithm on a standard digital signal processor",
// CRYPTO 1986) with mu = floor((2^64 - 1) / p): q = hi64(x * mu) underestimates
// floor(x / p) by at most 2, so at most two corrections follow.
//
// Dot products accumulate exact 64-bit products without reducing each one:
// products are < 2^62, and whenever the running sum reaches 2^63 a fixed
// multiple M of p with 2^62 < M <= 2^63 is subtracted, so the sum never wraps.
#pragma once
#include <cstdint>

struct FieldP {
    uint32_t p;
    uint32_t inv2;   // (p + 1) / 2, the inverse of 2 for odd p; 0 for p = 2
    uint64_t mu;     // floor((2^64 - 1) / p)
    uint64_t m63;    // multiple of p in (2^62, 2^63]
    uint32_t c32;    // 2^32 mod p
    uint32_t c32q;   // floor(c32 * 2^32 / p)   (Shoup companion of c32)
    uint32_t oneq;   // floor(2^32 / p)         (Shoup companion of 1)
    uint32_t kb;     // bit length k of p (2^(k-1) <= p < 2^k)
    uint32_t muk;    // floor(2^(2k) / p) < 2^(k+1) (Barrett constant for products)
    uint32_t pad2;
};

inline FieldP make_field(uint32_t p)
{
    FieldP f;
    f.p = p;
    f.inv2 = (p == 2) ? 0u : (p + 1u) / 2u;
    f.mu = ~0ull / (uint64_t)p;
    uint64_t pp = (uint64_t)p * (uint64_t)p;
    f.m63 = ((1ull << 63) / pp) * pp;  // > 2^62 because pp < 2^62
    f.c32 = (uint32_t)((1ull << 32) % p);
    f.c32q = (uint32_t)(((uint64_t)f.c32 << 32) / p);
    f.oneq = (uint32_t)((1ull << 32) / p);
    uint32_t k = 0;
    while (k < 32 && (p >> k) != 0) ++k;
    f.kb = k;
    f.muk = (uint32_t)((1ull << (2 * k)) / p);  // k <= 31, so 2k <= 62
    f.pad2 = 0;
    return f;
}

__device__ __forceinline__ uint32_t fp_reduce64(uint64_t x, const FieldP &f)
{
    uint64_t q = __umul64hi(x, f.mu);
    uint64_t r = x - q * (uint64_t)f.p;
    if (r >= f.p) r -= f.p;
    if (r >= f.p) r -= f.p;
    return (uint32_t)r;
}

// x mod p for any 64-bit x with 32-bit operations only: x = hi 2^32 + lo with
// hi * (2^32 mod p) and lo each reduced by Shoup's method (V. Shoup, NTL:
// multiplication by a fixed w with w' = floor(w 2^32 / p) leaves a remainder
// in [0, 2p)), then one final correction.  Fewer and cheaper instructions
// than fp_reduce64 (no 64 x 64-bit high product).
__device__ __forceinline__ uint32_t fp_reduce64_fold(uint64_t x, const FieldP &f)
{
    const uint32_t hi = (uint32_t)(x >> 32), lo = (uint32_t)x;
    uint32_t a = hi * f.c32 - __umulhi(hi, f.c32q) * f.p;
    uint32_t b = lo - __umulhi(lo, f.oneq) * f.p;
    a = a >= f.p ? a - f.p : a;
    b = b >= f.p ? b - f.p : b;
    const uint32_t s = a + b;  // < 2p < 2^32
    return s >= f.p ? s - f.p : s;
}

// a * b mod p for residues a, b < p by Barrett's method with the k-bit
// constant muk = floor(2^(2k) / p) (Handbook of Applied Cryptography,
// Algorithm 14.42, base 2): x = a b < 2^(2k), q = floor(floor(x / 2^(k-1)) muk /
// 2^(k+1)) underestimates floor(x / p) by at most 2.  Both products are 32 x
// 32 bits (x / 2^(k-1) < 2^(k+1) <= 2^32 and muk < 2^(k+1)).
__device__ __forceinline__ uint32_t fp_mul(uint32_t a, uint32_t b, const FieldP &f)
{
    const uint64_t x = (uint64_t)a * (uint64_t)b;
    const uint32_t t = (uint32_t)(x >> (f.kb - 1));
    const uint32_t q = (uint32_t)(((uint64_t)t * (uint64_t)f.muk) >> (f.kb + 1));
    uint64_t r = x - (uint64_t)q * (uint64_t)f.p;
    if (r >= f.p) r -= f.p;
    if (r >= f.p) r -= f.p;
    return (uint32_t)r;
}

__device__ __forceinline__ uint32_t fp_add(uint32_t a, uint32_t b, const FieldP &f)
{
    uint32_t s = a + b;  // < 2^32 since a, b < 2^31
    return s >= f.p ? s - f.p : s;
}

__device__ __forceinline__ uint32_t fp_sub(uint32_t a, uint32_t b, const FieldP &f)
{
    return a >= b ? a - b : a + (f.p - b);
}

// acc += a * b without overflow (see the header comment).
__device__ __forceinline__ void fp_mac(uint64_t &acc, uint32_t a, uint32_t b, const FieldP &f)
{
    acc += (uint64_t)a * (uint64_t)b;
    acc -= (acc >> 63) * f.m63;
}

// Inverse of a != 0 modulo the prime p: extended Euclidean algorithm on
// 32-bit values (the Bezout coefficient is tracked modulo p).
__device__ __forceinline__ uint32_t fp_inv(uint32_t a, const FieldP &f)
{
    uint32_t r0 = f.p, r1 = a;
    int64_t s0 = 0, s1 = 1;
    while (r1 != 0) {
        uint32_t q = r0 / r1;
        uint32_t r2 = r0 - q * r1;
        int64_t s2 = s0 - (int64_t)q * s1;
        r0 = r1; r1 = r2;
        s0 = s1; s1 = s2;
    }
    int64_t v = s0 % (int64_t)f.p;
    if (v < 0) v += f.p;
    return (uint32_t)v;
}

// Inverse of a != 0 modulo the odd prime p by the binary extended Euclidean
// algorithm (halvings and subtractions only; D. E. Knuth, TAOCP vol. 2,
// Section 4.5.2, and A. Menezes et al., Handbook of Applied Cryptography,
// Algorithm 14.61).  Invariants: x1 a = u and x2 a = v (mod p); a halving of u
// halves x1 mod p ((x1 + p) / 2 when x1 is odd).  p = 2 has the inverse 1;
// a = 0 returns 0.
__device__ __forceinline__ uint32_t fp_inv_bin(uint32_t a, const FieldP &f)
{
    const uint32_t p = f.p;
    if (p == 2) return 1u;
    if (a == 0u) return 0u;  // no inverse; never loop on it
    uint32_t u = a, v = p, x1 = 1u, x2 = 0u;
    while (u != 1u && v != 1u) {
        while ((u & 1u) == 0u) {
            u >>= 1;
            x1 = (x1 & 1u) ? (uint32_t)(((uint64_t)x1 + p) >> 1) : (x1 >> 1);
        }
        while ((v & 1u) == 0u) {
            v >>= 1;
            x2 = (x2 & 1u) ? (uint32_t)(((uint64_t)x2 + p) >> 1) : (x2 >> 1);
        }
        if (u >= v) {
            u -= v;
            x1 = fp_sub(x1, x2, f);
        } else {
            v -= u;
            x2 = fp_sub(x2, x1, f);
        }
    }
    return u == 1u ? x1 : x2;
}

