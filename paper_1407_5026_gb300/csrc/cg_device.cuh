// cg_device.cuh -- arithmetic building blocks of libcg shared by its host
// set-up code and its kernels: Philox-4x32-10, the acceptance exponential,
// minimum-image folding.  Every binary64 operation that feeds the chain is
// written with an explicit round-to-nearest intrinsic on the device, so the
// compiler cannot fuse a multiply and an add into one FMA.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cg {

// 32 x 32 -> 64-bit product as one wide multiply (both halves from one
// instruction instead of a high and a low multiply).
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo)
{
    unsigned long long p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
}

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies, key bumped by the Weyl constants between rounds.
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1,
                                                       uint32_t c2, uint32_t c3,
                                                       uint32_t k0, uint32_t k1,
                                                       uint32_t out[4])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        uint32_t hi0, lo0, hi1, lo1;
        mul_wide(0xD2511F53u, c0, hi0, lo0);
        mul_wide(0xCD9E8D57u, c2, hi1, lo1);
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Philox-4x32-10 split for counters (k, c1, c2, c3) whose words 1-3 are shared
// by many k: the parts of rounds 1 and 2 that do not depend on k are computed
// once (philox_prefix) and each k finishes the block (philox_finish).  The
// result is the same block as philox4x32_10(k, c1, c2, c3, k0, k1).
struct PhiloxPrefix {
    uint32_t A;     // c3 ^ k0-round-1 key word 1
    uint32_t B;     // round-2 high product of word 0, ^ key word 1
    uint32_t C;     // round-1 word 1, ^ round-2 key word 0
    uint32_t x3;    // round-2 low product of word 0 (the output's word 3 after round 2)
};

__device__ __forceinline__ PhiloxPrefix philox_prefix(uint32_t c1, uint32_t c2, uint32_t c3,
                                                      uint32_t k0, uint32_t k1)
{
    PhiloxPrefix P;
    // round 1: word 0 of the output and word 1 come from c1, c2 alone
    uint32_t hi1, lo1;
    mul_wide(0xCD9E8D57u, c2, hi1, lo1);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1;
    P.A = c3 ^ k1;
    // round 2 (keys bumped once): the product of word 0 is shared
    const uint32_t k0b = k0 + 0x9E3779B9u, k1b = k1 + 0xBB67AE85u;
    uint32_t hb;
    mul_wide(0xD2511F53u, n0, hb, P.x3);
    P.B = hb ^ k1b;
    P.C = n1 ^ k0b;
    return P;
}

__device__ __forceinline__ void philox_finish(uint32_t k, const PhiloxPrefix &P, uint32_t k0,
                                              uint32_t k1, uint32_t out[4])
{
    // round 1, the k-dependent half
    uint32_t h1, n3;
    mul_wide(0xD2511F53u, k, h1, n3);
    const uint32_t n2 = h1 ^ P.A;
    // round 2, the n2-dependent half
    uint32_t h2, c1;
    mul_wide(0xCD9E8D57u, n2, h2, c1);
    uint32_t c0 = h2 ^ P.C;
    uint32_t c2 = P.B ^ n3;
    uint32_t c3 = P.x3;
    k0 += 2u * 0x9E3779B9u;
    k1 += 2u * 0xBB67AE85u;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        if (r > 2) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        mul_wide(0xD2511F53u, c0, hi0, lo0);
        mul_wide(0xCD9E8D57u, c2, hi1, lo1);
        const uint32_t n0 = hi1 ^ c1 ^ k0, nn2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = nn2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Round-to-nearest binary64 operations that are never contracted to FMA.
__device__ __forceinline__ double d_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double d_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double d_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double d_div(double a, double b) { return __ddiv_rn(a, b); }

// exp(x) for -23 <= x <= 0 by Cody & Waite's additive argument reduction
// (Software Manual for the Elementary Functions, 1980) and the Taylor series
// of e^r to degree 13 in Horner form; 0 below -23, where e^x is smaller than
// the smallest acceptance variate 2^-33.  ln 2 is split as LN2_HI (29
// significant bits, so k*LN2_HI is exact) plus LN2_LO; the coefficients are
// 1/n! rounded to binary64.
__device__ __forceinline__ double cg_exp_accept(double x)
{
    if (x < -23.0) return 0.0;
    const double kd = rint(d_mul(x, 0x1.71547652b82fep+0));
    const double r = d_sub(d_sub(x, d_mul(kd, 0x1.62e42ffp-1)),
                           d_mul(kd, -0x1.718432a1b0e26p-35));
    double p = 0x1.6124613a86d09p-33;                 // 1/13!
    p = d_add(d_mul(p, r), 0x1.1eed8eff8d898p-29);    // 1/12!
    p = d_add(d_mul(p, r), 0x1.ae64567f544e4p-26);    // 1/11!
    p = d_add(d_mul(p, r), 0x1.27e4fb7789f5cp-22);    // 1/10!
    p = d_add(d_mul(p, r), 0x1.71de3a556c734p-19);    // 1/9!
    p = d_add(d_mul(p, r), 0x1.a01a01a01a01ap-16);    // 1/8!
    p = d_add(d_mul(p, r), 0x1.a01a01a01a01ap-13);    // 1/7!
    p = d_add(d_mul(p, r), 0x1.6c16c16c16c17p-10);    // 1/6!
    p = d_add(d_mul(p, r), 0x1.1111111111111p-7);     // 1/5!
    p = d_add(d_mul(p, r), 0x1.5555555555555p-5);     // 1/4!
    p = d_add(d_mul(p, r), 0x1.5555555555555p-3);     // 1/3!
    p = d_add(d_mul(p, r), 0x1.0p-1);                 // 1/2!
    p = d_add(d_mul(p, r), 1.0);                      // 1/1!
    p = d_add(d_mul(p, r), 1.0);                      // 1/0!
    // 2^k is exact and the product stays normal for k >= -34
    return d_mul(p, __hiloint2double((1023 + (int)kd) << 20, 0));
}

// ---- stochastic time increment (mixed PR algorithm, step 3c) ----
// Every binary64 operation below is one round-to-nearest step in a fixed
// order, so the host oracle's C code gives the same bits.

// Natural logarithm of a normal x > 0: x = 2^k m with m in [sqrt(1/2),
// sqrt(2)); ln m = 2 atanh(f), f = (m - 1)/(m + 1) (|f| <= 0.1716), by the
// odd series of atanh to f^23 (the next term is below 3e-21);
// ln x = k LN2_HI + (k LN2_LO + ln m), LN2_HI holding 29 significant bits.
__device__ __forceinline__ double cg_log(double x)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int k = (int)((b >> 52) & 0x7ffull) - 1023;
    b = (b & 0x000fffffffffffffull) | 0x3ff0000000000000ull;   // m in [1, 2)
    double m = __longlong_as_double((long long)b);
    if (m > 0x1.6a09e667f3bcdp+0) {                             // sqrt(2)
        m = d_mul(m, 0.5);
        k += 1;
    }
    const double f = d_div(d_sub(m, 1.0), d_add(m, 1.0));
    const double s = d_mul(f, f);
    double p = 0x1.642c8590b2164p-5;               // 1/23
    p = d_add(d_mul(p, s), 0x1.8618618618618p-5);  // 1/21
    p = d_add(d_mul(p, s), 0x1.af286bca1af28p-5);  // 1/19
    p = d_add(d_mul(p, s), 0x1.e1e1e1e1e1e1ep-5);  // 1/17
    p = d_add(d_mul(p, s), 0x1.1111111111111p-4);  // 1/15
    p = d_add(d_mul(p, s), 0x1.3b13b13b13b14p-4);  // 1/13
    p = d_add(d_mul(p, s), 0x1.745d1745d1746p-4);  // 1/11
    p = d_add(d_mul(p, s), 0x1.c71c71c71c71cp-4);  // 1/9
    p = d_add(d_mul(p, s), 0x1.2492492492492p-3);  // 1/7
    p = d_add(d_mul(p, s), 0x1.999999999999ap-3);  // 1/5
    p = d_add(d_mul(p, s), 0x1.5555555555555p-2);  // 1/3
    p = d_add(d_mul(p, s), 1.0);
    const double lm = d_mul(d_mul(2.0, f), p);
    const double kd = (double)k;
    return d_add(d_mul(kd, 0x1.62e42ffp-1), d_add(d_mul(kd, -0x1.718432a1b0e26p-35), lm));
}

// cos(2 pi u) for u in [0, 1): v = u - rint(u), q = rint(4 v) and
// w = v - q/4 in [-1/8, 1/8] are exact; theta = 2 pi w; cos(2 pi u) is
// cos(theta), -sin(theta), -cos(theta) or sin(theta) for q = 0, 1, 2, 3
// (mod 4), from the Taylor series of cos to theta^16 and of sin to
// theta^17 on |theta| <= pi/4.
__device__ __forceinline__ double cg_cos2pi(double u)
{
    const double v = d_sub(u, rint(u));
    const double q = rint(d_mul(4.0, v));
    const double w = d_sub(v, d_mul(0.25, q));
    const double t = d_mul(0x1.921fb54442d18p+2, w);   // 2 pi
    const double s = d_mul(t, t);
    const int qi = ((int)q) & 3;
    double p, r;
    if (qi == 0 || qi == 2) {
        p = 0x1.ae7f3e733b81fp-45;                        //  1/16!
        p = d_add(d_mul(p, s), -0x1.93974a8c07c9dp-37);   // -1/14!
        p = d_add(d_mul(p, s), 0x1.1eed8eff8d898p-29);    //  1/12!
        p = d_add(d_mul(p, s), -0x1.27e4fb7789f5cp-22);   // -1/10!
        p = d_add(d_mul(p, s), 0x1.a01a01a01a01ap-16);    //  1/8!
        p = d_add(d_mul(p, s), -0x1.6c16c16c16c17p-10);   // -1/6!
        p = d_add(d_mul(p, s), 0x1.5555555555555p-5);     //  1/4!
        p = d_add(d_mul(p, s), -0x1.0p-1);                // -1/2!
        r = d_add(d_mul(p, s), 1.0);
    } else {
        p = 0x1.952c77030ad4ap-49;                        //  1/17!
        p = d_add(d_mul(p, s), -0x1.ae7f3e733b81fp-41);   // -1/15!
        p = d_add(d_mul(p, s), 0x1.6124613a86d09p-33);    //  1/13!
        p = d_add(d_mul(p, s), -0x1.ae64567f544e4p-26);   // -1/11!
        p = d_add(d_mul(p, s), 0x1.71de3a556c734p-19);    //  1/9!
        p = d_add(d_mul(p, s), -0x1.a01a01a01a01ap-13);   // -1/7!
        p = d_add(d_mul(p, s), 0x1.1111111111111p-7);     //  1/5!
        p = d_add(d_mul(p, s), -0x1.5555555555555p-3);    // -1/3!
        p = d_add(d_mul(p, s), 1.0);
        r = d_mul(t, p);
    }
    return (qi == 1 || qi == 2) ? -r : r;
}

// Standard normal deviate of executed hop h of a replica: Box-Muller on the
// Philox block of counter (h lo, h hi, 0xFFFFFFFE, replica) under the
// replica's key, z = sqrt(-2 ln u1) cos(2 pi u2), u1 = (x0 + 1/2) 2^-32,
// u2 = x1 2^-32.
__device__ __forceinline__ double cg_gauss(uint32_t key0, uint32_t key1, uint32_t replica,
                                           unsigned long long h)
{
    uint32_t x[4];
    philox4x32_10((uint32_t)h, (uint32_t)(h >> 32), 0xFFFFFFFEu, replica, key0, key1, x);
    const double u1 = d_mul(d_add((double)x[0], 0.5), 0x1p-32);
    const double u2 = d_mul((double)x[1], 0x1p-32);
    return d_mul(__dsqrt_rn(d_mul(-2.0, cg_log(u1))), cg_cos2pi(u2));
}

// max(0, (m + sqrt(m) z) / Gamma): the time increment of one executed hop
// that took m attempts.
__device__ __forceinline__ double cg_time_increment(double Gamma, unsigned long long m, double z)
{
    const double dm = (double)m;
    double d = d_add(dm, d_mul(__dsqrt_rn(dm), z));
    if (d < 0.0) d = 0.0;
    return d_div(d, Gamma);
}

// Minimum-image |d| on a ring of length L for d in (-L, L).
__host__ __device__ __forceinline__ int fold_axis(int d, int L)
{
    d += (d < 0) ? L : 0;
    const int e = L - d;
    return d < e ? d : e;
}

}  // namespace cg
