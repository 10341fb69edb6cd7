// cg_device.cuh -- arithmetic building blocks of libcg shared by its host
// set-up code and its kernels: Philox-4x32-10, the acceptance exponential,
// minimum-image folding.  Every binary64 operation that feeds the chain is
// written with an explicit round-to-nearest intrinsic on the device, so the
// compiler cannot fuse a multiply and an add into one FMA.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cg {

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
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
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
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1;
    P.A = c3 ^ k1;
    // round 2 (keys bumped once): the product of word 0 is shared
    const uint32_t k0b = k0 + 0x9E3779B9u, k1b = k1 + 0xBB67AE85u;
    P.B = __umulhi(0xD2511F53u, n0) ^ k1b;
    P.x3 = 0xD2511F53u * n0;
    P.C = n1 ^ k0b;
    return P;
}

__device__ __forceinline__ void philox_finish(uint32_t k, const PhiloxPrefix &P, uint32_t k0,
                                              uint32_t k1, uint32_t out[4])
{
    // round 1, the k-dependent half
    const uint32_t n2 = __umulhi(0xD2511F53u, k) ^ P.A, n3 = 0xD2511F53u * k;
    // round 2, the n2-dependent half
    uint32_t c0 = __umulhi(0xCD9E8D57u, n2) ^ P.C;
    uint32_t c1 = 0xCD9E8D57u * n2;
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
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
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

// Minimum-image |d| on a ring of length L for d in (-L, L).
__host__ __device__ __forceinline__ int fold_axis(int d, int L)
{
    d += (d < 0) ? L : 0;
    const int e = L - d;
    return d < e ? d : e;
}

}  // namespace cg
