// cg_pr_common.cuh -- per-label building blocks of the persistent PR kernels
// (single CTA and thread-block cluster): Philox proposal, tower sampling,
// theta, and the Metropolis test in binary64 and binary32.
#pragma once

#include "cg_device.cuh"
#include "cg_internal.h"

namespace cg {

struct Cand {
    unsigned int i, j;
    int dxy;
    unsigned int pad_;
    double dE;
};

template <typename Real>
struct Prec;

template <>
struct Prec<double> {
    static __device__ __forceinline__ double add(double a, double b) { return d_add(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return d_sub(a, b); }
};

template <>
struct Prec<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
};

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Binary32 value of a binary64 from its high word: truncated to 20 mantissa
// bits (relative error < 2^-20); integer operations only.  Returns 0 when
// |x| < 2^-126 (callers fall back to the exact path).
__device__ __forceinline__ float approx_f32(double x)
{
    const int hi = __double2hiint(x);
    const int ex = (hi >> 20) & 0x7ff;
    if (ex < 1023 - 126 || ex > 1023 + 127) return 0.0f;
    const unsigned bits = ((unsigned)hi & 0x80000000u) | ((unsigned)(ex - 896) << 23) |
                          (((unsigned)hi & 0xfffffu) << 3);
    return __uint_as_float(bits);
}

struct Shared {
    void *eps;
    void *tinv;
    unsigned *occ;
    unsigned short *guide;
    unsigned *thr;
    int *disp;
    double *vr64, *edx64;     // 1/r_v and E dx_v (binary64)
    float *cv32;              // 1/r_v + E dx_v rounded once to binary32
};

// Tower sampling: the smallest vector index v with x1 <= thr[v] (thr[v] =
// C_v - 1, C the integer cumulative weights), for x1 <= thr[V-1].  The guide
// bucket of x1's top bits holds the first candidate; one threshold inside
// the bucket costs a predicated compare, several (rare) a scan.
__device__ __forceinline__ int tower_lookup(const unsigned short *guide, const unsigned *thr,
                                            uint32_t x1)
{
    const unsigned g = guide[x1 >> (32 - kGuideBits)];
    int v = (int)(g & 0x3fffu);
    const unsigned t0 = thr[v];
    v += (int)(((g >> 15) & 1u) & (unsigned)(x1 > t0));
    if (g & 0x4000u)
        while (x1 > thr[v]) ++v;
    return v;
}

struct Prop {
    unsigned i, j;
    int v, dxy;
    uint32_t x2;
    uint32_t x3;              // fourth word: the pair decision of two-electron hops
    bool theta;
};

// Step 1 of one label (Philox, site, tower, destination) and theta.  P is the
// Philox prefix of the label's round (counter words 1-3); kPow2 selects shift
// and mask site arithmetic when L is a power of two (log2L its exponent).
template <bool kPow2, int kDim = 2>
__device__ __forceinline__ Prop propose(const Shared &S, unsigned k, const PhiloxPrefix &P,
                                        uint32_t key0, uint32_t key1, int L, int log2L,
                                        unsigned N, unsigned magic, unsigned thr_last,
                                        bool valid)
{
    Prop p;
    uint32_t x[4];
    philox_finish(k, P, key0, key1, x);
    p.x2 = x[2];
    p.x3 = x[3];
    p.i = kPow2 ? (x[0] >> (32 - kDim * log2L)) : __umulhi(x[0], N);   // floor(x0 N / 2^32)
    // a label beyond M or a null proposal (x1 above the last threshold) is
    // evaluated on a clamped x1 without a branch and can never pass theta
    const uint32_t x1 = min(x[1], thr_last);
    const bool live = valid && x[1] <= thr_last;
    const int v = tower_lookup(S.guide, S.thr, x1);
    const int dxy = S.disp[v];
    if (kDim == 3) {
        // cubic lattice: 10-bit fields dx | dy << 10 | dz << 20, site
        // s = (z L + y) L + x
        const int dx = (dxy << 22) >> 22, dy = (dxy << 12) >> 22, dz = dxy >> 20;
        int xi, yi, zi;
        if (kPow2) {
            const int m = L - 1;
            xi = (int)p.i & m;
            yi = (int)(p.i >> log2L) & m;
            zi = (int)(p.i >> (2 * log2L));
            const int xj = (xi + dx) & m, yj = (yi + dy) & m, zj = (zi + dz) & m;
            p.j = (unsigned)((((zj << log2L) | yj) << log2L) | xj);
        } else {
            const unsigned q = __umulhi(p.i, magic);
            xi = (int)(p.i - q * (unsigned)L);
            zi = (int)__umulhi(q, magic);
            yi = (int)q - zi * L;
            int xj = xi + dx, yj = yi + dy, zj = zi + dz;
            xj += (xj < 0) ? L : 0;
            xj -= (xj >= L) ? L : 0;
            yj += (yj < 0) ? L : 0;
            yj -= (yj >= L) ? L : 0;
            zj += (zj < 0) ? L : 0;
            zj -= (zj >= L) ? L : 0;
            p.j = (unsigned)((zj * L + yj) * L + xj);
        }
    } else {
        const int dx = (int)(short)(dxy & 0xffff), dy = dxy >> 16;
        if (kPow2) {
            const int Lm = L - 1;
            const int xj = ((int)p.i + dx) & Lm;
            const int yj = (((int)p.i >> log2L) + dy) & Lm;
            p.j = (unsigned)((yj << log2L) | xj);
        } else {
            const int yi = (int)__umulhi(p.i, magic), xi = (int)p.i - yi * L;
            int xj = xi + dx, yj = yi + dy;
            xj += (xj < 0) ? L : 0;
            xj -= (xj >= L) ? L : 0;
            yj += (yj < 0) ? L : 0;
            yj -= (yj >= L) ? L : 0;
            p.j = (unsigned)(yj * L + xj);
        }
    }
    p.v = v;
    p.dxy = dxy;
    const unsigned wi = S.occ[p.i >> 5], wj = S.occ[p.j >> 5];
    p.theta = live && ((wi >> (p.i & 31)) & 1u) && !((wj >> (p.j & 31)) & 1u);
    return p;
}

// Binary32 Metropolis bound of the binary32 form: e^(-dH/T) 2^23 - 1/2, with
// e^(-dH/T) = 2^(dH c), c = -log2(e)/T folded into one constant (the
// multiply by it is loop-invariant), from the hardware's approximate 2^x.
__device__ __forceinline__ float metropolis_bound_f32(float dE, float invTf)
{
    const float c = -invTf * 1.44269504088896341f;
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(dE * c));
    return __fmaf_rn(e, 0x1p23f, -0.5f);
}

// Step 2 (accept test) for a proposal whose theta holds, from the two local
// energies (read from this CTA's shared memory or a cluster peer's).
template <typename Real>
__device__ __forceinline__ bool accept_vals(Real ei, Real ej, const Shared &S, const Prop &p,
                                            double T, float invTf, double &dE_out);

template <>
__device__ __forceinline__ bool accept_vals<double>(double ei, double ej, const Shared &S,
                                                    const Prop &p, double T, float invTf,
                                                    double &dE_out)
{
    double d = d_sub(ej, ei);
    d = d_sub(d, S.vr64[p.v]);
    const double dE = d_sub(d, S.edx64[p.v]);
    dE_out = dE;
    if (dE <= 0.0) return true;
    // binary32 estimate of y = -dE/T and of e^y, then a margin test
    const float df = approx_f32(dE);
    if (df > 0.0f) {
        const float y = -df * invTf;
        if (y < -23.01f) return false;                      // e^y below every u
        const float e = __expf(y);
        // u ~ x2 2^-32 differs from (x2 + 1/2) 2^-32 by at most 2^-33 plus a
        // relative 2^-24: the absolute slack 2^-31 covers the first, the
        // relative margin the second and the exponential's error
        const float u = __uint2float_rn(p.x2) * 0x1p-32f;
        if (u + 0x1p-31f < e * (1.0f - 2e-4f)) return true;
        if (u > e * (1.0f + 2e-4f) + 0x1p-31f) return false;
    }
    const double u = d_mul(d_add((double)p.x2, 0.5), 0x1p-32);
    return u < cg_exp_accept(d_div(-dE, T));
}

template <>
__device__ __forceinline__ bool accept_vals<float>(float ei, float ej, const Shared &S,
                                                   const Prop &p, double T, float invTf,
                                                   double &dE_out)
{
    const float dEf = __fsub_rn(__fsub_rn(ej, ei), S.cv32[p.v]);
    if (fabsf(dEf) < 1e-5f) {
        // near tie: decide in binary64 from the widened energies
        double d = d_sub((double)ej, (double)ei);
        d = d_sub(d, S.vr64[p.v]);
        const double dE = d_sub(d, S.edx64[p.v]);
        dE_out = dE;
        if (dE <= 0.0) return true;
        const double u = d_mul(d_add((double)p.x2, 0.5), 0x1p-32);
        return u < cg_exp_accept(d_div(-dE, T));
    }
    dE_out = 0.0;   // widened for the executed hop only
    if (dEf <= 0.0f) return true;
    // u = (m + 1/2) 2^-23 with m = x2 >> 9 (exact in binary32); u < e^(-dH/T)
    // tested as m < e 2^23 - 1/2
    return (float)(p.x2 >> 9) < metropolis_bound_f32(dEf, invTf);
}

// Step 2 for the two labels of a thread in the binary32 form, without a
// branch per label: the energies are read for every label (its sites are
// valid even when theta fails) and theta masks the result, so the two
// dependency chains interleave.  Near ties (|dH| < 1e-5) are re-decided in
// binary64 by accept_vals<float>.
__device__ __forceinline__ void accept2_f32(const Shared &S, const Prop &p0, const Prop &p1,
                                            double T, float invTf, bool &acc0, bool &acc1,
                                            double &dE0, double &dE1)
{
    const float *eps = reinterpret_cast<const float *>(S.eps);
    const float d0 = __fsub_rn(__fsub_rn(eps[p0.j], eps[p0.i]), S.cv32[p0.v]);
    const float d1 = __fsub_rn(__fsub_rn(eps[p1.j], eps[p1.i]), S.cv32[p1.v]);
    const float t0 = metropolis_bound_f32(d0, invTf);
    const float t1 = metropolis_bound_f32(d1, invTf);
    acc0 = p0.theta && (d0 <= 0.0f || (float)(p0.x2 >> 9) < t0);
    acc1 = p1.theta && (d1 <= 0.0f || (float)(p1.x2 >> 9) < t1);
    dE0 = 0.0;
    dE1 = 0.0;
    const bool tie0 = p0.theta && fabsf(d0) < 1e-5f, tie1 = p1.theta && fabsf(d1) < 1e-5f;
    if (tie0 || tie1) {
        if (tie0) acc0 = accept_vals<float>(eps[p0.i], eps[p0.j], S, p0, T, invTf, dE0);
        if (tie1) acc1 = accept_vals<float>(eps[p1.i], eps[p1.j], S, p1, T, invTf, dE1);
    }
}

// ---------------------------------------------------------------------------
// Two-electron hops.  A label whose fourth word x3 is below pair_T proposes a
// pair: from the Philox block of counter (k, r lo, r hi | 2^31, replica), y0
// and y2 give the offset e = (floor(y0 W / 2^32) - R, floor(y2 W / 2^32) - R),
// W = 2R + 1, of the second electron k = i + e, and y1 its hop vector d2 by
// the same tower, l = k + d2.  theta also needs n_k = 1, n_l = 0,
// 0 < |e|^2 <= R^2 and 0 < |e'|^2 <= R^2 for the reverse offset
// e' = e + d2 - d1, so that a pair and its reverse are proposed with the
// same probability.
// ---------------------------------------------------------------------------

struct PairProp {
    unsigned k, l;            // 0xFFFFFFFF for a single hop
    int v2, dxy2;
    bool pair;
};

template <bool kPow2>
__device__ __forceinline__ void site_xy(unsigned s, int L, int log2L, unsigned magic, int &x,
                                        int &y)
{
    y = kPow2 ? (int)(s >> log2L) : (int)__umulhi(s, magic);
    x = (int)s - y * L;
}

// x, y, z of site s = (z L + y) L + x of the cubic lattice
template <bool kPow2>
__device__ __forceinline__ void site_xyz(unsigned s, int L, int log2L, unsigned magic, int &x,
                                         int &y, int &z)
{
    if (kPow2) {
        const int m = L - 1;
        x = (int)s & m;
        y = (int)(s >> log2L) & m;
        z = (int)(s >> (2 * log2L));
    } else {
        const unsigned q = __umulhi(s, magic);      // s / L
        x = (int)(s - q * (unsigned)L);
        z = (int)__umulhi(q, magic);                 // s / L^2
        y = (int)q - z * L;
    }
}

__device__ __forceinline__ int wrap_axis(int c, int L)
{
    c += (c < 0) ? L : 0;
    c -= (c >= L) ? L : 0;
    return c;
}

// kDim = 3: vectors are 10-bit packed, the offset's z comes from y3 and
// sites are (z L + y) L + x.
template <bool kPow2, int kDim = 2>
__device__ __forceinline__ PairProp pair_extend(const Shared &S, Prop &p, unsigned k,
                                                const PhiloxPrefix &P2, uint32_t key0,
                                                uint32_t key1, int L, int log2L, unsigned magic,
                                                unsigned thr_last, uint32_t pair_T, int R)
{
    PairProp q;
    q.k = q.l = 0xFFFFFFFFu;
    q.v2 = 0;
    q.dxy2 = 0;
    q.pair = p.x3 < pair_T;
    if (!q.pair) return q;
    uint32_t y[4];
    philox_finish(k, P2, key0, key1, y);
    const unsigned W = (unsigned)(2 * R + 1);
    const int ex = (int)__umulhi(y[0], W) - R, ey = (int)__umulhi(y[2], W) - R;
    const int ez = kDim == 3 ? (int)__umulhi(y[3], W) - R : 0;
    const bool live2 = y[1] <= thr_last;
    const int v2 = tower_lookup(S.guide, S.thr, min(y[1], thr_last));
    const int dxy2 = S.disp[v2];
    int dx2, dy2, dz2 = 0, dx1, dy1, dz1 = 0;
    if (kDim == 3) {
        dx2 = (dxy2 << 22) >> 22; dy2 = (dxy2 << 12) >> 22; dz2 = dxy2 >> 20;
        dx1 = (p.dxy << 22) >> 22; dy1 = (p.dxy << 12) >> 22; dz1 = p.dxy >> 20;
    } else {
        dx2 = (int)(short)(dxy2 & 0xffff); dy2 = dxy2 >> 16;
        dx1 = (int)(short)(p.dxy & 0xffff); dy1 = p.dxy >> 16;
    }
    int xi, yi, zi = 0;
    if (kDim == 3)
        site_xyz<kPow2>(p.i, L, log2L, magic, xi, yi, zi);
    else
        site_xy<kPow2>(p.i, L, log2L, magic, xi, yi);
    const int xk = wrap_axis(xi + ex, L), yk = wrap_axis(yi + ey, L);
    const int xl = wrap_axis(xk + dx2, L), yl = wrap_axis(yk + dy2, L);
    unsigned ks, ls;
    if (kDim == 3) {
        const int zk = wrap_axis(zi + ez, L), zl = wrap_axis(zk + dz2, L);
        ks = (unsigned)((zk * L + yk) * L + xk);
        ls = (unsigned)((zl * L + yl) * L + xl);
    } else {
        ks = (unsigned)(yk * L + xk);
        ls = (unsigned)(yl * L + xl);
    }
    const int fx = ex + dx2 - dx1, fy = ey + dy2 - dy1, fz = ez + dz2 - dz1;
    const int e2 = ex * ex + ey * ey + ez * ez, f2 = fx * fx + fy * fy + fz * fz, R2 = R * R;
    const unsigned wk = S.occ[ks >> 5], wl = S.occ[ls >> 5];
    const bool ok = live2 && e2 > 0 && e2 <= R2 && f2 > 0 && f2 <= R2 &&
                    ((wk >> (ks & 31)) & 1u) && !((wl >> (ls & 31)) & 1u);
    p.theta = p.theta && ok;
    q.k = ks;
    q.l = ls;
    q.v2 = v2;
    q.dxy2 = dxy2;
    return q;
}

// 1/r between sites a and b from a folded table [fy * H1 + fx], or
// [(fz * H1 + fy) * H1 + fx] on the cubic lattice.
template <typename T, bool kPow2, int kDim = 2>
__device__ __forceinline__ T tinv_sites(const T *tab, unsigned a, unsigned b, int L, int log2L,
                                        unsigned magic, int H1)
{
    if (kDim == 3) {
        int xa, ya, za, xb, yb, zb;
        site_xyz<kPow2>(a, L, log2L, magic, xa, ya, za);
        site_xyz<kPow2>(b, L, log2L, magic, xb, yb, zb);
        return tab[(fold_axis(za - zb, L) * H1 + fold_axis(ya - yb, L)) * H1 +
                   fold_axis(xa - xb, L)];
    }
    int xa, ya, xb, yb;
    site_xy<kPow2>(a, L, log2L, magic, xa, ya);
    site_xy<kPow2>(b, L, log2L, magic, xb, yb);
    return tab[fold_axis(ya - yb, L) * H1 + fold_axis(xa - xb, L)];
}

// dH of the pair i -> j, k -> l in binary64, in the serial chain's order:
// (dH1 + dH2) + ((1/r_lj - 1/r_li) - (1/r_kj - 1/r_ki)), each dH as R9.
template <bool kPow2, int kDim = 2>
__device__ __forceinline__ double pair_dE64(const Shared &S, const double *tab64, double ei,
                                            double ej, double ek, double el, const Prop &p,
                                            const PairProp &q, int L, int log2L,
                                            unsigned magic, int H1)
{
    const double d1 = d_sub(d_sub(d_sub(ej, ei), S.vr64[p.v]), S.edx64[p.v]);
    const double d2 = d_sub(d_sub(d_sub(el, ek), S.vr64[q.v2]), S.edx64[q.v2]);
    const double tlj = tinv_sites<double, kPow2, kDim>(tab64, q.l, p.j, L, log2L, magic, H1);
    const double tli = tinv_sites<double, kPow2, kDim>(tab64, q.l, p.i, L, log2L, magic, H1);
    const double tkj = tinv_sites<double, kPow2, kDim>(tab64, q.k, p.j, L, log2L, magic, H1);
    const double tki = tinv_sites<double, kPow2, kDim>(tab64, q.k, p.i, L, log2L, magic, H1);
    return d_add(d_add(d1, d2), d_sub(d_sub(tlj, tli), d_sub(tkj, tki)));
}

// The Metropolis decision u < e^(-dH/T) for dH > 0 in binary64 semantics
// (a binary32 estimate with a margin decides most cases).
__device__ __forceinline__ bool metropolis64(double dE, uint32_t x2, double T, float invTf)
{
    if (dE <= 0.0) return true;
    const float df = approx_f32(dE);
    if (df > 0.0f) {
        const float y = -df * invTf;
        if (y < -23.01f) return false;
        const float e = __expf(y);
        const float u = __uint2float_rn(x2) * 0x1p-32f;
        if (u + 0x1p-31f < e * (1.0f - 2e-4f)) return true;
        if (u > e * (1.0f + 2e-4f) + 0x1p-31f) return false;
    }
    const double u = d_mul(d_add((double)x2, 0.5), 0x1p-32);
    return u < cg_exp_accept(d_div(-dE, T));
}

// Step 2 for a pair whose theta holds.  Binary64: exact dH.  Binary32: the
// same sum in binary32 from the binary32 table, re-decided in binary64 from
// the widened energies and the binary64 table when |dH| < 1e-5 (dE_out is
// then the binary64 value, else 0: the executed pair is widened once).
template <typename Real, bool kPow2, int kDim = 2>
__device__ __forceinline__ bool accept_pair_vals(Real ei, Real ej, Real ek, Real el,
                                                 const Shared &S, const DevReplica &Rg,
                                                 const Prop &p, const PairProp &q, double T,
                                                 float invTf, double &dE_out, int L, int log2L,
                                                 unsigned magic, int H1)
{
    if (sizeof(Real) == 8) {
        const double dE = pair_dE64<kPow2, kDim>(S, reinterpret_cast<const double *>(S.tinv),
                                                 (double)ei, (double)ej, (double)ek, (double)el,
                                                 p, q, L, log2L, magic, H1);
        dE_out = dE;
        return metropolis64(dE, p.x2, T, invTf);
    }
    const float *t32 = reinterpret_cast<const float *>(S.tinv);
    const float d1 = __fsub_rn(__fsub_rn((float)ej, (float)ei), S.cv32[p.v]);
    const float d2 = __fsub_rn(__fsub_rn((float)el, (float)ek), S.cv32[q.v2]);
    const float cr = __fsub_rn(
        __fsub_rn(tinv_sites<float, kPow2, kDim>(t32, q.l, p.j, L, log2L, magic, H1),
                  tinv_sites<float, kPow2, kDim>(t32, q.l, p.i, L, log2L, magic, H1)),
        __fsub_rn(tinv_sites<float, kPow2, kDim>(t32, q.k, p.j, L, log2L, magic, H1),
                  tinv_sites<float, kPow2, kDim>(t32, q.k, p.i, L, log2L, magic, H1)));
    const float dEf = __fadd_rn(__fadd_rn(d1, d2), cr);
    if (fabsf(dEf) < 1e-5f) {
        const double dE = pair_dE64<kPow2, kDim>(S, Rg.tinv64, (double)ei, (double)ej,
                                                 (double)ek, (double)el, p, q, L, log2L, magic, H1);
        dE_out = dE;
        return metropolis64(dE, p.x2, T, invTf);
    }
    dE_out = 0.0;
    if (dEf <= 0.0f) return true;
    return (float)(p.x2 >> 9) < __fmaf_rn(__expf(-dEf * invTf), 0x1p23f, -0.5f);
}

template <typename Real, bool kPow2, int kDim = 2>
__device__ __forceinline__ bool accept_pair(const Shared &S, const DevReplica &Rg, const Prop &p,
                                            const PairProp &q, double T, float invTf,
                                            double &dE_out, int L, int log2L, unsigned magic,
                                            int H1)
{
    const Real *eps = reinterpret_cast<const Real *>(S.eps);
    return accept_pair_vals<Real, kPow2, kDim>(eps[p.i], eps[p.j], eps[q.k], eps[q.l], S, Rg, p, q, T,
                                         invTf, dE_out, L, log2L, magic, H1);
}

// dH of an executed pair in binary64 (binary32 form: from the widened
// energies and the binary64 table, once per hop).
template <typename Real, bool kPow2, int kDim = 2>
__device__ __forceinline__ double pair_hop_dE_vals(Real ei, Real ej, Real ek, Real el,
                                                   const Shared &S, const DevReplica &Rg,
                                                   const Prop &p, const PairProp &q, double dE,
                                                   int L, int log2L, unsigned magic, int H1)
{
    if (sizeof(Real) == 8 || dE != 0.0) return dE;
    return pair_dE64<kPow2, kDim>(S, Rg.tinv64, (double)ei, (double)ej, (double)ek, (double)el, p,
                                  q, L, log2L, magic, H1);
}

template <typename Real, bool kPow2, int kDim = 2>
__device__ __forceinline__ double pair_hop_dE(const Shared &S, const DevReplica &Rg,
                                              const Prop &p, const PairProp &q, double dE,
                                              int L, int log2L, unsigned magic, int H1)
{
    const Real *eps = reinterpret_cast<const Real *>(S.eps);
    return pair_hop_dE_vals<Real, kPow2, kDim>(eps[p.i], eps[p.j], eps[q.k], eps[q.l], S, Rg, p, q,
                                         dE, L, log2L, magic, H1);
}

template <typename Real>
__device__ __forceinline__ bool accept(const Shared &S, const Prop &p, double T, float invTf,
                                       double &dE_out)
{
    const Real *eps = reinterpret_cast<const Real *>(S.eps);
    return accept_vals<Real>(eps[p.i], eps[p.j], S, p, T, invTf, dE_out);
}

// dH of the executed hop in binary64 (the binary32 form widens it here, once
// per hop, instead of on every label).
template <typename Real>
__device__ __forceinline__ double hop_dE_vals(Real ei, Real ej, const Shared &S, const Prop &p,
                                              double dE)
{
    if (sizeof(Real) == 8 || dE != 0.0) return dE;
    const float dEf = __fsub_rn(__fsub_rn((float)ej, (float)ei), S.cv32[p.v]);
    return (double)dEf;
}

template <typename Real>
__device__ __forceinline__ double hop_dE(const Shared &S, const Prop &p, double dE)
{
    const Real *eps = reinterpret_cast<const Real *>(S.eps);
    return hop_dE_vals<Real>(eps[p.i], eps[p.j], S, p, dE);
}

// dH of an accepting label in binary64, redone for the executed hop from its
// proposal: the value the accept test computed (binary64 form; binary32 near
// ties) or the binary32 dH widened.
template <typename Real>
__device__ __forceinline__ double winner_dE(const Shared &S, const Prop &p, double T, float invTf)
{
    double dE = 0.0;
    accept<Real>(S, p, T, invTf, dE);
    return hop_dE<Real>(S, p, dE);
}

}  // namespace cg
