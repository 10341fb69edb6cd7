// cg_pr_random.cuh -- the label of the random-site chain (partner lookup,
// theta, the binary64 energy change), shared by the single-CTA kernel
// (cg_pr_random.cu) and its cluster form (cg_pr_random_cluster.cu).
#pragma once

#include "cg_pr_common.cuh"

namespace cg {

struct RCand {
    unsigned i, j;
    double dE;
};

// Running weight C_m <= 2^32 of a packed pair record {C_m mod 2^32,
// partner | (C_m >> 32) << 31}.
__device__ __forceinline__ unsigned long long pair_weight(uint2 r)
{
    return (unsigned long long)r.x | ((unsigned long long)(r.y >> 31) << 32);
}

struct RLabel {
    unsigned i, j, m, x2;
    double2 gx;               // 1/r_ij and E dx_ij of partner m
    bool theta;
};

// Label k's site, partner and theta.  An empty site i has theta = 0 whatever
// its partner, so the partner is looked up for occupied sites only: the
// smallest m of i's list with x1 < C_m.  One 64-byte load of i's guide record
// gives the list's bounds, its last running weight (x1 at or above it: a null
// proposal) and the bucket of pairs x1 >> 29 can select; a four-way search
// (three independent probes per step) narrows the bucket to at most four
// records, and the last scan reads whole records, so the partner comes with
// its running weight; 1/r and E dx of each scanned record are loaded beside
// it, so the chosen partner's come with no further dependent load.
// gsm: the compacted guide records in shared memory (two uint4 per site:
// {first, last lo, length | last hi << 16, 0} and the 16 bucket starts as
// bytes), or null for the 64-byte records in global memory.
__device__ __forceinline__ RLabel propose_random(const DevReplica &Rg, const unsigned *occ,
                                                 unsigned k, const PhiloxPrefix &PP,
                                                 uint32_t key0, uint32_t key1, unsigned N,
                                                 bool valid, const uint4 *gsm = nullptr)
{
    RLabel p;
    p.theta = false;
    p.i = p.j = p.m = 0;
    p.x2 = 0;
    p.gx = make_double2(0.0, 0.0);
    if (!valid) return p;
    uint32_t x[4];
    philox_finish(k, PP, key0, key1, x);
    p.i = __umulhi(x[0], N);
    p.x2 = x[2];
    if (!((occ[p.i >> 5] >> (p.i & 31)) & 1u)) return p;
    const unsigned long long x1 = x[1];
    const unsigned b = x[1] >> 28, b1 = b + 1;
    int first, end, glo, ghi;
    unsigned long long last;
    if (gsm) {
        const uint4 ra = gsm[2 * p.i], rb = gsm[2 * p.i + 1];
        first = (int)ra.x;
        end = first + (int)(ra.z & 0xffffu);
        last = (unsigned long long)ra.y | ((unsigned long long)((ra.z >> 16) & 1u) << 32);
        if (first == end || x1 >= last) return p;
        // byte b of words 4..7: the start of bucket b
        const unsigned wb = (b >> 2) == 0 ? rb.x : (b >> 2) == 1 ? rb.y : (b >> 2) == 2 ? rb.z : rb.w;
        const unsigned wb1 = (b1 >> 2) == 0 ? rb.x : (b1 >> 2) == 1 ? rb.y
                           : (b1 >> 2) == 2 ? rb.z : rb.w;
        glo = first + (int)((wb >> (8 * (b & 3))) & 0xffu);
        ghi = b1 < (unsigned)kRandomBuckets ? first + (int)((wb1 >> (8 * (b1 & 3))) & 0xffu) : end;
    } else {
        const int4 *g4 = reinterpret_cast<const int4 *>(Rg.rguide + (size_t)p.i * kRandomGuide);
        const int4 ga = __ldg(g4), gb = __ldg(g4 + 1), gc = __ldg(g4 + 2);
        first = ga.x;
        end = ga.y;                                        // [0] and [1]
        last = (unsigned long long)(uint32_t)ga.z | ((unsigned long long)(uint32_t)ga.w << 32);
        if (first == end || x1 >= last) return p;
        // the 16-bit starts of buckets b = x1 >> 28 and b + 1 (words [4..11]
        // in gb, gc; bucket 16 starts at the list's end)
        const unsigned w0 = (b >> 1) < 4 ? (unsigned)((b >> 1) == 0 ? gb.x : (b >> 1) == 1 ? gb.y
                                                      : (b >> 1) == 2 ? gb.z : gb.w)
                                         : (unsigned)((b >> 1) == 4 ? gc.x : (b >> 1) == 5 ? gc.y
                                                      : (b >> 1) == 6 ? gc.z : gc.w);
        const unsigned w1 = (b1 >> 1) < 4 ? (unsigned)((b1 >> 1) == 0 ? gb.x : (b1 >> 1) == 1 ? gb.y
                                                       : (b1 >> 1) == 2 ? gb.z : gb.w)
                                          : (unsigned)((b1 >> 1) == 4 ? gc.x : (b1 >> 1) == 5 ? gc.y
                                                       : (b1 >> 1) == 6 ? gc.z : gc.w);
        glo = first + (int)((b & 1) ? (w0 >> 16) : (w0 & 0xffffu));
        ghi = b1 < (unsigned)kRandomBuckets
                  ? first + (int)((b1 & 1) ? (w1 >> 16) : (w1 & 0xffffu))
                  : end;
    }
    int lo = glo, hi = min(ghi, end - 1) + 1;
    const uint2 *rc = Rg.rrec;
    // the answer lies in [lo, hi); record m holds C_m in 33 bits
    while (hi - lo > 4) {
        const int q = (hi - lo) >> 2;
        const int m1 = lo + q, m2 = m1 + q, m3 = m2 + q;
        const unsigned long long c1 = pair_weight(__ldg(rc + m1)), c2 = pair_weight(__ldg(rc + m2)),
                                 c3 = pair_weight(__ldg(rc + m3));
        if (x1 < c1) {
            hi = m1 + 1;
        } else if (x1 < c2) {
            lo = m1 + 1;
            hi = m2 + 1;
        } else if (x1 < c3) {
            lo = m2 + 1;
            hi = m3 + 1;
        } else {
            lo = m3 + 1;
        }
    }
    // the records with x1 < C_m form a suffix of [lo, hi): walking down, the
    // last one that holds is the smallest
    int m = hi - 1;
    unsigned j = __ldg(rc + m).y & 0x7fffffffu;
    double2 gx = __ldg(Rg.rgx + m);
#pragma unroll
    for (int t = 1; t <= 3; ++t) {
        const int mt = hi - 1 - t;
        if (mt >= lo) {
            const uint2 r = __ldg(rc + mt);
            const double2 gt = __ldg(Rg.rgx + mt);
            if (x1 < pair_weight(r)) {
                m = mt;
                j = r.y & 0x7fffffffu;
                gx = gt;
            }
        }
    }
    p.m = (unsigned)m;
    p.j = j;
    p.gx = gx;
    p.theta = !((occ[p.j >> 5] >> (p.j & 31)) & 1u);     // n_i = 1 here
    return p;
}

// dH = ((eps_j - eps_i) - 1/r_ij) - E dx_ij, each step rounded (binary64)
__device__ __forceinline__ double dE_random_vals(double ei, double ej, const RLabel &p)
{
    return d_sub(d_sub(d_sub(ej, ei), p.gx.x), p.gx.y);
}

__device__ __forceinline__ double dE_random(const DevReplica &Rg, const double *eps,
                                            const RLabel &p)
{
    return dE_random_vals(eps[p.i], eps[p.j], p);
}

// Stage the compacted guide records of all N sites into shared memory (two
// uint4 per site, from the 64-byte records; every list below 256 pairs).
template <int kThreads>
__device__ __forceinline__ void stage_guide(uint4 *gsm, const DevReplica &Rg, int N, int tid)
{
    for (int s = tid; s < N; s += kThreads) {
        const int4 *g4 = reinterpret_cast<const int4 *>(Rg.rguide + (size_t)s * kRandomGuide);
        const int4 ga = g4[0], gb = g4[1], gc = g4[2];
        const unsigned w16[8] = {(unsigned)gb.x, (unsigned)gb.y, (unsigned)gb.z, (unsigned)gb.w,
                                 (unsigned)gc.x, (unsigned)gc.y, (unsigned)gc.z, (unsigned)gc.w};
        unsigned bytes[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int b = 0; b < kRandomBuckets; ++b) {
            const unsigned off = (b & 1) ? (w16[b >> 1] >> 16) : (w16[b >> 1] & 0xffffu);
            bytes[b >> 2] |= (off & 0xffu) << (8 * (b & 3));
        }
        gsm[2 * s] = make_uint4((unsigned)ga.x, (unsigned)ga.z,
                                (unsigned)(ga.y - ga.x) | (((unsigned)ga.w & 1u) << 16), 0u);
        gsm[2 * s + 1] = make_uint4(bytes[0], bytes[1], bytes[2], bytes[3]);
    }
}

}  // namespace cg
