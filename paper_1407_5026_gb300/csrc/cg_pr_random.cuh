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
__device__ __forceinline__ RLabel propose_random(const DevReplica &Rg, const unsigned *occ,
                                                 unsigned k, const PhiloxPrefix &PP,
                                                 uint32_t key0, uint32_t key1, unsigned N,
                                                 bool valid)
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
    const int4 *g4 = reinterpret_cast<const int4 *>(Rg.rguide + (size_t)p.i * kRandomGuide);
    const int4 ga = __ldg(g4), gb = __ldg(g4 + 1), gc = __ldg(g4 + 2);
    const int first = ga.x, end = ga.y;                    // [0] and [1]
    const unsigned long long last =
        (unsigned long long)(uint32_t)ga.z | ((unsigned long long)(uint32_t)ga.w << 32);
    if (first == end || x1 >= last) return p;
    // the 16-bit starts of buckets b = x1 >> 28 and b + 1 (words [4..11] in
    // gb, gc; bucket 16 starts at the list's end)
    const unsigned b = x[1] >> 28;
    const unsigned w0 = (b >> 1) < 4 ? (unsigned)((b >> 1) == 0 ? gb.x : (b >> 1) == 1 ? gb.y
                                                  : (b >> 1) == 2 ? gb.z : gb.w)
                                     : (unsigned)((b >> 1) == 4 ? gc.x : (b >> 1) == 5 ? gc.y
                                                  : (b >> 1) == 6 ? gc.z : gc.w);
    const unsigned b1 = b + 1;
    const unsigned w1 = (b1 >> 1) < 4 ? (unsigned)((b1 >> 1) == 0 ? gb.x : (b1 >> 1) == 1 ? gb.y
                                                   : (b1 >> 1) == 2 ? gb.z : gb.w)
                                      : (unsigned)((b1 >> 1) == 4 ? gc.x : (b1 >> 1) == 5 ? gc.y
                                                   : (b1 >> 1) == 6 ? gc.z : gc.w);
    const int glo = first + (int)((b & 1) ? (w0 >> 16) : (w0 & 0xffffu));
    const int ghi = b1 < (unsigned)kRandomBuckets
                        ? first + (int)((b1 & 1) ? (w1 >> 16) : (w1 & 0xffffu))
                        : end;
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

}  // namespace cg
