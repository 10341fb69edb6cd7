// cg_pr_cluster.cuh -- the persistent parallel-rejection kernel for lattices
// whose local energies do not fit one CTA's shared memory (e.g. L = 256 in
// binary32, 256 KiB of eps): one replica per thread-block cluster of C CTAs.
//
// Same chain as cg_pr_kernel.cu (mixed PR algorithm, steps 1-3); the work of
// a replica is spread over the cluster:
//   * on the square lattice CTA `rank` owns the base rows
//     [rank B, (rank+1) B), B = L/(2C), and their partner rows y + L/2 of eps
//     in its shared memory (local row yl < B is base row rank B + yl, yl >= B
//     the partner of base row rank B + yl - B), so each CTA updates its sites
//     four at a time with one folded offset per axis, as the single-CTA
//     kernel does; the 1/r table, the occupation bitmask and the tower are
//     replicated in every CTA, and every CTA applies each executed hop to its
//     bitmask copy;
//   * a chunk of labels is split into C contiguous sub-ranges, CTA rank
//     evaluating sub-range rank; eps_i and eps_j of a proposal are read from
//     the owning CTA's shared memory through distributed shared memory;
//   * each CTA finds its lowest accepting label (OR barrier, ballot, warp
//     minimum), then thread 0 writes it and its payload into every CTA's
//     exchange slot (double-buffered by chunk parity); one cluster barrier
//     later every CTA holds all C candidates and takes the minimum, so the
//     executed hop is the lowest accepting label of the whole chunk;
//   * each CTA updates its own rows; a cluster barrier ends the hop so that
//     the next hop's remote reads see updated energies.
// On the L x L x L cubic lattice (kDim = 3) CTA `rank` owns the z-planes
// [rank L/C, (rank+1) L/C) instead of rows, and every CTA holds the
// (L/2+1)^3 folded table.  With two-electron hops (kPair, square lattice) the
// four energies of a pair label come through distributed shared memory, the
// second electron of each CTA's candidate travels in a second exchange slot,
// and an executed pair applies the two single-hop updates to the CTA's rows
// in turn.
// The wall-clock limit of a hop is decided by rank 0 and published in its
// exchange slot, so every exit decision is uniform over the cluster.
// On the cubic lattice with single hops the update reads 1/r indexed by
// r^2 = fx^2 + fy^2 + fz^2 of the folded offsets (3 (L/2)^2 + 1 entries, the
// folded table's own values: 1/r depends on r^2 alone) instead of the
// (L/2+1)^3 folded table: 12 KiB instead of 144 KiB at L = 64 in binary32,
// where the folded table fits beside no share of eps.  The labels never read
// either table (their 1/r comes from the per-vector tables).
#pragma once

#include <cooperative_groups.h>

#include "cg_pr_common.cuh"

namespace coop = cooperative_groups;

namespace cg {

struct Slot {
    unsigned int label;      // lowest accepting label of the sending CTA, or ~0
    unsigned int late;       // rank 0 only: the hop ran past its time limit
    Cand cand;
};

// Square lattice: the CTA that owns row y and the row's local index there
// (base rows of B = L/(2C) per CTA, partner rows y + L/2 after them);
// magicB = floor(2^32 / B) + 1 divides by B for y < L <= 1024 when B >= 2;
// B = 1 (L = 2C), where that multiplier would need 33 bits, has magicB = 0
// and owner = y mod L/2.
__device__ __forceinline__ void cluster_row_owner(int y, int Lh, int B, unsigned magicB,
                                                  unsigned &owner, int &yl)
{
    const bool upper = y >= Lh;
    const int yb = upper ? y - Lh : y;
    owner = magicB ? __umulhi((unsigned)yb, magicB) : (unsigned)yb;
    yl = yb - (int)owner * B + (upper ? B : 0);
}

// Global row of local row yl of CTA rank (square lattice).
__device__ __forceinline__ int cluster_global_row(int yl, unsigned rank, int Lh, int B)
{
    return yl < B ? (int)rank * B + yl : Lh + (int)rank * B + (yl - B);
}

// eps of site s, from the CTA that owns its row (square lattice) or z-plane
// (cubic lattice: CTA rank owns planes [rank L/C, (rank+1) L/C)).
template <typename Real, int kDim>
__device__ __forceinline__ Real cluster_eps(coop::cluster_group &cl, Real *local, unsigned s,
                                            int rows_local, int log2L, int L, unsigned magic,
                                            bool pow2, unsigned rank, unsigned magicB)
{
    unsigned owner, off;
    if (kDim == 3) {
        const int z = pow2 ? (int)(s >> (2 * log2L)) : (int)__umulhi(__umulhi(s, magic), magic);
        owner = (unsigned)(z / rows_local);
        off = s - owner * (unsigned)rows_local * (unsigned)(L * L);
    } else {
        const int y = pow2 ? (int)(s >> log2L) : (int)__umulhi(s, magic);
        const int x = (int)s - y * L;
        int yl;
        cluster_row_owner(y, L >> 1, rows_local >> 1, magicB, owner, yl);
        off = (unsigned)(yl * L + x);
    }
    if (owner == rank) return local[off];
    Real *peer = cl.map_shared_rank(local, owner);
    return peer[off];
}

template <typename Real, int kThreads, bool kPow2, int kDim, bool kPair = false>
__global__ void __launch_bounds__(kThreads, 1)
pr_cluster(const DevReplica *__restrict__ reps, const int *__restrict__ index, RunArgs a)
{
    // the update's 1/r indexed by r^2 (cubic lattice, single hops)
    constexpr bool kR2 = kDim == 3 && !kPair;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int s_wlabel[32];
    __shared__ Cand s_cand[32];
    // step-3c deviates of the next hops (CG_TIME_GAUSSIAN): warp 0 draws 32
    // at a time, one per lane, so the binary64 Box-Muller chain runs once
    // per 32 hops instead of on thread 0's path at every commit
    __shared__ double s_z[32];
    __shared__ unsigned long long s_zbase;
    __shared__ Slot s_slot[2][8];
    __shared__ PairProp s_pcand[kPair ? 32 : 1];          // pair data of each warp's candidate
    __shared__ PairProp s_pslot[kPair ? 2 : 1][kPair ? 8 : 1];   // ... of each CTA's
    __shared__ struct {
        unsigned long long hops, attempts, evaluated, cyc_rej, cyc_upd, wall0;
        long long P, t0;
        double energy, time;
        float m_ema;
    } s_c;

    coop::cluster_group cl = coop::this_cluster();
    const unsigned rank = cl.block_rank(), C = cl.num_blocks();
    const DevReplica &Rg = reps[index[blockIdx.x / C]];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = Rg.L, N = Rg.N, H1 = Rg.H1, V = Rg.V, words = Rg.words;
    const unsigned magic = Rg.magicL;
    const uint32_t key0 = Rg.key0, key1 = Rg.key1, rep = Rg.replica;
    const double T = Rg.T, E = Rg.E;
    const float invTf = (float)(1.0 / T);
    // rows (square lattice) or z-planes (cubic lattice) of this CTA
    const int plane = kDim == 3 ? L * L : L;
    const int rows_local = L / (int)C, N_local = rows_local * plane;
    const int row0 = (int)rank * rows_local;
    const int log2L = __ffs(L) - 1;
    // square lattice: base rows per CTA and the multiplier that divides by it
    const int Bq = rows_local >> 1;
    const unsigned magicB =
        (kDim == 3 || Bq < 2) ? 0u : (unsigned)(4294967296ull / (unsigned)Bq + 1ull);
    const int ntab = kR2 ? 3 * (L >> 1) * (L >> 1) + 1 : kDim == 3 ? H1 * H1 * H1 : H1 * H1;

    const SmemLayout lay = smem_layout(N_local, ntab, V, words, (int)sizeof(Real));
    Shared S;
    S.eps = smem + lay.off_eps;
    S.tinv = smem + lay.off_tinv;
    S.occ = reinterpret_cast<unsigned *>(smem + lay.off_occ);
    S.guide = reinterpret_cast<unsigned short *>(smem + lay.off_guide);
    S.thr = reinterpret_cast<unsigned *>(smem + lay.off_thr);
    S.disp = reinterpret_cast<int *>(smem + lay.off_disp);
    S.vr64 = reinterpret_cast<double *>(smem + lay.off_vr64);
    S.edx64 = reinterpret_cast<double *>(smem + lay.off_edx64);
    S.cv32 = reinterpret_cast<float *>(smem + lay.off_cv32);
    Real *eps = reinterpret_cast<Real *>(S.eps);
    const Real *tinv = reinterpret_cast<const Real *>(S.tinv);

    // ---- stage: own rows of eps, full tables and bitmask ----
    {
        if (kDim == 3) {
            const Real *eps_g = reinterpret_cast<const Real *>(Rg.eps) + (size_t)row0 * plane;
            for (int l = tid; l < N_local; l += kThreads) eps[l] = eps_g[l];
        } else {
            const Real *eps_g = reinterpret_cast<const Real *>(Rg.eps);
            for (int l = tid; l < N_local; l += kThreads) {
                const int yl = kPow2 ? (l >> log2L) : (int)__umulhi((unsigned)l, magic);
                const int x = l - yl * L;
                eps[l] = eps_g[(size_t)cluster_global_row(yl, rank, L >> 1, Bq) * L + x];
            }
        }
        const Real *tab_g =
            (sizeof(Real) == 8)
                ? reinterpret_cast<const Real *>(kR2 ? Rg.tinv_r2_64 : Rg.tinv64)
                : reinterpret_cast<const Real *>(kR2 ? Rg.tinv_r2_32 : Rg.tinv32);
        Real *tab_s = reinterpret_cast<Real *>(S.tinv);
        for (int l = tid; l < ntab; l += kThreads) tab_s[l] = tab_g[l];
        for (int l = tid; l < words; l += kThreads) S.occ[l] = Rg.occ[l];
        for (int l = tid; l < kGuide; l += kThreads) S.guide[l] = Rg.guide[l];
        for (int l = tid; l < V; l += kThreads) {
            const int dxy = Rg.disp[l];
            // dx of the packed vector (10-bit fields on the cubic lattice)
            const int dx = kDim == 3 ? (dxy << 22) >> 22 : (int)(short)(dxy & 0xffff);
            S.thr[l] = Rg.thr[l];
            S.disp[l] = dxy;
            S.vr64[l] = Rg.tinvd[l];
            S.edx64[l] = d_mul(E, (double)dx);
            S.cv32[l] = (float)d_add(Rg.tinvd[l], S.edx64[l]);   // one rounding to binary32
        }
    }
    DevCounters *cnt = Rg.ctr;
    unsigned long long rounds = cnt->rounds;
    if (tid == 0) {
        s_c.hops = cnt->hops;
        s_c.attempts = cnt->attempts;
        s_c.evaluated = cnt->evaluated;
        s_c.P = cnt->P;
        s_c.energy = cnt->energy;
        s_c.time = cnt->time;
        s_c.m_ema = cnt->m_ema > 0.f ? cnt->m_ema : 64.0f;
        s_c.cyc_rej = 0;
        s_c.cyc_upd = 0;
    }
    int status = CG_OK;
    unsigned parity = 0;
    cl.sync();   // every CTA staged before any remote read

    const unsigned M = a.M;
    const unsigned thr_last = S.thr[V - 1];
    const int rows_per_pass = kThreads / L;
    const int active = rows_per_pass * L;
    const int ux = tid % L, uy0 = tid / L;
    // square lattice update: base rows per pass and the threads that work
    const int qrpp = kThreads / (L >> 1);
    const int qactive = qrpp * (L >> 1);

    if (tid == 0) s_zbase = ~0ull;
    __syncthreads();
    for (unsigned long long h = 0; h < a.n_hops; ++h) {
        if (a.time_mode && warp == 0) {
            // s_c.hops was last written before the previous hop's final barrier
            const unsigned long long hcur = s_c.hops;
            if (hcur < s_zbase || hcur - s_zbase >= 32ull) {
                s_z[lane] = cg_gauss(key0, key1, rep, hcur + (unsigned long long)lane);
                __syncwarp();
                if (lane == 0) s_zbase = hcur;
                __syncwarp();
            }
        }
        if (tid == 0) {
            s_c.t0 = clock64();
            s_c.wall0 = globaltimer_ns();
        }
        // cluster chunk: C sub-chunks of up to 2 * blockDim labels, ~ sqrt(2 m b)
        // labels in all for m expected labels and a chunk's fixed cost b (its
        // two CTA barriers and the cluster barrier; ~1000 labels measured)
        unsigned sub = 64;
        {
            const float want = sqrtf(2048.0f * s_c.m_ema) / (float)C;
            while (sub < (unsigned)(2 * kThreads) && (float)sub < want) sub <<= 1;
        }
        const unsigned chunk = sub * C, half = sub >> 1;
        unsigned long long p = 0;
        unsigned q = 0;
        Cand win{};
        PairProp wpq{};                    // the executed hop's second electron (kPair)
        wpq.pair = false;
        bool found = false;
        while (!found) {
            ++p;
            const PhiloxPrefix PP =
                philox_prefix((uint32_t)rounds, (uint32_t)(rounds >> 32), rep, key0, key1);
            PhiloxPrefix PP2{};
            if (kPair)
                PP2 = philox_prefix((uint32_t)rounds, (uint32_t)(rounds >> 32) | 0x80000000u, rep,
                                    key0, key1);
            for (unsigned kb = 0; kb < M; kb += chunk) {
                const unsigned base = kb + rank * sub;
                const bool mine = (unsigned)tid < half;
                const unsigned k0 = base + (unsigned)tid, k1 = k0 + half;
                Prop p0{}, p1{};
                PairProp q0{}, q1{};
                double dE0 = 0.0, dE1 = 0.0;
                bool acc0 = false, acc1 = false;
                Real ei0 = 0, ej0 = 0, ei1 = 0, ej1 = 0;
                Real ek0 = 0, el0 = 0, ek1 = 0, el1 = 0;
                // the threads past the CTA's sub-chunk (whole warps: half is a
                // multiple of 32) skip the label work
                if (mine) {
                p0 = propose<kPow2, kDim>(S, k0, PP, key0, key1, L, log2L, (unsigned)N, magic,
                                          thr_last, k0 < M);
                p1 = propose<kPow2, kDim>(S, k1, PP, key0, key1, L, log2L, (unsigned)N, magic,
                                          thr_last, k1 < M);
                if (kPair && !a.toy) {
                    q0 = pair_extend<kPow2, kDim>(S, p0, k0, PP2, key0, key1, L, log2L, magic, thr_last,
                                            Rg.pair_T, Rg.pair_R);
                    q1 = pair_extend<kPow2, kDim>(S, p1, k1, PP2, key0, key1, L, log2L, magic, thr_last,
                                            Rg.pair_T, Rg.pair_R);
                }
                if (a.toy) {
                    const double u0 = d_mul(d_add((double)p0.x2, 0.5), 0x1p-32);
                    const double u1 = d_mul(d_add((double)p1.x2, 0.5), 0x1p-32);
                    acc0 = k0 < M && u0 < a.toy_A0;
                    acc1 = k1 < M && u1 < a.toy_A0;
                } else {
                    if (p0.theta) {
                        ei0 = cluster_eps<Real, kDim>(cl, eps, p0.i, rows_local, log2L, L, magic, kPow2, rank, magicB);
                        ej0 = cluster_eps<Real, kDim>(cl, eps, p0.j, rows_local, log2L, L, magic, kPow2, rank, magicB);
                        if (kPair && q0.pair) {
                            ek0 = cluster_eps<Real, kDim>(cl, eps, q0.k, rows_local, log2L, L, magic, kPow2, rank, magicB);
                            el0 = cluster_eps<Real, kDim>(cl, eps, q0.l, rows_local, log2L, L, magic, kPow2, rank, magicB);
                            acc0 = accept_pair_vals<Real, kPow2, kDim>(ei0, ej0, ek0, el0, S, Rg, p0, q0, T,
                                                                 invTf, dE0, L, log2L, magic, H1);
                        } else {
                            acc0 = accept_vals<Real>(ei0, ej0, S, p0, T, invTf, dE0);
                        }
                    }
                    if (p1.theta) {
                        ei1 = cluster_eps<Real, kDim>(cl, eps, p1.i, rows_local, log2L, L, magic, kPow2, rank, magicB);
                        ej1 = cluster_eps<Real, kDim>(cl, eps, p1.j, rows_local, log2L, L, magic, kPow2, rank, magicB);
                        if (kPair && q1.pair) {
                            ek1 = cluster_eps<Real, kDim>(cl, eps, q1.k, rows_local, log2L, L, magic, kPow2, rank, magicB);
                            el1 = cluster_eps<Real, kDim>(cl, eps, q1.l, rows_local, log2L, L, magic, kPow2, rank, magicB);
                            acc1 = accept_pair_vals<Real, kPow2, kDim>(ei1, ej1, ek1, el1, S, Rg, p1, q1, T,
                                                                 invTf, dE1, L, log2L, magic, H1);
                        } else {
                            acc1 = accept_vals<Real>(ei1, ej1, S, p1, T, invTf, dE1);
                        }
                    }
                }
                }
                const int any = __syncthreads_or(acc0 || acc1);
                unsigned best = 0xffffffffu;
                if (any) {
                    const unsigned b0 = __ballot_sync(0xffffffffu, acc0);
                    const unsigned b1 = __ballot_sync(0xffffffffu, acc1);
                    unsigned off = 0xffffffffu;
                    if (b0) {
                        const int first = __ffs(b0) - 1;
                        off = (unsigned)(warp * 32 + first);
                        if (lane == first) {
                            s_cand[warp].i = p0.i;
                            s_cand[warp].j = p0.j;
                            s_cand[warp].dxy = p0.dxy;
                            s_cand[warp].dE =
                                a.toy ? 0.0
                                : (kPair && q0.pair)
                                    ? pair_hop_dE_vals<Real, kPow2, kDim>(ei0, ej0, ek0, el0, S, Rg, p0,
                                                                    q0, dE0, L, log2L, magic, H1)
                                    : hop_dE_vals<Real>(ei0, ej0, S, p0, dE0);
                            if (kPair) s_pcand[warp] = q0;
                        }
                    } else if (b1) {
                        const int first = __ffs(b1) - 1;
                        off = half + (unsigned)(warp * 32 + first);
                        if (lane == first) {
                            s_cand[warp].i = p1.i;
                            s_cand[warp].j = p1.j;
                            s_cand[warp].dxy = p1.dxy;
                            s_cand[warp].dE =
                                a.toy ? 0.0
                                : (kPair && q1.pair)
                                    ? pair_hop_dE_vals<Real, kPow2, kDim>(ei1, ej1, ek1, el1, S, Rg, p1,
                                                                    q1, dE1, L, log2L, magic, H1)
                                    : hop_dE_vals<Real>(ei1, ej1, S, p1, dE1);
                            if (kPair) s_pcand[warp] = q1;
                        }
                    }
                    if (lane == 0) s_wlabel[warp] = off;
                    __syncthreads();
                    unsigned wl = (lane < kThreads / 32) ? s_wlabel[lane] : 0xffffffffu;
#pragma unroll
                    for (int o = 16; o; o >>= 1) wl = min(wl, __shfl_xor_sync(0xffffffffu, wl, o));
                    best = wl;
                }
                // publish this CTA's candidate (and rank 0's clock decision)
                if (tid == 0) {
                    Slot sl;
                    sl.label = (best == 0xffffffffu) ? 0xffffffffu : base + best;
                    sl.late = (rank == 0) &&
                              (globaltimer_ns() - s_c.wall0) > a.hop_timeout_ns;
                    PairProp pq{};
                    pq.pair = false;
                    if (best != 0xffffffffu) {
                        sl.cand = s_cand[(best >= half ? best - half : best) >> 5];
                        if (kPair) pq = s_pcand[(best >= half ? best - half : best) >> 5];
                    }
                    for (unsigned r = 0; r < C; ++r) {
                        Slot *dst = cl.map_shared_rank(&s_slot[parity][rank], r);
                        *dst = sl;
                        if (kPair) {
                            PairProp *pd = cl.map_shared_rank(&s_pslot[kPair ? parity : 0][kPair ? rank : 0], r);
                            *pd = pq;
                        }
                    }
                    s_c.evaluated += (M - kb < chunk) ? (M - kb) : chunk;
                }
                cl.sync();
                unsigned gbest = 0xffffffffu, gwin = 0;
                for (unsigned r = 0; r < C; ++r) {
                    const unsigned lab = s_slot[parity][r].label;
                    if (lab < gbest) { gbest = lab; gwin = r; }
                }
                const bool late = s_slot[parity][0].late != 0;
                if (gbest != 0xffffffffu) {
                    q = gbest + 1;
                    win = s_slot[parity][gwin].cand;
                    if (kPair) wpq = s_pslot[kPair ? parity : 0][kPair ? gwin : 0];
                    found = true;
                }
                parity ^= 1u;
                if (found) break;
                if (late) {
                    status = CG_ETIMEOUT;
                    break;
                }
            }
            if (status != CG_OK) break;
            if (!found) {
                if (tid == 0) s_c.attempts += M;
                rounds += 1;
                if (p >= a.max_rounds) {
                    status = CG_ESTUCK;
                    break;
                }
            }
        }
        if (!found) break;

        // ---- commit (step 3a, 3c): every CTA flips its bitmask copy ----
        const unsigned ci = win.i, cj = win.j;
        const int cdx = kDim == 3 ? (win.dxy << 22) >> 22 : (int)(short)(win.dxy & 0xffff);
        const int cdy = kDim == 3 ? (win.dxy << 12) >> 22 : win.dxy >> 16;
        const bool cpair = kPair && !a.toy && wpq.pair;
        const int cdx2 = !cpair ? 0 : kDim == 3 ? (wpq.dxy2 << 22) >> 22 : (int)(short)(wpq.dxy2 & 0xffff);
        const int cdy2 = !cpair ? 0 : kDim == 3 ? (wpq.dxy2 << 12) >> 22 : wpq.dxy2 >> 16;
        long long t1 = 0;
        if (tid == 0) {
            const unsigned long long m_hop = (p - 1) * (unsigned long long)M + q;
            if (a.time_mode)     // step 3c: Gaussian dt of hop number s_c.hops
                s_c.time = d_add(s_c.time, cg_time_increment(Rg.Gamma, m_hop,
                                                            s_z[s_c.hops - s_zbase]));
            s_c.m_ema = 0.9f * s_c.m_ema + 0.1f * (float)m_hop;
            s_c.attempts += q;
            s_c.hops += 1;
            if (!a.toy) {
                s_c.P += cdx + cdx2;
                s_c.energy = d_add(s_c.energy, win.dE);
            }
            if (rank == 0)
                trace_hop(Rg, s_c.attempts, s_c.hops, s_c.P, s_c.energy, a.time_mode, s_c.time);
            t1 = clock64();
            s_c.cyc_rej += (unsigned long long)(t1 - s_c.t0);
            if (rank == 0 && Rg.log) {
                cg_hop e;
                e.i = ci; e.j = cj; e.q = q; e.p = (uint32_t)p; e.round = rounds;
                e.dx = a.toy ? 0 : cdx; e.dy = a.toy ? 0 : cdy;
                e.dE = a.toy ? 0.0 : win.dE;
                e.k = cpair ? wpq.k : 0xFFFFFFFFu;
                e.l = cpair ? wpq.l : 0xFFFFFFFFu;
                e.dx2 = cdx2;
                e.dy2 = cdy2;
                Rg.log[a.log_offset + h] = e;
            }
            if (!a.toy) {
                S.occ[ci >> 5] &= ~(1u << (ci & 31));
                S.occ[cj >> 5] |= (1u << (cj & 31));
                if (cpair) {
                    S.occ[wpq.k >> 5] &= ~(1u << (wpq.k & 31));
                    S.occ[wpq.l >> 5] |= (1u << (wpq.l & 31));
                }
            }
        }
        rounds += 1;

        // ---- local-energy update of this CTA's rows (step 3b) ----
        if (kDim == 3 && !a.toy && tid < active) {
            // thread -> column x = ux of the (z, y) rows uy0, uy0 + rows_per_pass,
            // ... of this CTA's planes (row r = zl L + y, site r L + x); an
            // executed pair applies the second electron's update after the
            // first one's
#pragma unroll 1
            for (int pass = 0; pass < (cpair ? 2 : 1); ++pass) {
            const unsigned ui = pass ? wpq.k : ci, uj = pass ? wpq.l : cj;
            int xi, yi, zi, xj, yj, zj;
            if (kPow2) {
                const int m = L - 1;
                xi = (int)ui & m; yi = (int)(ui >> log2L) & m; zi = (int)(ui >> (2 * log2L));
                xj = (int)uj & m; yj = (int)(uj >> log2L) & m; zj = (int)(uj >> (2 * log2L));
            } else {
                const unsigned qi = __umulhi(ui, magic), qj = __umulhi(uj, magic);
                xi = (int)(ui - qi * (unsigned)L); zi = (int)__umulhi(qi, magic);
                yi = (int)qi - zi * L;
                xj = (int)(uj - qj * (unsigned)L); zj = (int)__umulhi(qj, magic);
                yj = (int)qj - zj * L;
            }
            const int fxj = fold_axis(ux - xj, L), fxi = fold_axis(ux - xi, L);
            if constexpr (kR2) {
                const int qj = fxj * fxj, qi = fxi * fxi;
                for (int r = uy0; r < rows_local * L; r += rows_per_pass) {
                    const int zl = kPow2 ? (r >> log2L) : (int)__umulhi((unsigned)r, magic);
                    const int y = r - zl * L, z = row0 + zl;
                    const int fzj = fold_axis(z - zj, L), fyj = fold_axis(y - yj, L);
                    const int fzi = fold_axis(z - zi, L), fyi = fold_axis(y - yi, L);
                    Real *e = eps + r * L + ux;
                    *e = Prec<Real>::add(*e, Prec<Real>::sub(tinv[qj + fyj * fyj + fzj * fzj],
                                                             tinv[qi + fyi * fyi + fzi * fzi]));
                }
            } else {
                for (int r = uy0; r < rows_local * L; r += rows_per_pass) {
                    const int zl = kPow2 ? (r >> log2L) : (int)__umulhi((unsigned)r, magic);
                    const int y = r - zl * L, z = row0 + zl;
                    const int oj = (fold_axis(z - zj, L) * H1 + fold_axis(y - yj, L)) * H1 + fxj;
                    const int oi = (fold_axis(z - zi, L) * H1 + fold_axis(y - yi, L)) * H1 + fxi;
                    Real *e = eps + r * L + ux;
                    *e = Prec<Real>::add(*e, Prec<Real>::sub(tinv[oj], tinv[oi]));
                }
            }
            }
        } else if (kDim == 2 && !a.toy && tid < qactive) {
            // thread -> base column bx < L/2 and base rows yb0, yb0 + qrpp, ...
            // of this CTA; each base site (x, y) serves the four sites
            // (x, y), (x + L/2, y), (x, y + L/2), (x + L/2, y + L/2) (local rows
            // yb and yb + B): on an even ring fold(d + L/2) = L/2 - fold(d).
            // An executed pair applies the second electron's update after the
            // first one's (each site rounds twice, in the serial order).
            const int passes = cpair ? 2 : 1;
            const int Lh = L >> 1;
            const int bx = tid % Lh, yb0 = tid / Lh;
#pragma unroll 1
            for (int pass = 0; pass < passes; ++pass) {
                const unsigned ui = pass ? wpq.k : ci, uj = pass ? wpq.l : cj;
                int yi, xi, yj, xj;
                if (kPow2) {
                    yi = (int)(ui >> log2L); xi = (int)ui & (L - 1);
                    yj = (int)(uj >> log2L); xj = (int)uj & (L - 1);
                } else {
                    yi = (int)__umulhi(ui, magic); xi = (int)ui - yi * L;
                    yj = (int)__umulhi(uj, magic); xj = (int)uj - yj * L;
                }
                const int fxj = fold_axis(bx - xj, L), fxi = fold_axis(bx - xi, L);
                // columns of (x, .) and (x + L/2, .) relative to j and to i
                const Real *cj0 = tinv + fxj, *cj1 = tinv + (Lh - fxj);
                const Real *ci0 = tinv + fxi, *ci1 = tinv + (Lh - fxi);
                const int LhH1 = Lh * H1, BL = Bq * L;
                Real *e = eps + yb0 * L + bx;
#pragma unroll 4
                for (int yb = yb0; yb < Bq; yb += qrpp, e += qrpp * L) {
                    const int y = (int)rank * Bq + yb;
                    int fyj, fyi;
                    if (kPow2) {
                        const int dj = (y - yj) & (L - 1), di = (y - yi) & (L - 1);
                        fyj = min(dj, L - dj);
                        fyi = min(di, L - di);
                    } else {
                        fyj = fold_axis(y - yj, L);
                        fyi = fold_axis(y - yi, L);
                    }
                    // rows fold(y - .) and L/2 - fold(y - .) = fold(y + L/2 - .)
                    const int oj0 = fyj * H1, oj1 = LhH1 - oj0;
                    const int oi0 = fyi * H1, oi1 = LhH1 - oi0;
                    const Real a00 = cj0[oj0], b00 = ci0[oi0];
                    const Real a10 = cj1[oj0], b10 = ci1[oi0];
                    const Real a01 = cj0[oj1], b01 = ci0[oi1];
                    const Real a11 = cj1[oj1], b11 = ci1[oi1];
                    e[0] = Prec<Real>::add(e[0], Prec<Real>::sub(a00, b00));
                    e[Lh] = Prec<Real>::add(e[Lh], Prec<Real>::sub(a10, b10));
                    e[BL] = Prec<Real>::add(e[BL], Prec<Real>::sub(a01, b01));
                    e[BL + Lh] = Prec<Real>::add(e[BL + Lh], Prec<Real>::sub(a11, b11));
                }
            }
        }
        cl.sync();   // updated rows visible to every peer before the next hop
        if (tid == 0) s_c.cyc_upd += (unsigned long long)(clock64() - t1);
    }

    // ---- store back: own rows of eps; rank 0 the bitmask and counters ----
    {
        if (kDim == 3) {
            Real *eps_g = reinterpret_cast<Real *>(Rg.eps) + (size_t)row0 * plane;
            for (int l = tid; l < N_local; l += kThreads) eps_g[l] = eps[l];
        } else {
            Real *eps_g = reinterpret_cast<Real *>(Rg.eps);
            for (int l = tid; l < N_local; l += kThreads) {
                const int yl = kPow2 ? (l >> log2L) : (int)__umulhi((unsigned)l, magic);
                const int x = l - yl * L;
                eps_g[(size_t)cluster_global_row(yl, rank, L >> 1, Bq) * L + x] = eps[l];
            }
        }
        if (rank == 0)
            for (int l = tid; l < words; l += kThreads) Rg.occ[l] = S.occ[l];
    }
    if (tid == 0 && rank == 0) {
        cnt->rounds = rounds;
        cnt->hops = s_c.hops;
        cnt->attempts = s_c.attempts;
        cnt->evaluated = s_c.evaluated;
        cnt->P = s_c.P;
        cnt->energy = s_c.energy;
        cnt->time = s_c.time;
        cnt->cycles_reject += s_c.cyc_rej;
        cnt->cycles_update += s_c.cyc_upd;
        cnt->m_ema = s_c.m_ema;
        cnt->status = status;
    }
    cl.sync();   // no CTA leaves while a peer may still read its shared memory
}

}  // namespace cg
