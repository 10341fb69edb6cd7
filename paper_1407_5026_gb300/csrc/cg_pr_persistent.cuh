// cg_pr_persistent.cuh -- the persistent parallel-rejection kernel (template;
// instantiated for the square lattice in cg_pr_kernel.cu and for the cubic
// lattice in cg_pr_kernel3d.cu).
//
// One CTA runs one disorder replica for a whole launch.  Its local energies
// eps (N values), the folded minimum-image 1/r table, the occupation bitmask
// and the tower (thresholds + a guide table) live in shared memory; global
// memory is touched only to load the state at the start and store it at the
// end.
//
// Per executed hop (mixed PR algorithm, section "Hopping conduction in the
// Coulomb glass", steps 1-3):
//   rounds r = 0, 1, ...: the M labels of a round are evaluated in chunks of
//   C labels in increasing order, two labels per thread.  Label k draws
//   Philox(key = seed, ctr = (k, r lo, r hi, replica)) -> site i from word 0,
//   hop vector from word 1 by tower sampling, acceptance variate from word 2
//   (step 1 and the three random numbers per label of the GPU paragraph);
//   theta = n_i (1 - n_j) and the Metropolis test on
//   dH = eps_j - eps_i - 1/r_ij - E dx (step 2, Eq. 2).  A chunk with no
//   accept costs one block-wide OR barrier; the first chunk with an accept
//   gives the lowest accepting label q by warp ballot + find-first-set and a
//   minimum over the warps.  Labels after q are never looked at, so the hop
//   equals the serial rejection chain's on the same random numbers.  C follows
//   the replica's recent attempts per hop (C ~ sqrt(128 m), clamped to
//   [64, 2 * blockDim]); it changes which labels are evaluated, never the hop.
//   Commit (step 3a/3c): flip n_i, n_j, P += dx, attempts += (p-1)M + q.
//   Update (step 3b): eps_l += 1/r_lj - 1/r_li for every l, with the table
//   holding 0 at the origin so l = i and l = j need no special case.  A
//   thread takes the four sites (x, y), (x + L/2, y), (x, y + L/2),
//   (x + L/2, y + L/2): on an even ring fold(d + L/2) = L/2 - fold(d), so one
//   folded offset per axis serves all four.
//
// Binary64 form: every operation that feeds the chain is a round-to-nearest
// intrinsic in the serial chain's order, so the trajectory is bit-identical
// to the serial CPU chain.  The Metropolis comparison u < exp(-dH/T) is first
// decided by a binary32 estimate with a relative margin of 2e-4 (ten times
// its error bound); only the undecided cases evaluate the binary64
// exponential, so every decision is the binary64 one.
// Binary32 form: eps, the table and dH in binary32 (dH in binary64 when
// |dH| < 1e-5), exp from the fast intrinsic.
#pragma once

#include "cg_pr_common.cuh"

namespace cg {

// kLog2L: L = 2^kLog2L fixed at compile time (> 0), any power of two (0),
// any even L (-1), or the even L = -kLog2L fixed at compile time (< -1).
// kTime: CG_TIME_GAUSSIAN runs (the step-3c deviates are drawn in the
// kernel); the default deterministic clock compiles without that code.
// kDim: 2 for the L x L square lattice, 3 for the L x L x L cubic lattice
// (site s = (z L + y) L + x; hop vectors packed in 10-bit fields).
// kPair: two-electron hops (square lattice): labels whose fourth Philox word
// is below Rg.pair_T propose a pair move (pair_extend); an executed pair
// applies the two single-hop eps updates in turn.
// 2 b of the chunk rule C ~ sqrt(2 m b) (b: a chunk's fixed cost in labels)
constexpr float kChunkCost = 128.0f;

template <typename Real, int kThreads, int kLog2L, bool kTime, int kDim = 2, bool kPair = false>
__global__ void __launch_bounds__(kThreads, (kThreads >= 1024 ? 1 : 1024 / kThreads))
pr_persistent(const DevReplica *__restrict__ reps, const int *__restrict__ index, RunArgs a)
{
    constexpr bool kPow2 = kLog2L >= 0;
    // L fixed at compile time: 2^kLog2L (kLog2L > 0), or -kLog2L, an even L
    // that is not a power of two (kLog2L < -1); 0 when L is read at run time
    constexpr int kFixL = kLog2L > 0 ? (1 << kLog2L) : (kLog2L < -1 ? -kLog2L : 0);
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int s_wlabel[32];
    __shared__ Cand s_cand[32];
    __shared__ PairProp s_pcand[kPair ? 32 : 1];   // the second electron of a pair candidate
    // step-3c deviates of the next hops (CG_TIME_GAUSSIAN): warp 0 draws 32
    // at a time, one per lane, so the binary64 Box-Muller chain runs once
    // per 32 hops instead of on thread 0's path at every commit
    __shared__ double s_z[32];
    __shared__ unsigned long long s_zbase;
    // counters and pointers only thread 0 uses (registers stay free for the
    // labels)
    __shared__ struct {
        unsigned long long hops, attempts, evaluated, cyc_rej, cyc_upd;
        long long P, t0;
        double energy, time;
        cg_hop *log;
        int tracing;
        float m_ema;
    } s_c;

    const DevReplica &Rg = reps[index[blockIdx.x]];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = kFixL ? kFixL : Rg.L;
    const int N = kDim == 3 ? L * L * L : L * L, H1 = L / 2 + 1, words = (N + 31) / 32;
    const int ntab = kDim == 3 ? H1 * H1 * H1 : H1 * H1;
    const int V = Rg.V;
    // floor(s / L) = umulhi(s, floor(2^32 / L) + 1) for the site indices used;
    // the host computes the same multiplier for run-time L
    const unsigned magic = kPow2  ? 0u
                           : kFixL ? (unsigned)(4294967296ull / (unsigned long long)kFixL + 1ull)
                                   : Rg.magicL;
    const int log2L = kLog2L > 0 ? kLog2L : __ffs(L) - 1;   // used when L is a power of two
    const uint32_t key0 = Rg.key0, key1 = Rg.key1, rep = Rg.replica;
    const double T = Rg.T;
    const float invTf = (float)(1.0 / T);

    const SmemLayout lay = smem_layout(N, ntab, V, words, (int)sizeof(Real));
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

    // ---- stage the replica into shared memory ----
    {
        const Real *eps_g = reinterpret_cast<const Real *>(Rg.eps);
        for (int l = tid; l < N; l += kThreads) eps[l] = eps_g[l];
        const Real *tab_g = (sizeof(Real) == 8)
                                ? reinterpret_cast<const Real *>(Rg.tinv64)
                                : reinterpret_cast<const Real *>(Rg.tinv32);
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
            S.edx64[l] = d_mul(Rg.E, (double)dx);       // E * dx, as in the serial chain
            S.cv32[l] = (float)d_add(Rg.tinvd[l], S.edx64[l]);   // one rounding to binary32
        }
    }
    unsigned long long rounds = Rg.ctr->rounds;
    if (tid == 0) {
        const DevCounters *cnt = Rg.ctr;
        s_c.log = Rg.log;
        s_c.tracing = Rg.trace != nullptr;
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
    __syncthreads();

    const unsigned M = a.M;
    const unsigned thr_last = S.thr[V - 1];

    if (kTime) {
        if (tid == 0) s_zbase = ~0ull;
        __syncthreads();
    }
    for (unsigned long long h = 0; h < a.n_hops; ++h) {
        if (kTime && warp == 0) {
            // s_c.hops was last written before the previous hop's final barrier
            const unsigned long long hcur = s_c.hops;
            if (hcur < s_zbase || hcur - s_zbase >= 32ull) {
                s_z[lane] = cg_gauss(key0, key1, rep, hcur + (unsigned long long)lane);
                __syncwarp();
                if (lane == 0) s_zbase = hcur;
                __syncwarp();
            }
        }
        if (tid == 0) s_c.t0 = clock64();
        // labels per chunk ~ sqrt(2 m b) for m expected labels and a chunk's
        // fixed cost (the OR barrier and the warps' imbalance before it) worth
        // b labels: nl = 4 or 2 labels per thread (C = nl blockDim) when that
        // exceeds blockDim, else one per thread for the first C threads (C a
        // power of two >= 64); m_ema is identical in every thread, so the
        // choice is uniform and idle warps skip the labels whole.  Pair
        // instances take at most two labels per thread.
        const float want = sqrtf(kChunkCost * s_c.m_ema);
        unsigned C, nl;
        if (!kPair && want > 2.0f * (float)kThreads) {
            nl = 4;
            C = 4u * kThreads;
        } else if (want > (float)kThreads) {
            nl = 2;
            C = 2u * kThreads;
        } else {
            nl = 1;
            C = 64;
            while (C < (unsigned)kThreads && (float)C < want) C <<= 1;
            if (C > (unsigned)kThreads) C = kThreads;
        }
        const bool two = nl > 1;
        const bool act = (unsigned)tid < C;
        unsigned long long p = 0;
        unsigned q = 0, win = 0, kb_hit = 0;
        bool found = false;
        while (!found) {
            ++p;
            const PhiloxPrefix PP =
                philox_prefix((uint32_t)rounds, (uint32_t)(rounds >> 32), rep, key0, key1);
            PhiloxPrefix PP2{};
            if (kPair)
                PP2 = philox_prefix((uint32_t)rounds, (uint32_t)(rounds >> 32) | 0x80000000u, rep,
                                    key0, key1);
            if constexpr (!kPair) {
            for (unsigned kb = 0; kb < M; kb += C) {
                // bit u of accm: label kb + u blockDim + tid accepts; only the
                // decisions stay live, the winning lane redoes its proposal
                unsigned accm = 0;
                if (act) {
#pragma unroll
                    for (unsigned u = 0; u < 4; u += 2) {
                        if (u < nl) {
                            const unsigned ka = kb + u * (unsigned)kThreads + (unsigned)tid;
                            const unsigned kc = ka + (unsigned)kThreads;
                            const bool hasc = u + 1 < nl;
                            const bool va = ka < M, vc = hasc && kc < M;
                            const Prop pa = propose<kPow2, kDim>(S, ka, PP, key0, key1, L, log2L,
                                                                 (unsigned)N, magic, thr_last, va);
                            Prop pc{};
                            if (hasc)
                                pc = propose<kPow2, kDim>(S, kc, PP, key0, key1, L, log2L,
                                                          (unsigned)N, magic, thr_last, vc);
                            bool aa = false, ac = false;
                            double da = 0.0, dc = 0.0;
                            if (a.toy) {
                                aa = va && d_mul(d_add((double)pa.x2, 0.5), 0x1p-32) < a.toy_A0;
                                ac = vc && d_mul(d_add((double)pc.x2, 0.5), 0x1p-32) < a.toy_A0;
                            } else if (sizeof(Real) == 4 && hasc) {
                                accept2_f32(S, pa, pc, T, invTf, aa, ac, da, dc);
                            } else {
                                if (pa.theta) aa = accept<Real>(S, pa, T, invTf, da);
                                if (pc.theta) ac = accept<Real>(S, pc, T, invTf, dc);
                            }
                            accm |= (aa ? 1u : 0u) << u;
                            accm |= (ac ? 1u : 0u) << (u + 1);
                        }
                    }
                }
                const int any = __syncthreads_or(accm != 0u);
                if (any) {
                    // the warp's lowest accepting label: the first sub-chunk
                    // u with an accept, then the lowest lane
                    unsigned off = 0xffffffffu;
                    for (unsigned u = 0; u < nl; ++u) {
                        const unsigned bu = __ballot_sync(0xffffffffu, (accm >> u) & 1u);
                        if (bu) {
                            off = u * (unsigned)kThreads + (unsigned)(warp * 32) +
                                  (unsigned)(__ffs(bu) - 1);
                            break;
                        }
                    }
                    if (off != 0xffffffffu && (unsigned)lane == (off & 31u)) {
                        const Prop pw = propose<kPow2, kDim>(S, kb + off, PP, key0, key1, L, log2L,
                                                             (unsigned)N, magic, thr_last, true);
                        s_cand[warp].i = pw.i;
                        s_cand[warp].j = pw.j;
                        s_cand[warp].dxy = pw.dxy;
                        s_cand[warp].dE = a.toy ? 0.0 : winner_dE<Real>(S, pw, T, invTf);
                    }
                    if (lane == 0) s_wlabel[warp] = off;
                    __syncthreads();
                    unsigned wl = (lane < kThreads / 32) ? s_wlabel[lane] : 0xffffffffu;
#pragma unroll
                    for (int o = 16; o; o >>= 1) wl = min(wl, __shfl_xor_sync(0xffffffffu, wl, o));
                    q = kb + wl + 1;                 // 1-based label in the round
                    kb_hit = kb;
                    win = (wl % (unsigned)kThreads) >> 5;
                    found = true;
                    break;
                }
            }
            } else {
            for (unsigned kb = 0; kb < M; kb += C) {
                const unsigned k0 = kb + (unsigned)tid, k1 = k0 + (unsigned)kThreads;
                const bool v0 = k0 < M, v1 = two && k1 < M;
                Prop p0{}, p1{};
                PairProp q0{}, q1{};
                double dE0 = 0.0, dE1 = 0.0;
                bool acc0 = false, acc1 = false;
                if (act) {
                    p0 = propose<kPow2, kDim>(S, k0, PP, key0, key1, L, log2L, (unsigned)N, magic,
                                        thr_last, v0);
                    if (two)
                        p1 = propose<kPow2, kDim>(S, k1, PP, key0, key1, L, log2L, (unsigned)N, magic,
                                            thr_last, v1);
                    if (kPair && !a.toy) {
                        q0 = pair_extend<kPow2, kDim>(S, p0, k0, PP2, key0, key1, L, log2L, magic,
                                                thr_last, Rg.pair_T, Rg.pair_R);
                        if (two)
                            q1 = pair_extend<kPow2, kDim>(S, p1, k1, PP2, key0, key1, L, log2L, magic,
                                                    thr_last, Rg.pair_T, Rg.pair_R);
                    }
                    if (a.toy) {
                        const double u0 = d_mul(d_add((double)p0.x2, 0.5), 0x1p-32);
                        const double u1 = d_mul(d_add((double)p1.x2, 0.5), 0x1p-32);
                        acc0 = v0 && u0 < a.toy_A0;
                        acc1 = v1 && u1 < a.toy_A0;
                    } else if (kPair) {
                        if (p0.theta)
                            acc0 = q0.pair ? accept_pair<Real, kPow2, kDim>(S, Rg, p0, q0, T, invTf, dE0,
                                                                     L, log2L, magic, H1)
                                           : accept<Real>(S, p0, T, invTf, dE0);
                        if (p1.theta)
                            acc1 = q1.pair ? accept_pair<Real, kPow2, kDim>(S, Rg, p1, q1, T, invTf, dE1,
                                                                     L, log2L, magic, H1)
                                           : accept<Real>(S, p1, T, invTf, dE1);
                    } else if (sizeof(Real) == 4 && two) {
                        accept2_f32(S, p0, p1, T, invTf, acc0, acc1, dE0, dE1);
                    } else {
                        if (p0.theta) acc0 = accept<Real>(S, p0, T, invTf, dE0);
                        if (p1.theta) acc1 = accept<Real>(S, p1, T, invTf, dE1);
                    }
                }
                const int any = __syncthreads_or(acc0 || acc1);
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
                            if (kPair) {
                                s_pcand[warp] = q0;
                                s_cand[warp].dE =
                                    a.toy ? 0.0
                                    : q0.pair ? pair_hop_dE<Real, kPow2, kDim>(S, Rg, p0, q0, dE0, L,
                                                                         log2L, magic, H1)
                                              : hop_dE<Real>(S, p0, dE0);
                            } else {
                                s_cand[warp].dE = a.toy ? 0.0 : hop_dE<Real>(S, p0, dE0);
                            }
                        }
                    } else if (b1) {
                        const int first = __ffs(b1) - 1;
                        off = (unsigned)(kThreads + warp * 32 + first);
                        if (lane == first) {
                            s_cand[warp].i = p1.i;
                            s_cand[warp].j = p1.j;
                            s_cand[warp].dxy = p1.dxy;
                            if (kPair) {
                                s_pcand[warp] = q1;
                                s_cand[warp].dE =
                                    a.toy ? 0.0
                                    : q1.pair ? pair_hop_dE<Real, kPow2, kDim>(S, Rg, p1, q1, dE1, L,
                                                                         log2L, magic, H1)
                                              : hop_dE<Real>(S, p1, dE1);
                            } else {
                                s_cand[warp].dE = a.toy ? 0.0 : hop_dE<Real>(S, p1, dE1);
                            }
                        }
                    }
                    if (lane == 0) s_wlabel[warp] = off;
                    __syncthreads();
                    unsigned wl = (lane < kThreads / 32) ? s_wlabel[lane] : 0xffffffffu;
#pragma unroll
                    for (int o = 16; o; o >>= 1) wl = min(wl, __shfl_xor_sync(0xffffffffu, wl, o));
                    q = kb + wl + 1;                 // 1-based label in the round
                    kb_hit = kb;
                    win = (wl >= (unsigned)kThreads ? wl - (unsigned)kThreads : wl) >> 5;
                    found = true;
                    break;
                }
            }
            }
            if (!found) {
                if (tid == 0) {
                    s_c.attempts += M;
                    s_c.evaluated += M;
                }
                rounds += 1;
                // bounded hop: thread 0 reads its SM's cycle counter (the limit
                // is in cycles at the peak clock), the block-wide OR makes the
                // decision uniform
                const int late = __syncthreads_or(
                    tid == 0 && (unsigned long long)(clock64() - s_c.t0) > a.hop_timeout_cyc);
                if (late) {
                    status = CG_ETIMEOUT;
                    break;
                }
                if (p >= a.max_rounds) {
                    status = CG_ESTUCK;
                    break;
                }
            }
        }
        if (!found) break;

        // ---- commit (step 3a, 3c) ----
        const Cand c = s_cand[win];
        const unsigned ci = c.i, cj = c.j;
        const int cdx = kDim == 3 ? (c.dxy << 22) >> 22 : (int)(short)(c.dxy & 0xffff);
        const int cdy = kDim == 3 ? (c.dxy << 12) >> 22 : c.dxy >> 16;
        // second electron of an executed pair (toy mode has none)
        PairProp cq{};
        if (kPair) cq = s_pcand[win];
        const bool cpair = kPair && !a.toy && cq.pair;
        const int cdx2 = !cpair ? 0 : kDim == 3 ? (cq.dxy2 << 22) >> 22 : (int)(short)(cq.dxy2 & 0xffff);
        const int cdy2 = !cpair ? 0 : kDim == 3 ? (cq.dxy2 << 12) >> 22 : cq.dxy2 >> 16;
        long long t1 = 0;
        if (tid == 0) {
            const unsigned long long m_hop = (p - 1) * (unsigned long long)M + q;
            if (kTime)           // step 3c: Gaussian dt of hop number s_c.hops
                s_c.time = d_add(s_c.time, cg_time_increment(Rg.Gamma, m_hop,
                                                            s_z[s_c.hops - s_zbase]));
            s_c.m_ema = 0.9f * s_c.m_ema + 0.1f * (float)m_hop;
            s_c.attempts += q;
            // the chunks of the hop's round up to the accepting one
            s_c.evaluated += (kb_hit + C < M) ? (kb_hit + C) : M;
            s_c.hops += 1;
            if (!a.toy) {
                s_c.P += cdx + cdx2;
                s_c.energy = d_add(s_c.energy, c.dE);
            }
            if (s_c.tracing)
                trace_hop(Rg, s_c.attempts, s_c.hops, s_c.P, s_c.energy, kTime ? 1 : 0, s_c.time);
            t1 = clock64();
            s_c.cyc_rej += (unsigned long long)(t1 - s_c.t0);
            if (s_c.log) {
                cg_hop e;
                e.i = ci; e.j = cj; e.q = q; e.p = (uint32_t)p; e.round = rounds;
                e.dx = a.toy ? 0 : cdx; e.dy = a.toy ? 0 : cdy;
                e.dE = a.toy ? 0.0 : c.dE;
                e.k = cpair ? cq.k : 0xFFFFFFFFu; e.l = cpair ? cq.l : 0xFFFFFFFFu;
                e.dx2 = cdx2; e.dy2 = cdy2;
                s_c.log[a.log_offset + h] = e;
            }
            if (!a.toy) {
                S.occ[ci >> 5] &= ~(1u << (ci & 31));
                S.occ[cj >> 5] |= (1u << (cj & 31));
                if (cpair) {
                    S.occ[cq.k >> 5] &= ~(1u << (cq.k & 31));
                    S.occ[cq.l >> 5] |= (1u << (cq.l & 31));
                }
            }
        }
        rounds += 1;

        // ---- local-energy update (step 3b) ----
        if (kDim == 3) {
            // thread -> base column bx < L/2 and base (y, z) planes p0, p0 + rpp,
            // ...; each base site (x, y, z) < L/2 serves the eight sites
            // (x + a L/2, y + b L/2, z + c L/2), a, b, c in {0, 1}
            const int Lh = L >> 1;
            const int rpp = kThreads / Lh;
            // an executed pair applies the second electron's update after the
            // first one's (each site rounds twice, in the serial order)
            const int passes3 = (kPair && cpair) ? 2 : 1;
#pragma unroll 1
            for (int pass = 0; pass < passes3; ++pass)
            if (!a.toy && tid < rpp * Lh) {
                const unsigned ui = pass ? cq.k : ci, uj = pass ? cq.l : cj;
                const int bx = tid % Lh, p0 = tid / Lh;
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
                const int fxj = fold_axis(bx - xj, L), fxi = fold_axis(bx - xi, L);
                const Real *cj0 = tinv + fxj, *cj1 = tinv + (Lh - fxj);
                const Real *ci0 = tinv + fxi, *ci1 = tinv + (Lh - fxi);
                const int LL = L * L;
#pragma unroll 2
                for (int pz = p0; pz < Lh * Lh; pz += rpp) {
                    int by, bz, fyj, fyi, fzj, fzi;
                    if (kPow2) {
                        // power-of-two L: shifts, masks and a min for the folds
                        by = pz & (Lh - 1);
                        bz = pz >> (log2L - 1);
                        const int m = L - 1;
                        const int dyj = (by - yj) & m, dyi = (by - yi) & m;
                        const int dzj = (bz - zj) & m, dzi = (bz - zi) & m;
                        fyj = min(dyj, L - dyj); fyi = min(dyi, L - dyi);
                        fzj = min(dzj, L - dzj); fzi = min(dzi, L - dzi);
                    } else {
                        by = pz % Lh;
                        bz = pz / Lh;
                        fyj = fold_axis(by - yj, L); fyi = fold_axis(by - yi, L);
                        fzj = fold_axis(bz - zj, L); fzi = fold_axis(bz - zi, L);
                    }
                    // rows (fz H1 + fy) H1 of the folded table for the four
                    // (z, y) images of the base site, relative to j and to i
                    int oj[2][2], oi[2][2];
#pragma unroll
                    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
                        for (int cy = 0; cy < 2; ++cy) {
                            oj[cz][cy] = ((cz ? Lh - fzj : fzj) * H1 + (cy ? Lh - fyj : fyj)) * H1;
                            oi[cz][cy] = ((cz ? Lh - fzi : fzi) * H1 + (cy ? Lh - fyi : fyi)) * H1;
                        }
                    Real *e = eps + (bz * L + by) * L + bx;
                    // odd base rows take the two x-images in swapped order, so
                    // the half-warps of consecutive rows (L/2 = 16) touch
                    // opposite halves of the banks at each access
                    const int sw = p0 & 1;
#pragma unroll
                    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
                        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
                            for (int c = 0; c < 2; ++c) {
                                const int cx = c ^ sw;
                                const Real ta = (cx ? cj1 : cj0)[oj[cz][cy]];
                                const Real tb = (cx ? ci1 : ci0)[oi[cz][cy]];
                                Real *ep = e + cz * Lh * LL + cy * Lh * L + cx * Lh;
                                *ep = Prec<Real>::add(*ep, Prec<Real>::sub(ta, tb));
                            }
                }
            }
        } else {
            // thread -> base column bx < L/2, base rows by0, by0 + rpp, ...
            const int Lh = L >> 1;
            const int rpp = kThreads / Lh;
            // an executed pair applies the second electron's update after the
            // first one's (each site rounds twice, in the serial order)
            const int passes = (kPair && cpair) ? 2 : 1;
#pragma unroll 1
            for (int pass = 0; pass < passes; ++pass) {
            const unsigned ui = pass ? cq.k : ci, uj = pass ? cq.l : cj;
            if (!a.toy && tid < rpp * Lh) {
                const int bx = tid % Lh, by0 = tid / Lh;
                const int yi = kPow2 ? (int)(ui >> log2L) : (int)__umulhi(ui, magic);
                const int yj = kPow2 ? (int)(uj >> log2L) : (int)__umulhi(uj, magic);
                const int xi = (int)ui - yi * L, xj = (int)uj - yj * L;
                const int fxj = fold_axis(bx - xj, L), fxi = fold_axis(bx - xi, L);
                // columns of (x, .) and (x + L/2, .) relative to j and to i
                const Real *cj0 = tinv + fxj, *cj1 = tinv + (Lh - fxj);
                const Real *ci0 = tinv + fxi, *ci1 = tinv + (Lh - fxi);
                const int LhH1 = Lh * H1, LhL = Lh * L;
                Real *e = eps + by0 * L + bx;
#pragma unroll 4
                for (int y = by0; y < Lh; y += rpp, e += rpp * L) {
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
                    e[LhL] = Prec<Real>::add(e[LhL], Prec<Real>::sub(a01, b01));
                    e[LhL + Lh] = Prec<Real>::add(e[LhL + Lh], Prec<Real>::sub(a11, b11));
                }
            }
            }
        }
        __syncthreads();
        if (tid == 0) s_c.cyc_upd += (unsigned long long)(clock64() - t1);
    }

    // ---- store the replica back ----
    {
        Real *eps_g = reinterpret_cast<Real *>(Rg.eps);
        for (int l = tid; l < N; l += kThreads) eps_g[l] = eps[l];
        for (int l = tid; l < words; l += kThreads) Rg.occ[l] = S.occ[l];
    }
    if (tid == 0) {
        DevCounters *cnt = Rg.ctr;
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
}

}  // namespace cg
