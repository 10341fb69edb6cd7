// cg_pr_random_cluster.cu -- the random-site chain over a thread-block
// cluster of C CTAs per replica, for boxes whose eps (8 N bytes) outgrows one
// CTA's shared memory, or to spread one replica's work over C SMs.
//
// Same chain as pr_random (mixed PR algorithm, steps 1-3), so the same
// trajectory bit for bit:
//   * CTA `rank` owns the eps of sites [rank Nc, min(N, (rank+1) Nc)),
//     Nc = random_cluster_sites(N, C) (a multiple of 32); the occupation
//     bitmask is replicated, and every CTA applies each executed hop to its
//     copy;
//   * a chunk of labels is C kThreads labels, CTA rank evaluating the
//     contiguous sub-range rank, one label per thread; eps_i and eps_j of a
//     proposal come from the owning CTA through distributed shared memory;
//   * each CTA finds its lowest accepting label (OR barrier, ballot, warp
//     minimum) and thread 0 writes it with its payload into every CTA's
//     exchange slot (double-buffered by chunk parity); after one cluster
//     barrier every CTA takes the minimum of the C candidates, the lowest
//     accepting label of the whole chunk;
//   * each CTA updates its own sites from rows j and i of G (step 3b), so a
//     hop reads 16 N bytes of G spread over C SMs; a cluster barrier ends the
//     hop so that the next hop's remote reads see the updated energies.
// The wall-clock limit of a hop is decided by rank 0 and published in its
// exchange slot, so every exit decision is uniform over the cluster.
#include <cooperative_groups.h>

#include "cg_pr_random.cuh"

namespace coop = cooperative_groups;

namespace cg {

namespace {

struct RSlot {
    unsigned int label;      // lowest accepting label of the sending CTA, or ~0
    unsigned int late;       // rank 0 only: the hop ran past its time limit
    RCand cand;
};

// eps of site s from the CTA that owns it: owner = s / Nc, computed on the
// 32-site blocks (s >> 5) / (Nc >> 5): with magicW = floor(2^32 / (Nc >> 5)) + 1
// (exact while (s >> 5) (Nc >> 5) < 2^32) when Nc >> 5 >= 2, else (one
// block per CTA, where that multiplier would need 33 bits) magicW = 0 and
// owner = s >> 5.
__device__ __forceinline__ double cluster_eps_random(coop::cluster_group &cl, double *local,
                                                     unsigned s, unsigned Nc, unsigned magicW,
                                                     unsigned rank)
{
    const unsigned owner = magicW ? __umulhi(s >> 5, magicW) : (s >> 5);
    const unsigned off = s - owner * Nc;
    if (owner == rank) return local[off];
    const double *peer = cl.map_shared_rank(local, owner);
    return peer[off];
}

template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1)
pr_random_cluster(const DevReplica *__restrict__ reps, const int *__restrict__ index, RunArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int s_wlabel[32];
    __shared__ RCand s_cand[32];
    __shared__ RSlot s_slot[2][8];
    __shared__ struct {
        unsigned long long hops, attempts, evaluated, cyc_rej, cyc_upd, wall0;
        long long t0;
        double energy;
        float m_ema;
    } s_c;

    coop::cluster_group cl = coop::this_cluster();
    const unsigned rank = cl.block_rank(), C = cl.num_blocks();
    const DevReplica &Rg = reps[index[blockIdx.x / C]];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = Rg.N, words = (N + 31) / 32;
    const uint32_t key0 = Rg.key0, key1 = Rg.key1, rep = Rg.replica;
    const double T = Rg.T;
    const float invTf = (float)(1.0 / T);
    const unsigned Nc = (unsigned)random_cluster_sites(N, (int)C);
    const unsigned magicW = (Nc >> 5) > 1 ? (unsigned)(4294967296ull / (Nc >> 5) + 1ull) : 0u;
    const int s0 = (int)(rank * Nc);
    const int n_own = max(0, min(N - s0, (int)Nc));
    double *eps = reinterpret_cast<double *>(smem);
    unsigned *occ = reinterpret_cast<unsigned *>(smem + cg_align16((int)Nc * 8));

    // ---- stage: own eps, the whole bitmask ----
    {
        const double *eps_g = reinterpret_cast<const double *>(Rg.eps) + s0;
        for (int l = tid; l < n_own; l += kThreads) eps[l] = eps_g[l];
        for (int l = tid; l < words; l += kThreads) occ[l] = Rg.occ[l];
    }
    DevCounters *cnt = Rg.ctr;
    unsigned long long rounds = cnt->rounds;
    if (tid == 0) {
        s_c.hops = cnt->hops;
        s_c.attempts = cnt->attempts;
        s_c.evaluated = cnt->evaluated;
        s_c.energy = cnt->energy;
        s_c.m_ema = cnt->m_ema > 0.f ? cnt->m_ema : 64.0f;
        s_c.cyc_rej = 0;
        s_c.cyc_upd = 0;
    }
    int status = CG_OK;
    unsigned parity = 0;
    cl.sync();   // every CTA staged before any remote read

    const unsigned M = a.M;
    // one label per thread per chunk, as in pr_random: a chunk costs one
    // chain of dependent global loads however many labels it holds
    const unsigned chunk = (unsigned)kThreads * C;
    for (unsigned long long h = 0; h < a.n_hops; ++h) {
        if (tid == 0) {
            s_c.t0 = clock64();
            s_c.wall0 = globaltimer_ns();
        }
        unsigned long long p = 0;
        unsigned q = 0;
        RCand win{};
        bool found = false;
        while (!found) {
            ++p;
            const PhiloxPrefix PP =
                philox_prefix((uint32_t)rounds, (uint32_t)(rounds >> 32), rep, key0, key1);
            for (unsigned kb = 0; kb < M; kb += chunk) {
                const unsigned base = kb + rank * (unsigned)kThreads;
                const unsigned k0 = base + (unsigned)tid;
                const RLabel p0 = propose_random(Rg, occ, k0, PP, key0, key1, (unsigned)N, k0 < M);
                double dE0 = 0.0;
                bool acc0 = false;
                if (p0.theta) {
                    const double ei = cluster_eps_random(cl, eps, p0.i, Nc, magicW, rank);
                    const double ej = cluster_eps_random(cl, eps, p0.j, Nc, magicW, rank);
                    dE0 = dE_random_vals(ei, ej, p0);
                    acc0 = metropolis64(dE0, p0.x2, T, invTf);
                }
                const int any = __syncthreads_or(acc0);
                unsigned best = 0xffffffffu;
                if (any) {
                    const unsigned b0 = __ballot_sync(0xffffffffu, acc0);
                    unsigned off = 0xffffffffu;
                    if (b0) {
                        const int first = __ffs(b0) - 1;
                        off = (unsigned)(warp * 32 + first);
                        if (lane == first) s_cand[warp] = RCand{p0.i, p0.j, dE0};
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
                    RSlot sl;
                    sl.label = (best == 0xffffffffu) ? 0xffffffffu : base + best;
                    sl.late = (rank == 0) && (globaltimer_ns() - s_c.wall0) > a.hop_timeout_ns;
                    sl.cand = RCand{0u, 0u, 0.0};
                    if (best != 0xffffffffu) sl.cand = s_cand[best >> 5];
                    for (unsigned r = 0; r < C; ++r) *cl.map_shared_rank(&s_slot[parity][rank], r) = sl;
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
                    q = gbest + 1;                  // 1-based label in the round
                    win = s_slot[parity][gwin].cand;
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

        // ---- commit (step 3a, 3c): every CTA flips its bitmask copy; no
        // dipole is kept on random sites ----
        long long t1 = 0;
        if (tid == 0) {
            const unsigned long long m_hop = (p - 1) * (unsigned long long)M + q;
            s_c.m_ema = 0.9f * s_c.m_ema + 0.1f * (float)m_hop;
            s_c.attempts += q;
            s_c.hops += 1;
            s_c.energy = d_add(s_c.energy, win.dE);
            if (rank == 0) trace_hop(Rg, s_c.attempts, s_c.hops, 0, s_c.energy, 0, 0.0);
            t1 = clock64();
            s_c.cyc_rej += (unsigned long long)(t1 - s_c.t0);
            if (rank == 0 && Rg.log) {
                cg_hop e;
                e.i = win.i; e.j = win.j; e.q = q; e.p = (uint32_t)p; e.round = rounds;
                e.dx = 0; e.dy = 0; e.dE = win.dE;
                e.k = 0xFFFFFFFFu; e.l = 0xFFFFFFFFu;
                e.dx2 = 0; e.dy2 = 0;
                Rg.log[a.log_offset + h] = e;
            }
            occ[win.i >> 5] &= ~(1u << (win.i & 31));
            occ[win.j >> 5] |= (1u << (win.j & 31));
        }
        rounds += 1;

        // ---- local-energy update of this CTA's sites (step 3b) ----
        {
            const double *gj = Rg.G + (size_t)win.j * N + s0, *gi = Rg.G + (size_t)win.i * N + s0;
#pragma unroll 4
            for (int l = tid; l < n_own; l += kThreads)
                eps[l] = d_add(eps[l], d_sub(__ldg(gj + l), __ldg(gi + l)));
        }
        cl.sync();   // updated energies visible to every peer before the next hop
        if (tid == 0) s_c.cyc_upd += (unsigned long long)(clock64() - t1);
    }

    // ---- store back: own eps; rank 0 the bitmask and counters ----
    {
        double *eps_g = reinterpret_cast<double *>(Rg.eps) + s0;
        for (int l = tid; l < n_own; l += kThreads) eps_g[l] = eps[l];
        if (rank == 0)
            for (int l = tid; l < words; l += kThreads) Rg.occ[l] = occ[l];
    }
    if (tid == 0 && rank == 0) {
        cnt->rounds = rounds;
        cnt->hops = s_c.hops;
        cnt->attempts = s_c.attempts;
        cnt->evaluated = s_c.evaluated;
        cnt->energy = s_c.energy;
        cnt->cycles_reject += s_c.cyc_rej;
        cnt->cycles_update += s_c.cyc_upd;
        cnt->m_ema = s_c.m_ema;
        cnt->status = status;
    }
    cl.sync();   // no CTA leaves while a peer may still read its shared memory
}

template <int kThreads>
cudaError_t launch_rc(const DevReplica *d_reps, const int *d_index, int n_reps, int cluster,
                      int smem_bytes, const RunArgs &args, cudaStream_t st)
{
    auto kern = pr_random_cluster<kThreads>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
    if (e) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_reps * cluster), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, d_reps, d_index, args);
}

}  // namespace

cudaError_t launch_pr_random_cluster(const DevReplica *d_reps, const int *d_index, int n_reps,
                                     int cluster, int threads, int smem_bytes,
                                     const RunArgs &args, cudaStream_t st)
{
    if (cluster != 2 && cluster != 4 && cluster != 8) return cudaErrorInvalidValue;
    switch (threads) {
    case 256: return launch_rc<256>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st);
    case 512: return launch_rc<512>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st);
    case 1024: return launch_rc<1024>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace cg
