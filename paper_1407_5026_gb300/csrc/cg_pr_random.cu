// cg_pr_random.cu -- the random-site Coulomb glass: N = L^2 sites at random
// positions in the L x L periodic box (the model of the paper's introduction
// and of its closing remarks on off-lattice systems).  Hops go from a site to
// one of its partners within r_max, chosen with probability proportional to
// exp(-2 r_ij / xi) by an integer tower over the site's partner list.
//
// The geometry replaces the lattice's folded table by the N x N matrix
// G_st = 1 / |x_t - x_s| (minimum image, G_ss = 0), built on the device with
// correctly rounded binary64 operations in the serial chain's order, so it
// is bit-identical to the host's.  It is symmetric bit for bit: the rounded
// difference of two positions changes sign exactly with its operands, and
// the minimum-image fold maps d to -d exactly.
//
// pr_random: one CTA per replica, binary64; eps and the occupation bitmask in
// shared memory, the partner lists (a 64-byte guide record per site, 8-byte
// pair records) and G in global memory (read-only path).  The round and
// lowest-accepting-label structure is that of the lattice's persistent
// kernel (mixed PR algorithm, steps 1-3), with one label per thread in every
// chunk, so the trajectory equals the serial chain's on the same random
// numbers:
//   label k of round r: Philox(ctr = (k, r lo, r hi, replica)) -> site
//   i = floor(x0 N 2^-32), partner m = smallest in i's list with
//   x1 < C_m (C the running integer weights; none: a null proposal),
//   u from x2; theta = n_i (1 - n_j); dH = ((eps_j - eps_i) - 1/r_ij) - E dx_ij.
//   Update (step 3b): eps_l += G_jl - G_il for every l, two coalesced rows.
#include "cg_pr_random.cuh"

namespace cg {

namespace {

__device__ __forceinline__ double min_image_d(double d, double L, double halfL)
{
    if (d > halfL) return d_sub(d, L);
    if (d < -halfL) return d_add(d, L);
    return d;
}

// G_st = 1 / sqrt(dx^2 + dy^2) with (dx, dy) the minimum image of x_t - x_s;
// one thread per entry, rows s from blockIdx.y in steps of gridDim.y.
__global__ void g_build_kernel(const double *__restrict__ px, const double *__restrict__ py,
                               double Ld, int N, double *__restrict__ G)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const double halfL = 0.5 * Ld;
    for (int s = blockIdx.y; s < N; s += gridDim.y) {
        double g = 0.0;
        if (t != s) {
            const double dx = min_image_d(d_sub(px[t], px[s]), Ld, halfL);
            const double dy = min_image_d(d_sub(py[t], py[s]), Ld, halfL);
            g = __ddiv_rn(1.0, __dsqrt_rn(d_add(d_mul(dx, dx), d_mul(dy, dy))));
        }
        G[(size_t)s * N + t] = g;
    }
}

// eps_s = phi_s + sum_{t != s} (n_t - nu) G_st, t ascending, each product
// rounded before the sum; thread s reads column s of the symmetric G (rows t
// are contiguous across the warp).
__global__ void eps_init_random_kernel(const DevReplica *__restrict__ rep)
{
    const DevReplica &Rg = *rep;
    const int N = Rg.N;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const double nu = Rg.nu;
    const double om = 1.0 - nu, mn = 0.0 - nu;     // (n_t - nu) for n_t = 1, 0
    double acc = 0.0;
    for (int t = 0; t < N; ++t) {
        if (t == s) continue;
        const double nt = ((Rg.occ[t >> 5] >> (t & 31)) & 1u) ? om : mn;
        acc = d_add(acc, d_mul(nt, __ldg(Rg.G + (size_t)t * N + s)));
    }
    reinterpret_cast<double *>(Rg.eps)[s] = d_add(Rg.phi[s], acc);
}

template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1)
pr_random(const DevReplica *__restrict__ reps, const int *__restrict__ index, RunArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int s_wlabel[32];
    __shared__ RCand s_cand[32];
    __shared__ struct {
        unsigned long long hops, attempts, evaluated, cyc_rej, cyc_upd;
        long long t0;
        double energy;
        cg_hop *log;
        int tracing;
        float m_ema;
    } s_c;

    const DevReplica &Rg = reps[index[blockIdx.x]];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = Rg.N, words = (N + 31) / 32;
    const uint32_t key0 = Rg.key0, key1 = Rg.key1, rep = Rg.replica;
    const double T = Rg.T;
    const float invTf = (float)(1.0 / T);
    double *eps = reinterpret_cast<double *>(smem);
    unsigned *occ = reinterpret_cast<unsigned *>(smem + cg_align16(N * 8));
    // the compacted guide records after eps and the bitmask (every list of
    // the group below 256 pairs and room for them), else the global records
    uint4 *gsm = a.smem_guide
                     ? reinterpret_cast<uint4 *>(smem + cg_align16(N * 8) + cg_align16(words * 4))
                     : nullptr;

    {
        const double *eps_g = reinterpret_cast<const double *>(Rg.eps);
        for (int l = tid; l < N; l += kThreads) eps[l] = eps_g[l];
        for (int l = tid; l < words; l += kThreads) occ[l] = Rg.occ[l];
        if (gsm) stage_guide<kThreads>(gsm, Rg, N, tid);
    }
    unsigned long long rounds = Rg.ctr->rounds;
    if (tid == 0) {
        const DevCounters *cnt = Rg.ctr;
        s_c.log = Rg.log;
        s_c.tracing = Rg.trace != nullptr;
        s_c.hops = cnt->hops;
        s_c.attempts = cnt->attempts;
        s_c.evaluated = cnt->evaluated;
        s_c.energy = cnt->energy;
        s_c.m_ema = cnt->m_ema > 0.f ? cnt->m_ema : 64.0f;
        s_c.cyc_rej = 0;
        s_c.cyc_upd = 0;
    }
    int status = CG_OK;
    __syncthreads();

    const unsigned M = a.M;
    // one label per thread in every chunk: a chunk costs the latency of one
    // chain of dependent global loads (list offsets, search probes, partner,
    // 1/r) however many labels it holds, so the widest chunk settles a hop in
    // the fewest chunks; a second label per thread would run a second chain
    // after the first.  C changes which labels are evaluated, never the hop.
    const unsigned C = kThreads;
    for (unsigned long long h = 0; h < a.n_hops; ++h) {
        if (tid == 0) s_c.t0 = clock64();
        unsigned long long p = 0;
        unsigned q = 0, win = 0, kb_hit = 0;
        bool found = false;
        while (!found) {
            ++p;
            const PhiloxPrefix PP =
                philox_prefix((uint32_t)rounds, (uint32_t)(rounds >> 32), rep, key0, key1);
            for (unsigned kb = 0; kb < M; kb += C) {
                const unsigned k0 = kb + (unsigned)tid;
                const RLabel p0 = propose_random(Rg, occ, k0, PP, key0, key1, (unsigned)N, k0 < M,
                                                 gsm);
                double dE0 = 0.0;
                bool acc0 = false;
                if (p0.theta) {
                    dE0 = dE_random(Rg, eps, p0);
                    acc0 = metropolis64(dE0, p0.x2, T, invTf);
                }
                const int any = __syncthreads_or(acc0);
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
                    q = kb + wl + 1;                 // 1-based label in the round
                    kb_hit = kb;
                    win = wl >> 5;
                    found = true;
                    break;
                }
            }
            if (!found) {
                if (tid == 0) {
                    s_c.attempts += M;
                    s_c.evaluated += M;
                }
                rounds += 1;
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

        // ---- commit (step 3a, 3c); no dipole is kept on random sites ----
        const RCand c = s_cand[win];
        long long t1 = 0;
        if (tid == 0) {
            const unsigned long long m_hop = (p - 1) * (unsigned long long)M + q;
            s_c.m_ema = 0.9f * s_c.m_ema + 0.1f * (float)m_hop;
            s_c.attempts += q;
            s_c.evaluated += (kb_hit + C < M) ? (kb_hit + C) : M;
            s_c.hops += 1;
            s_c.energy = d_add(s_c.energy, c.dE);
            if (s_c.tracing) trace_hop(Rg, s_c.attempts, s_c.hops, 0, s_c.energy, 0, 0.0);
            t1 = clock64();
            s_c.cyc_rej += (unsigned long long)(t1 - s_c.t0);
            if (s_c.log) {
                cg_hop e;
                e.i = c.i; e.j = c.j; e.q = q; e.p = (uint32_t)p; e.round = rounds;
                e.dx = 0; e.dy = 0; e.dE = c.dE;
                e.k = 0xFFFFFFFFu; e.l = 0xFFFFFFFFu;
                e.dx2 = 0; e.dy2 = 0;
                s_c.log[a.log_offset + h] = e;
            }
            occ[c.i >> 5] &= ~(1u << (c.i & 31));
            occ[c.j >> 5] |= (1u << (c.j & 31));
        }
        rounds += 1;

        // ---- local-energy update (step 3b): rows j and i of G ----
        {
            const double *gj = Rg.G + (size_t)c.j * N, *gi = Rg.G + (size_t)c.i * N;
#pragma unroll 4
            for (int l = tid; l < N; l += kThreads)
                eps[l] = d_add(eps[l], d_sub(__ldg(gj + l), __ldg(gi + l)));
        }
        __syncthreads();
        if (tid == 0) s_c.cyc_upd += (unsigned long long)(clock64() - t1);
    }

    {
        double *eps_g = reinterpret_cast<double *>(Rg.eps);
        for (int l = tid; l < N; l += kThreads) eps_g[l] = eps[l];
        for (int l = tid; l < words; l += kThreads) Rg.occ[l] = occ[l];
    }
    if (tid == 0) {
        DevCounters *cnt = Rg.ctr;
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
}

}  // namespace

cudaError_t launch_g_build(const double *px, const double *py, int L, int N, double *G,
                           cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((N + 255) / 256), (unsigned)(N < 65535 ? N : 65535));
    g_build_kernel<<<grid, 256, 0, st>>>(px, py, (double)L, N, G);
    return cudaGetLastError();
}

cudaError_t launch_eps_init_random(const DevReplica *d_rep, int N, cudaStream_t st)
{
    eps_init_random_kernel<<<(N + 127) / 128, 128, 0, st>>>(d_rep);
    return cudaGetLastError();
}

cudaError_t set_pr_random_smem_limit(int bytes)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(pr_random<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  bytes)))
        return e;
    if ((e = cudaFuncSetAttribute(pr_random<384>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  bytes)))
        return e;
    if ((e = cudaFuncSetAttribute(pr_random<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  bytes)))
        return e;
    return cudaFuncSetAttribute(pr_random<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes);
}

cudaError_t launch_pr_random(const DevReplica *d_reps, const int *d_index, int n_ctas,
                             int threads, int smem_bytes, const RunArgs &args, cudaStream_t st)
{
    switch (threads) {
    case 256: pr_random<256><<<n_ctas, 256, smem_bytes, st>>>(d_reps, d_index, args); break;
    case 384: pr_random<384><<<n_ctas, 384, smem_bytes, st>>>(d_reps, d_index, args); break;
    case 512: pr_random<512><<<n_ctas, 512, smem_bytes, st>>>(d_reps, d_index, args); break;
    case 1024: pr_random<1024><<<n_ctas, 1024, smem_bytes, st>>>(d_reps, d_index, args); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cg
