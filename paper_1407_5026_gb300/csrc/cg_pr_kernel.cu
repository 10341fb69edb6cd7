// cg_pr_kernel.cu -- the persistent parallel-rejection kernel.
//
// One CTA runs one disorder replica for a whole launch.  Its local energies
// eps (N values), the folded minimum-image 1/r table, the occupation bitmask
// and the tower live in shared memory; global memory is touched only to load
// the state at the start and store it at the end.
//
// Per executed hop (mixed PR algorithm, section "Hopping conduction in the
// Coulomb glass", steps 1-3):
//   rounds r = 0, 1, ...: the M labels of a round are evaluated in chunks of
//   blockDim labels in increasing order, one label per thread.  Label k draws
//   Philox(key = seed, ctr = (k, r lo, r hi, replica)) -> site i from word 0,
//   hop vector from word 1 by tower sampling, acceptance variate from word 2
//   (step 1 and the three random numbers per label of the GPU paragraph);
//   theta = n_i (1 - n_j) and the Metropolis test on
//   dH = eps_j - eps_i - 1/r_ij - E dx (step 2, Eq. 2).  A chunk with no
//   accept costs one block-wide OR barrier; the first chunk with an accept
//   gives the lowest accepting label q by warp ballot + find-first-set and
//   a minimum over the warps.  Labels after q are never looked at, so the
//   result equals the serial rejection chain on the same random numbers.
//   Commit (step 3a/3b/3c): flip n_i, n_j, P += dx, attempts += (p-1)M + q.
//   Update (step 3b): eps_l += 1/r_lj - 1/r_li for every l, with the table
//   holding 0 at the origin so l = i and l = j need no special case.
#include <cstdio>

#include "cg_device.cuh"
#include "cg_internal.h"

namespace cg {

struct Cand {
    unsigned int i, j;
    int dxy;           // packed hop vector
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

// Step 2 for one proposal whose theta holds: returns accept, writes dE.
template <typename Real>
__device__ __forceinline__ bool accept_test(const Real *eps, const double *tinvd, int v,
                                            unsigned i, unsigned j, int dx, uint32_t x2,
                                            double E, double T, float Ef, float invTf,
                                            double &dE_out);

template <>
__device__ __forceinline__ bool accept_test<double>(const double *eps, const double *tinvd,
                                                    int v, unsigned i, unsigned j, int dx,
                                                    uint32_t x2, double E, double T, float,
                                                    float, double &dE_out)
{
    double d = d_sub(eps[j], eps[i]);
    d = d_sub(d, tinvd[v]);
    const double dE = d_sub(d, d_mul(E, (double)dx));
    dE_out = dE;
    if (dE <= 0.0) return true;
    const double u = d_mul(d_add((double)x2, 0.5), 0x1p-32);
    return u < cg_exp_accept(d_div(-dE, T));
}

template <>
__device__ __forceinline__ bool accept_test<float>(const float *eps, const double *tinvd,
                                                   int v, unsigned i, unsigned j, int dx,
                                                   uint32_t x2, double E, double T, float Ef,
                                                   float invTf, double &dE_out)
{
    const float ei = eps[i], ej = eps[j];
    const float dEf = ((ej - ei) - (float)tinvd[v]) - Ef * (float)dx;
    if (fabsf(dEf) < 1e-5f) {
        // near tie: decide in binary64 from the widened energies
        double d = d_sub((double)ej, (double)ei);
        d = d_sub(d, tinvd[v]);
        const double dE = d_sub(d, d_mul(E, (double)dx));
        dE_out = dE;
        if (dE <= 0.0) return true;
        const double u = d_mul(d_add((double)x2, 0.5), 0x1p-32);
        return u < cg_exp_accept(d_div(-dE, T));
    }
    dE_out = (double)dEf;
    if (dEf <= 0.0f) return true;
    const float u = ((float)(x2 >> 9) + 0.5f) * 0x1p-23f;
    return u < expf(-dEf * invTf);
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename Real, int kThreads>
__global__ void __launch_bounds__(kThreads, (kThreads >= 1024 ? 1 : 2048 / kThreads / 2))
pr_persistent(const DevReplica *__restrict__ reps, const int *__restrict__ index, RunArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int s_wlabel[32];
    __shared__ Cand s_cand[32];

    const DevReplica &Rg = reps[index[blockIdx.x]];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = Rg.L, N = Rg.N, H1 = Rg.H1, V = Rg.V, words = Rg.words;
    const unsigned magic = Rg.magicL;
    const uint32_t key0 = Rg.key0, key1 = Rg.key1, rep = Rg.replica;
    const double T = Rg.T, E = Rg.E;
    const float Ef = (float)E, invTf = (float)(1.0 / T);

    const SmemLayout lay = smem_layout(N, H1, V, words, (int)sizeof(Real));
    Real *eps = reinterpret_cast<Real *>(smem + lay.off_eps);
    Real *tinv = reinterpret_cast<Real *>(smem + lay.off_tinv);
    unsigned *occ = reinterpret_cast<unsigned *>(smem + lay.off_occ);
    unsigned *thr = reinterpret_cast<unsigned *>(smem + lay.off_thr);
    int *disp = reinterpret_cast<int *>(smem + lay.off_disp);
    double *tinvd = reinterpret_cast<double *>(smem + lay.off_tinvd);

    // ---- stage the replica into shared memory ----
    {
        const Real *eps_g = reinterpret_cast<const Real *>(Rg.eps);
        for (int l = tid; l < N; l += kThreads) eps[l] = eps_g[l];
        const Real *tab_g = (sizeof(Real) == 8)
                                ? reinterpret_cast<const Real *>(Rg.tinv64)
                                : reinterpret_cast<const Real *>(Rg.tinv32);
        for (int l = tid; l < H1 * H1; l += kThreads) tinv[l] = tab_g[l];
        for (int l = tid; l < words; l += kThreads) occ[l] = Rg.occ[l];
        for (int l = tid; l < V; l += kThreads) {
            thr[l] = Rg.thr[l];
            disp[l] = Rg.disp[l];
            tinvd[l] = Rg.tinvd[l];
        }
    }
    DevCounters *cnt = Rg.ctr;
    unsigned long long rounds = cnt->rounds, hops = cnt->hops;
    unsigned long long attempts = cnt->attempts, evaluated = cnt->evaluated;
    long long P = cnt->P;
    double energy = cnt->energy;
    unsigned long long cyc_rej = 0, cyc_upd = 0;
    int status = CG_OK;
    __syncthreads();

    const unsigned M = a.M;
    const unsigned thr_last = thr[V - 1];
    // update mapping: thread -> fixed column ux, rows uy0, uy0 + rows_per_pass, ...
    const int rows_per_pass = kThreads / L;
    const int active = rows_per_pass * L;
    const int ux = tid % L, uy0 = tid / L;

    for (unsigned long long h = 0; h < a.n_hops; ++h) {
        long long t0 = 0;
        unsigned long long wall0 = 0;
        if (tid == 0) {
            t0 = clock64();
            wall0 = globaltimer_ns();
        }
        unsigned long long p = 0;
        unsigned q = 0, win = 0;
        bool found = false;
        while (!found) {
            ++p;
            for (unsigned kb = 0; kb < M; kb += kThreads) {
                const unsigned k = kb + (unsigned)tid;
                bool acc = false;
                unsigned i = 0, j = 0;
                int dxy = 0;
                double dE = 0.0;
                if (k < M) {
                    uint32_t x[4];
                    philox4x32_10(k, (uint32_t)rounds, (uint32_t)(rounds >> 32), rep,
                                  key0, key1, x);
                    i = __umulhi(x[0], (unsigned)N);
                    if (a.toy) {
                        const double u = d_mul(d_add((double)x[2], 0.5), 0x1p-32);
                        acc = u < a.toy_A0;
                    } else if (x[1] <= thr_last) {
                        // tower: smallest v with x1 <= C_v - 1
                        int lo = 0, hi = V - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (x[1] <= thr[mid]) hi = mid; else lo = mid + 1;
                        }
                        dxy = disp[lo];
                        const int dx = (int)(short)(dxy & 0xffff), dy = dxy >> 16;
                        const int yi = (int)__umulhi(i, magic), xi = (int)i - yi * L;
                        int xj = xi + dx, yj = yi + dy;
                        xj += (xj < 0) ? L : 0; xj -= (xj >= L) ? L : 0;
                        yj += (yj < 0) ? L : 0; yj -= (yj >= L) ? L : 0;
                        j = (unsigned)(yj * L + xj);
                        const bool ni = (occ[i >> 5] >> (i & 31)) & 1u;
                        if (ni) {
                            const bool nj = (occ[j >> 5] >> (j & 31)) & 1u;
                            if (!nj)
                                acc = accept_test<Real>(eps, tinvd, lo, i, j, dx, x[2], E, T,
                                                        Ef, invTf, dE);
                        }
                    }
                }
                const int any = __syncthreads_or(acc);
                const unsigned span = (M - kb < (unsigned)kThreads) ? (M - kb) : (unsigned)kThreads;
                evaluated += span;
                if (any) {
                    const unsigned b = __ballot_sync(0xffffffffu, acc);
                    if (b) {
                        const int first = __ffs(b) - 1;
                        if (lane == first) {
                            s_cand[warp].i = i;
                            s_cand[warp].j = j;
                            s_cand[warp].dxy = dxy;
                            s_cand[warp].dE = dE;
                        }
                        if (lane == 0) s_wlabel[warp] = (unsigned)(warp * 32 + first);
                    } else if (lane == 0) {
                        s_wlabel[warp] = 0xffffffffu;
                    }
                    __syncthreads();
                    unsigned wl = (lane < kThreads / 32) ? s_wlabel[lane] : 0xffffffffu;
#pragma unroll
                    for (int o = 16; o; o >>= 1) wl = min(wl, __shfl_xor_sync(0xffffffffu, wl, o));
                    q = kb + wl + 1;               // 1-based label in the round
                    win = wl;
                    found = true;
                    break;
                }
            }
            if (!found) {
                attempts += M;
                rounds += 1;
                // bounded hop: thread 0 reads the wall clock, the block-wide OR
                // makes the decision uniform
                const int late = __syncthreads_or(
                    tid == 0 && (globaltimer_ns() - wall0) > a.hop_timeout_ns);
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
        const Cand c = s_cand[win >> 5];
        const unsigned ci = c.i, cj = c.j;
        const int cdx = (int)(short)(c.dxy & 0xffff), cdy = c.dxy >> 16;
        attempts += q;
        if (!a.toy) {
            P += cdx;
            energy = d_add(energy, c.dE);
        }
        long long t1 = 0;
        if (tid == 0) {
            t1 = clock64();
            cyc_rej += (unsigned long long)(t1 - t0);
            if (Rg.log) {
                cg_hop e;
                e.i = ci; e.j = cj; e.q = q; e.p = (uint32_t)p; e.round = rounds;
                e.dx = a.toy ? 0 : cdx; e.dy = a.toy ? 0 : cdy;
                e.dE = a.toy ? 0.0 : c.dE;
                Rg.log[a.log_offset + h] = e;
            }
            if (!a.toy) {
                occ[ci >> 5] &= ~(1u << (ci & 31));
                occ[cj >> 5] |= (1u << (cj & 31));
            }
        }
        rounds += 1;
        hops += 1;

        // ---- local-energy update (step 3b) ----
        if (!a.toy && tid < active) {
            const int yi = (int)__umulhi(ci, magic), xi = (int)ci - yi * L;
            const int yj = (int)__umulhi(cj, magic), xj = (int)cj - yj * L;
            const int fxj = fold_axis(ux - xj, L), fxi = fold_axis(ux - xi, L);
            for (int y = uy0; y < L; y += rows_per_pass) {
                const int fyj = fold_axis(y - yj, L), fyi = fold_axis(y - yi, L);
                const Real ta = tinv[fyj * H1 + fxj], tb = tinv[fyi * H1 + fxi];
                const int l = y * L + ux;
                eps[l] = Prec<Real>::add(eps[l], Prec<Real>::sub(ta, tb));
            }
        }
        __syncthreads();
        if (tid == 0) cyc_upd += (unsigned long long)(clock64() - t1);
    }

    // ---- store the replica back ----
    {
        Real *eps_g = reinterpret_cast<Real *>(Rg.eps);
        for (int l = tid; l < N; l += kThreads) eps_g[l] = eps[l];
        for (int l = tid; l < words; l += kThreads) Rg.occ[l] = occ[l];
    }
    if (tid == 0) {
        cnt->rounds = rounds;
        cnt->hops = hops;
        cnt->attempts = attempts;
        cnt->evaluated = evaluated;
        cnt->P = P;
        cnt->energy = energy;
        cnt->cycles_reject += cyc_rej;
        cnt->cycles_update += cyc_upd;
        cnt->status = status;
    }
}

template <typename Real, int kThreads>
static cudaError_t launch_t(const DevReplica *d_reps, const int *d_index, int n_ctas,
                            int smem_bytes, const RunArgs &args, cudaStream_t st)
{
    pr_persistent<Real, kThreads><<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
    return cudaGetLastError();
}

template <typename Real>
static cudaError_t set_smem_t(int bytes)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(pr_persistent<Real, 1024>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    if ((e = cudaFuncSetAttribute(pr_persistent<Real, 512>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    return cudaFuncSetAttribute(pr_persistent<Real, 256>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t set_pr_smem_limit(int precision, int bytes)
{
    return precision == CG_FP64 ? set_smem_t<double>(bytes) : set_smem_t<float>(bytes);
}

cudaError_t launch_pr_persistent(int precision, const DevReplica *d_reps, const int *d_index,
                                 int n_ctas, int threads, int smem_bytes, const RunArgs &args,
                                 cudaStream_t st)
{
    if (precision == CG_FP64) {
        switch (threads) {
        case 1024: return launch_t<double, 1024>(d_reps, d_index, n_ctas, smem_bytes, args, st);
        case 512: return launch_t<double, 512>(d_reps, d_index, n_ctas, smem_bytes, args, st);
        case 256: return launch_t<double, 256>(d_reps, d_index, n_ctas, smem_bytes, args, st);
        }
    } else {
        switch (threads) {
        case 1024: return launch_t<float, 1024>(d_reps, d_index, n_ctas, smem_bytes, args, st);
        case 512: return launch_t<float, 512>(d_reps, d_index, n_ctas, smem_bytes, args, st);
        case 256: return launch_t<float, 256>(d_reps, d_index, n_ctas, smem_bytes, args, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace cg
