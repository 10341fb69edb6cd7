// cg_aux_kernels.cu -- set-up and refresh kernels of libcg.
//
//   eps_init:     eps_s = phi_s + sum_{t != s} (n_t - nu) / r_st, the single-
//                 particle energies defined below Eq. 2, summed over t in
//                 increasing order with each product rounded before the add,
//                 so the result is bit-identical to a serial evaluation of the
//                 same definition.
//   refresh_fp64: the periodic from-scratch rebuild of binary32 eps in
//                 binary64: eps_s = phi_s + sum_{t occupied} 1/r_st
//                 - nu * sum_{t != s} 1/r_st, records max |eps_old - eps_new|.
//   debug_*:      Philox and the acceptance exponential evaluated on the GPU
//                 for tests.
#include "cg_device.cuh"
#include "cg_internal.h"
#include "cg_pr_common.cuh"

namespace cg {

// Site s = (z L + y) L + x of a square (z = 0) or cubic lattice: x, y, z
// from two exact multiply-high divisions by L.
__device__ __forceinline__ void site_xyz(unsigned s, const DevReplica &R, int &x, int &y, int &z)
{
    const unsigned q = __umulhi(s, R.magicL);           // s / L
    x = (int)(s - q * (unsigned)R.L);
    z = (int)__umulhi(q, R.magicL);                     // s / L^2
    y = (int)q - z * R.L;
}

// (L/2+1)^dim entries of the folded 1/r table
__device__ __forceinline__ int tab_entries(const DevReplica &R)
{
    return R.dim == 3 ? R.H1 * R.H1 * R.H1 : R.H1 * R.H1;
}

// kTabGlobal: the binary64 table stays in global memory (read through the
// read-only cache) when it does not fit shared memory beside the bitmask
// (the 64^3 lattice: 288 KB); the sums are the same.
template <bool kTabGlobal>
__global__ void __launch_bounds__(128) eps_init_kernel(const DevReplica *__restrict__ rp,
                                                       int precision)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const DevReplica &R = *rp;
    const int L = R.L, N = R.N, H1 = R.H1, words = R.words, ntab = tab_entries(R);
    const int Lz = R.dim == 3 ? L : 1;
    double *tab_s = reinterpret_cast<double *>(sm);
    unsigned *occ = reinterpret_cast<unsigned *>(sm + (kTabGlobal ? 0 : cg_align16(ntab * 8)));
    const double *tab = kTabGlobal ? R.tinv64 : tab_s;
    if (!kTabGlobal)
        for (int l = threadIdx.x; l < ntab; l += blockDim.x) tab_s[l] = R.tinv64[l];
    for (int l = threadIdx.x; l < words; l += blockDim.x) occ[l] = R.occ[l];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    int xs, ys, zs;
    site_xyz((unsigned)s, R, xs, ys, zs);
    const double c_occ = d_sub(1.0, R.nu), c_emp = d_sub(0.0, R.nu);
    // t = 0 .. N-1 in increasing order, as the serial chain sums
    double acc = 0.0;
    for (int zt = 0; zt < Lz; ++zt) {
        const double *plane = tab + fold_axis(zs - zt, Lz) * H1 * H1;
        for (int yt = 0; yt < L; ++yt) {
            const double *row = plane + fold_axis(ys - yt, L) * H1;
            const int base = (zt * L + yt) * L;
            for (int xt = 0; xt < L; ++xt) {
                const int t = base + xt;
                if (t == s) continue;
                const double c = ((occ[t >> 5] >> (t & 31)) & 1u) ? c_occ : c_emp;
                const double g = kTabGlobal ? __ldg(row + fold_axis(xs - xt, L))
                                            : row[fold_axis(xs - xt, L)];
                acc = d_add(acc, d_mul(c, g));
            }
        }
    }
    const double e = d_add(R.phi[s], acc);
    if (precision == CG_FP64)
        reinterpret_cast<double *>(R.eps)[s] = e;
    else
        reinterpret_cast<float *>(R.eps)[s] = __double2float_rn(e);
}

// Shared memory of the set-up and refresh kernels above which the table is
// read from global memory instead.
constexpr int kAuxSmemLimit = 200 * 1024;

cudaError_t launch_eps_init(const DevReplica *d_rep, int N, int ntab, int words, int precision,
                            cudaStream_t st)
{
    const int smem = cg_align16(ntab * 8) + words * 4;
    cudaError_t e;
    if (smem > kAuxSmemLimit) {
        const int sm2 = words * 4;
        if ((e = cudaFuncSetAttribute(eps_init_kernel<true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm2)))
            return e;
        eps_init_kernel<true><<<(N + 127) / 128, 128, sm2, st>>>(d_rep, precision);
        return cudaGetLastError();
    }
    if ((e = cudaFuncSetAttribute(eps_init_kernel<false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    eps_init_kernel<false><<<(N + 127) / 128, 128, smem, st>>>(d_rep, precision);
    return cudaGetLastError();
}

template <bool kTabGlobal>
__global__ void __launch_bounds__(256) refresh_fp64_kernel(const DevReplica *__restrict__ rp)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ unsigned long long s_max;
    const DevReplica &R = *rp;
    const int L = R.L, N = R.N, H1 = R.H1, words = R.words, ntab = tab_entries(R);
    const int Lz = R.dim == 3 ? L : 1;
    double *tab_s = reinterpret_cast<double *>(sm);
    unsigned *occ = reinterpret_cast<unsigned *>(sm + (kTabGlobal ? 0 : cg_align16(ntab * 8)));
    const double *tab = kTabGlobal ? R.tinv64 : tab_s;
    if (!kTabGlobal)
        for (int l = threadIdx.x; l < ntab; l += blockDim.x) tab_s[l] = R.tinv64[l];
    for (int l = threadIdx.x; l < words; l += blockDim.x) occ[l] = R.occ[l];
    if (threadIdx.x == 0) s_max = 0ull;
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double err = 0.0;
    if (s < N) {
        int xs, ys, zs;
        site_xyz((unsigned)s, R, xs, ys, zs);
        double acc = 0.0;
        for (int w = 0; w < words; ++w) {
            unsigned bits = occ[w];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int t = w * 32 + b;
                int xt, yt, zt;
                site_xyz((unsigned)t, R, xt, yt, zt);
                const int o = (fold_axis(zs - zt, Lz) * H1 + fold_axis(ys - yt, L)) * H1 +
                              fold_axis(xs - xt, L);
                acc += kTabGlobal ? __ldg(tab + o) : tab[o];
            }
        }
        const double e = R.phi[s] + (acc + R.negC0nu);
        float *eps = reinterpret_cast<float *>(R.eps);
        err = fabs((double)eps[s] - e);
        eps[s] = __double2float_rn(e);
    }
    // block max of the non-negative errors through their bit patterns
    unsigned long long bits = (unsigned long long)__double_as_longlong(err);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = bits > other ? bits : other;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, bits);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMax(&R.ctr->max_err_bits, s_max);
        if (blockIdx.x == 0) atomicAdd(&R.ctr->refreshes, 1ull);
    }
}

cudaError_t launch_refresh_fp64(const DevReplica *d_rep, int N, int ntab, int words,
                                cudaStream_t st)
{
    const int smem = cg_align16(ntab * 8) + words * 4;
    cudaError_t e;
    if (smem > kAuxSmemLimit) {
        const int sm2 = words * 4;
        if ((e = cudaFuncSetAttribute(refresh_fp64_kernel<true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm2)))
            return e;
        refresh_fp64_kernel<true><<<(N + 255) / 256, 256, sm2, st>>>(d_rep);
        return cudaGetLastError();
    }
    if ((e = cudaFuncSetAttribute(refresh_fp64_kernel<false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    refresh_fp64_kernel<false><<<(N + 255) / 256, 256, smem, st>>>(d_rep);
    return cudaGetLastError();
}

__global__ void reset_refresh_err_kernel(const DevReplica *__restrict__ reps,
                                         const int *__restrict__ index, int R)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) reps[index[r]].ctr->max_err_bits = 0ull;
}

cudaError_t launch_reset_refresh_err(const DevReplica *d_reps, const int *d_index, int R,
                                     cudaStream_t st)
{
    reset_refresh_err_kernel<<<(R + 127) / 128, 128, 0, st>>>(d_reps, d_index, R);
    return cudaGetLastError();
}

__global__ void debug_philox_kernel(const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                                    int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    // the split form the PR kernels use (prefix shared by counters that differ
    // only in word 0)
    uint32_t x[4];
    const PhiloxPrefix P = philox_prefix(ctr[4 * t + 1], ctr[4 * t + 2], ctr[4 * t + 3],
                                         key[2 * t], key[2 * t + 1]);
    philox_finish(ctr[4 * t], P, key[2 * t], key[2 * t + 1], x);
    for (int w = 0; w < 4; ++w) out[4 * t + w] = x[w];
}

__global__ void debug_exp_kernel(const double *x, double *out, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = cg_exp_accept(x[t]);
}

__global__ void debug_tower_kernel(const unsigned short *guide, const unsigned *thr, int V,
                                   const uint32_t *x1, int *out, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    // the PR kernels' sampler (on the global copies of the tables); -1 marks a
    // null proposal
    out[t] = x1[t] > thr[V - 1] ? -1 : tower_lookup(guide, thr, x1[t]);
}

// g(eps): one CTA per (chunk of sites, replica) builds a shared-memory
// histogram and adds it to the output; bin floor((eps - lo) * scale) in
// binary64, for eps >= lo and (eps - lo) * scale < nbins.
template <typename Real>
__global__ void eps_histogram_kernel(const DevReplica *__restrict__ reps, int nbins, double lo,
                                     double scale, unsigned long long *__restrict__ out)
{
    extern __shared__ unsigned int hist[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    const DevReplica &R = reps[blockIdx.y];
    const Real *eps = reinterpret_cast<const Real *>(R.eps);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < R.N; s += gridDim.x * blockDim.x) {
        const double e = (double)eps[s];
        const double x = d_mul(d_sub(e, lo), scale);
        if (e >= lo && x < (double)nbins) atomicAdd(&hist[(int)floor(x)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (hist[b]) atomicAdd(&out[b], (unsigned long long)hist[b]);
}

cudaError_t launch_eps_histogram(const DevReplica *d_reps, int count, int max_N, int precision,
                                 int nbins, double lo, double scale, unsigned long long *out,
                                 cudaStream_t st)
{
    const int per = (max_N + 255) / 256;
    const dim3 grid((unsigned)(per < 16 ? per : 16), (unsigned)count);
    const size_t smem = sizeof(unsigned int) * (size_t)nbins;
    if (precision == CG_FP64)
        eps_histogram_kernel<double><<<grid, 256, smem, st>>>(d_reps, nbins, lo, scale, out);
    else
        eps_histogram_kernel<float><<<grid, 256, smem, st>>>(d_reps, nbins, lo, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_debug_tower(const unsigned short *guide, const unsigned *thr, int V,
                               const uint32_t *x1, int *out, int n, cudaStream_t st)
{
    debug_tower_kernel<<<(n + 127) / 128, 128, 0, st>>>(guide, thr, V, x1, out, n);
    return cudaGetLastError();
}

__global__ void debug_gauss_kernel(const uint64_t *seed, const uint32_t *rep, const uint64_t *hop,
                                   double *z, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n)
        z[t] = cg_gauss((uint32_t)seed[t], (uint32_t)(seed[t] >> 32), rep[t], hop[t]);
}

cudaError_t launch_debug_gauss(const uint64_t *seed, const uint32_t *rep, const uint64_t *hop,
                               double *z, int n, cudaStream_t st)
{
    debug_gauss_kernel<<<(n + 127) / 128, 128, 0, st>>>(seed, rep, hop, z, n);
    return cudaGetLastError();
}

cudaError_t launch_debug_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n,
                                cudaStream_t st)
{
    debug_philox_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctr, key, out, n);
    return cudaGetLastError();
}

cudaError_t launch_debug_exp(const double *x, double *out, int n, cudaStream_t st)
{
    debug_exp_kernel<<<(n + 127) / 128, 128, 0, st>>>(x, out, n);
    return cudaGetLastError();
}

}  // namespace cg
