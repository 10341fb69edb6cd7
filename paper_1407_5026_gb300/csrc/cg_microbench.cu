// cg_microbench.cu -- peak rates that bound the eps update, measured on the
// GPU the library runs on (no vendor figure is assumed):
//   kind 0  aggregate shared-memory bandwidth (bytes/s) of a read-modify-write
//           stream of 32-bit words, the access pattern of the binary32 eps
//           update (each warp touches 32 consecutive words per instruction);
//   kind 1  aggregate binary64 add rate (adds/s), which bounds the binary64
//           eps update (two adds per site and hop);
//   kind 2  aggregate shared-memory bandwidth (bytes/s) of the same stream with
//           64-bit words (the binary64 eps update's pattern);
//   kind 3  aggregate Philox-4x32-10 rate (blocks/s) of the PR kernels' own
//           label generator (per-round prefix + per-label finish, two labels
//           per thread, 2 x 512 threads per SM), the ceiling of the rejection
//           phase: every evaluated label costs one block;
//   kind 4, 5, 6  seconds per cluster barrier (cluster.sync) of 2, 4 or 8
//           CTAs of 1024 threads, one CTA per SM, every SM's clusters busy:
//           the fixed cost the cluster kernels pay per chunk and per hop;
//   kind 7  seconds per CTA barrier (__syncthreads) of 1024 threads, one CTA
//           per SM: the single-CTA kernels' per-chunk cost.
// Barrier times are the difference of two launch lengths (4096 and 1024
// barriers) over 3072 barriers, so the launch overhead cancels.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "cg_device.cuh"
#include "cg_internal.h"

namespace cg {

template <typename T>
__global__ void __launch_bounds__(1024) smem_rmw_kernel(int iters, T *sink)
{
    extern __shared__ __align__(16) unsigned char sm[];
    // volatile: every load and store is issued (no promotion to registers)
    volatile T *buf = reinterpret_cast<volatile T *>(sm);
    const int n = 16384;   // words per CTA buffer
    for (int k = threadIdx.x; k < n; k += blockDim.x) buf[k] = (T)k;
    __syncthreads();
    T acc = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll 4
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const T v = buf[k];
            buf[k] = v + (T)1;
            acc += v;
        }
    }
    if (acc == (T)12345) sink[0] = acc;   // practically never true; keeps the loop alive
}

__global__ void __launch_bounds__(256) dadd_kernel(int iters, double seed, double *sink)
{
    double a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    double a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    const double b = 1e-300;
    for (int it = 0; it < iters; ++it) {
        a0 = __dadd_rn(a0, b); a1 = __dadd_rn(a1, b); a2 = __dadd_rn(a2, b); a3 = __dadd_rn(a3, b);
        a4 = __dadd_rn(a4, b); a5 = __dadd_rn(a5, b); a6 = __dadd_rn(a6, b); a7 = __dadd_rn(a7, b);
    }
    const double s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == -1.0) sink[0] = s;
}

// Labels k of rounds r = it / 4 under the CTA's key, counter (k, r, 0, CTA):
// the blocks of every thread are XOR-folded into one word per CTA.
__global__ void __launch_bounds__(512, 2) philox_rate_kernel(int iters, uint32_t *sink)
{
    const uint32_t key0 = 0x9E3779B9u * (blockIdx.x + 1), key1 = 0x85EBCA6Bu ^ blockIdx.x;
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
        const PhiloxPrefix P = philox_prefix((uint32_t)(it >> 2), 0u, blockIdx.x, key0, key1);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            uint32_t x[4];
            philox_finish((uint32_t)((it & 3) * 1024 + u * 512 + threadIdx.x), P, key0, key1, x);
            acc ^= x[0] ^ x[1] ^ x[2] ^ x[3];
        }
    }
    acc = __reduce_xor_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0) atomicXor(&sink[blockIdx.x & 15], acc);
}

// iters barriers of the whole cluster (kCluster) or of the CTA; the dynamic
// shared memory only keeps one CTA per SM, as in the persistent kernels
template <bool kCluster>
__global__ void __launch_bounds__(1024) barrier_kernel(int iters, unsigned *sink)
{
    unsigned acc = threadIdx.x;
    if (kCluster) {
        cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
        for (int it = 0; it < iters; ++it) {
            cl.sync();
            acc += (unsigned)it;
        }
    } else {
        for (int it = 0; it < iters; ++it) {
            __syncthreads();
            acc += (unsigned)it;
        }
    }
    if (acc == 0xFFFFFFFFu) sink[0] = acc;            // keeps the loop
}

static double time_ms(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return (double)ms;
}

int microbench(int kind, int device, double *result)
{
    cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    void *sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return CG_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    cudaError_t err = cudaSuccess;
    if (kind == 0 || kind == 2) {
        const int word = kind == 0 ? 4 : 8;
        const int smem = 16384 * word;
        const int iters = 200, blocks = 2 * sms;
        // integer adds keep the ALU side trivial next to the shared-memory
        // traffic (a binary64 add would measure GB300's slow FP64 pipe)
        if (kind == 0)
            err = cudaFuncSetAttribute(smem_rmw_kernel<unsigned int>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        else
            err = cudaFuncSetAttribute(smem_rmw_kernel<unsigned long long>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
            cudaEventRecord(e0);
            if (kind == 0)
                smem_rmw_kernel<unsigned int><<<blocks, 1024, smem>>>(iters, (unsigned int *)sink);
            else
                smem_rmw_kernel<unsigned long long>
                    <<<blocks, 1024, smem>>>(iters, (unsigned long long *)sink);
            cudaEventRecord(e1);
            err = cudaEventSynchronize(e1);
            const double bytes = 2.0 * word * 16384.0 * iters * blocks;   // load + store
            const double rate = bytes / (time_ms(e0, e1) * 1e-3);
            if (rep > 0 && rate > best) best = rate;
        }
    } else if (kind == 1) {
        const int iters = 4096, blocks = 8 * sms;
        for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
            cudaEventRecord(e0);
            dadd_kernel<<<blocks, 256>>>(iters, 1.0, (double *)sink);
            cudaEventRecord(e1);
            err = cudaEventSynchronize(e1);
            const double adds = 8.0 * iters * 256.0 * blocks;
            const double rate = adds / (time_ms(e0, e1) * 1e-3);
            if (rep > 0 && rate > best) best = rate;
        }
    } else if (kind == 3) {
        const int iters = 2048, blocks = 2 * sms;
        for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
            cudaEventRecord(e0);
            philox_rate_kernel<<<blocks, 512>>>(iters, (uint32_t *)sink);
            cudaEventRecord(e1);
            err = cudaEventSynchronize(e1);
            const double labels = 2.0 * iters * 512.0 * blocks;
            const double rate = labels / (time_ms(e0, e1) * 1e-3);
            if (rep > 0 && rate > best) best = rate;
        }
    } else if (kind >= 4 && kind <= 7) {
        const int C = kind == 4 ? 2 : kind == 5 ? 4 : kind == 6 ? 8 : 1;
        const int smem = 120 * 1024;                      // one CTA per SM
        const int blocks = (sms / C) * C;
        auto kern = C > 1 ? barrier_kernel<true> : barrier_kernel<false>;
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        double ms_short = 0.0;
        best = 1e30;
        for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
            for (int len = 0; len < 2 && err == cudaSuccess; ++len) {
                const int iters = len ? 4096 : 1024;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)blocks, 1, 1);
                cfg.blockDim = dim3(1024, 1, 1);
                cfg.dynamicSmemBytes = (size_t)smem;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = (unsigned)C;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = C > 1 ? 1 : 0;
                cudaEventRecord(e0);
                err = cudaLaunchKernelEx(&cfg, kern, iters, (unsigned *)sink);
                cudaEventRecord(e1);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                const double ms = time_ms(e0, e1);
                if (!len) {
                    ms_short = ms;
                } else if (rep > 0) {
                    const double t = (ms - ms_short) * 1e-3 / 3072.0;
                    if (t < best) best = t;
                }
            }
        }
    } else {
        err = cudaErrorInvalidValue;
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return CG_ECUDA;
    *result = best;
    return CG_OK;
}

}  // namespace cg
