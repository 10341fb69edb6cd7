// Test probe: Philox-4x32-10 blocks from cuRAND's device API, used as an
// outside reference for all four counter words of the oracle's Philox.
//
// curand_init(seed, subsequence, offset) on a Philox state starts from the
// counter (0, 0, 0, 0) and key (seed lo, seed hi), adds `subsequence` to
// counter words 2-3 and offset / 4 to words 0-1; with offset a multiple of 4
// the first curand4() returns the block of exactly that counter.  So the
// block of counter (c0, c1, c2, c3) under key (k0, k1) is the first curand4
// after curand_init(k0 | k1 << 32, c2 | c3 << 32, 4 (c0 | c1 << 32)), which
// needs c1 < 2^30 for the offset to fit in 64 bits.
//
// Built by tests/test_gpu_philox_curand.py with nvcc into a temporary folder;
// nothing in the library uses it.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void probe_kernel(const uint4 *ctr, const uint2 *key, uint4 *out, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint4 c = ctr[t];
    const uint2 k = key[t];
    curandStatePhilox4_32_10_t s;
    const unsigned long long seed = (unsigned long long)k.x | ((unsigned long long)k.y << 32);
    const unsigned long long sub = (unsigned long long)c.z | ((unsigned long long)c.w << 32);
    const unsigned long long blk = (unsigned long long)c.x | ((unsigned long long)c.y << 32);
    curand_init(seed, sub, 4ull * blk, &s);
    out[t] = curand4(&s);
}

// n blocks: ctr_host 4n words, key_host 2n words, out_host 4n words (host
// arrays).  Returns 0, 1 for bad arguments, 2 for a CUDA error.
extern "C" int probe_philox(const uint32_t *ctr_host, const uint32_t *key_host, uint32_t *out_host,
                            int n)
{
    if (n <= 0 || !ctr_host || !key_host || !out_host) return 1;
    for (int t = 0; t < n; ++t)
        if (ctr_host[4 * t + 1] >= (1u << 30)) return 1;
    uint4 *d_ctr = nullptr, *d_out = nullptr;
    uint2 *d_key = nullptr;
    int rc = 0;
    if (cudaMalloc(&d_ctr, sizeof(uint4) * n) || cudaMalloc(&d_out, sizeof(uint4) * n) ||
        cudaMalloc(&d_key, sizeof(uint2) * n)) {
        rc = 2;
    } else if (cudaMemcpy(d_ctr, ctr_host, sizeof(uint4) * n, cudaMemcpyHostToDevice) ||
               cudaMemcpy(d_key, key_host, sizeof(uint2) * n, cudaMemcpyHostToDevice)) {
        rc = 2;
    } else {
        probe_kernel<<<(n + 127) / 128, 128>>>(d_ctr, d_key, d_out, n);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(out_host, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost))
            rc = 2;
    }
    cudaFree(d_ctr);
    cudaFree(d_out);
    cudaFree(d_key);
    return rc;
}
