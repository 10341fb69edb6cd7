// cg_internal.h -- structures shared by the host side of libcg and its
// kernels.  Not part of the public ABI (include/cg.h is).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/cg.h"

namespace cg {

// Device-resident counters of one replica (written back at the end of every
// persistent launch; read by cg_read_state / cg_observables).
struct alignas(16) DevCounters {
    unsigned long long rounds;
    unsigned long long hops;
    unsigned long long attempts;
    unsigned long long evaluated;
    long long P;
    double energy;
    unsigned long long cycles_reject;
    unsigned long long cycles_update;
    unsigned long long refreshes;
    unsigned long long max_err_bits;   // max |eps - eps_ref| of the last refresh (binary64 bits)
    int status;                        // CG_OK or CG_ESTUCK
    int pad_[3];
};

// Everything one CTA needs to run one replica.
struct alignas(16) DevReplica {
    int L, N, H1, V;          // side, sites, folded extent L/2+1, hop vectors
    int words;                // occupation bitmask words, ceil(N/32)
    unsigned int magicL;      // y = umulhi(s, magicL) == s / L for s < N
    unsigned int key0, key1;  // Philox key (seed lo, seed hi)
    unsigned int replica;     // Philox counter word 3
    int pad0_;
    double nu, T, E;
    double negC0nu;           // -nu * sum_{t != s} 1/r_st (same for every s)
    // tables (device)
    const double *tinv64;     // H1*H1, [fy*H1 + fx] = 1/sqrt(fx^2+fy^2), 0 at origin
    const float *tinv32;      // the same rounded to binary32
    const unsigned int *thr;  // V tower thresholds C_k - 1
    const int *disp;          // V packed hop vectors: (dx & 0xffff) | (dy << 16)
    const double *tinvd;      // V: 1/r of each hop vector (binary64)
    // state (device)
    void *eps;                // N binary64 (CG_FP64) or binary32 (CG_FP32)
    unsigned int *occ;        // occupation bitmask, bit s%32 of word s/32
    const double *phi;        // N site energies
    DevCounters *ctr;
    cg_hop *log;              // NULL, or n_hops entries for this replica
};

struct RunArgs {
    unsigned long long n_hops;     // hops every replica executes in this launch
    unsigned long long max_rounds; // rounds per hop before CG_ESTUCK
    unsigned long long log_offset; // index of this launch's first hop in each log
    unsigned long long hop_timeout_ns; // wall-clock limit of one hop
    unsigned int M;                // labels per round
    int toy;                       // constant-acceptance test mode
    double toy_A0;
};

// Shared-memory carve-up of the persistent kernel (bytes, 16-aligned).
struct SmemLayout {
    int off_eps, off_tinv, off_occ, off_thr, off_disp, off_tinvd, total;
};

__host__ __device__ inline int cg_align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SmemLayout smem_layout(int N, int H1, int V, int words,
                                                  int real_bytes)
{
    SmemLayout s;
    int o = 0;
    s.off_eps = o;   o = cg_align16(o + N * real_bytes);
    s.off_tinv = o;  o = cg_align16(o + H1 * H1 * real_bytes);
    s.off_occ = o;   o = cg_align16(o + words * 4);
    s.off_thr = o;   o = cg_align16(o + V * 4);
    s.off_disp = o;  o = cg_align16(o + V * 4);
    s.off_tinvd = o; o = cg_align16(o + V * 8);
    s.total = o;
    return s;
}

// Launchers (defined in the .cu files).
cudaError_t launch_pr_persistent(int precision, const DevReplica *d_reps,
                                 const int *d_index, int n_ctas, int threads,
                                 int smem_bytes, const RunArgs &args,
                                 cudaStream_t st);
int pr_persistent_max_threads(int precision);
cudaError_t launch_eps_init(const DevReplica *d_rep, int N, int H1, int words,
                            int precision, cudaStream_t st);
cudaError_t launch_refresh_fp64(const DevReplica *d_rep, int N, int H1, int words,
                                cudaStream_t st);
cudaError_t launch_debug_philox(const uint32_t *ctr, const uint32_t *key,
                                uint32_t *out, int n, cudaStream_t st);
cudaError_t launch_debug_exp(const double *x, double *out, int n, cudaStream_t st);
cudaError_t set_pr_smem_limit(int precision, int bytes);
int microbench(int kind, int device, double *result);

}  // namespace cg
