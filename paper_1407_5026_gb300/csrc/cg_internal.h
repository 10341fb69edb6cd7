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
    int status;                        // CG_OK, CG_ESTUCK or CG_ETIMEOUT
    float m_ema;                       // running mean of attempts per hop (chunk sizing)
    int trace_count;                   // points recorded
    int trace_cap;                     // trace capacity (0: no trace)
    double trace_next;                 // attempt count of the next trace point
    double trace_ratio;                // ratio between consecutive trace points
    double time;                       // stochastic time (CG_TIME_GAUSSIAN), else 0
};

// Guide table of the tower: bucket b = x1 >> (32 - kGuideBits) holds the
// smallest vector index whose threshold is >= the bucket's first value (14
// bits), bit 15 set when a threshold falls strictly inside the bucket (one
// compare decides between that vector and the next) and bit 14 when two or
// more do (a scan finds the exact vector); see tower_lookup.
constexpr int kGuideBits = 12;
constexpr int kGuide = 1 << kGuideBits;

// Everything one CTA needs to run one replica.
struct alignas(16) DevReplica {
    int L, N, H1, V;          // side, sites, folded extent L/2+1, hop vectors
    int words;                // occupation bitmask words, ceil(N/32)
    unsigned int magicL;      // y = umulhi(s, magicL) == s / L for s < N
    unsigned int key0, key1;  // Philox key (seed lo, seed hi)
    unsigned int replica;     // Philox counter word 3
    int dim;                  // 2 (square lattice) or 3 (cubic lattice)
    unsigned int pair_T;      // two-electron hops: a label pairs iff its word x3 < pair_T
    int pair_R;               // their offset bound |e| <= pair_R
    double nu, T, E;
    double negC0nu;           // -nu * sum_{t != s} 1/r_st (same for every s)
    double C0;                // sum_{t != s} 1/r_st
    double Gamma;             // N * Z (/ (1 - pair_T 2^-32)), the total proposal rate
    // tables (device)
    const double *tinv64;     // H1*H1, [fy*H1 + fx] = 1/sqrt(fx^2+fy^2), 0 at origin
    const float *tinv32;      // the same rounded to binary32
    const unsigned int *thr;  // V tower thresholds C_k - 1
    const int *disp;          // V packed hop vectors: (dx & 0xffff) | (dy << 16)
    const double *tinvd;      // V: 1/r of each hop vector (binary64)
    const double *tinv_r2_64; // cubic lattice: 1/r by r^2 = fx^2+fy^2+fz^2, 3 (L/2)^2 + 1
    const float *tinv_r2_32;  // entries (the folded table's values); null on the square one
    const unsigned short *guide; // kGuide entries
    // state (device)
    void *eps;                // N binary64 (CG_FP64) or binary32 (CG_FP32)
    unsigned int *occ;        // occupation bitmask, bit s%32 of word s/32
    const double *phi;        // N site energies
    DevCounters *ctr;
    cg_hop *log;              // NULL, or n_hops entries for this replica
    cg_trace_point *trace;    // NULL, or ctr->trace_cap points
    // random-site geometry (CG_SITES_RANDOM; null otherwise)
    const double *G;          // N x N minimum-image 1/r, 0 on the diagonal
    const int *rguide;        // 16 ints per site: kRandomGuide layout
    const uint2 *rrec;        // per pair: C mod 2^32, partner j | (C >> 32) << 31 (C <= 2^32)
    const double2 *rgx;       // per pair: 1/r, E dx (minimum-image dx, binary64)
    int rguide_small;         // 1: every partner list holds at most 255 pairs
};

// Thread 0 at commit: record trace points whose attempt threshold the
// replica's attempt count has reached (several if one hop spans them).
__device__ __forceinline__ void trace_hop(const DevReplica &Rg, unsigned long long attempts,
                                          unsigned long long hops, long long P, double energy,
                                          int time_mode, double time)
{
    DevCounters *c = Rg.ctr;
    if (!Rg.trace || c->trace_count >= c->trace_cap || (double)attempts < c->trace_next) return;
    cg_trace_point pt;
    pt.attempts = attempts;
    pt.hops = hops;
    pt.P = P;
    pt.energy = energy;
    pt.time = time_mode ? time : __ddiv_rn((double)attempts, Rg.Gamma);
    Rg.trace[c->trace_count++] = pt;
    double next = c->trace_next;
    while (next <= (double)attempts) next = next * c->trace_ratio > next + 1.0 ? next * c->trace_ratio : next + 1.0;
    c->trace_next = next;
}

struct RunArgs {
    unsigned long long n_hops;     // hops every replica executes in this launch
    unsigned long long max_rounds; // rounds per hop before CG_ESTUCK
    unsigned long long log_offset; // index of this launch's first hop in each log
    unsigned long long hop_timeout_ns; // wall-clock limit of one hop
    unsigned long long hop_timeout_cyc; // the same in SM cycles at the peak clock
    unsigned int M;                // labels per round
    int toy;                       // constant-acceptance test mode
    int time_mode;                 // CG_TIME_DETERMINISTIC or CG_TIME_GAUSSIAN
    int pair;                      // 1: two-electron hops (the kPair instances)
    int smem_guide;                // random sites, one CTA: guide records in shared memory
    double toy_A0;
};

// Shared-memory carve-up of the persistent kernel (bytes, 16-aligned).
struct SmemLayout {
    int off_eps, off_tinv, off_occ, off_guide, off_thr, off_disp;
    int off_vr64, off_edx64, off_cv32, total;
};

__host__ __device__ inline int cg_align16(int x) { return (x + 15) & ~15; }

// tab_entries: (L/2+1)^dim entries of the folded 1/r table
__host__ __device__ inline SmemLayout smem_layout(int N, int tab_entries, int V, int words,
                                                  int real_bytes)
{
    SmemLayout s;
    int o = 0;
    s.off_eps = o;   o = cg_align16(o + N * real_bytes);
    s.off_tinv = o;  o = cg_align16(o + tab_entries * real_bytes);
    s.off_occ = o;   o = cg_align16(o + words * 4);
    s.off_guide = o; o = cg_align16(o + kGuide * 2);
    s.off_thr = o;   o = cg_align16(o + V * 4);
    s.off_disp = o;  o = cg_align16(o + V * 4);
    s.off_vr64 = o;  o = cg_align16(o + V * 8);
    s.off_edx64 = o; o = cg_align16(o + V * 8);
    s.off_cv32 = o;  o = cg_align16(o + V * 4);
    s.total = o;
    return s;
}

// Random sites (cg_pr_random.cu): the coupling matrix from the positions,
// eps from its definition, and the persistent binary64 PR kernel.
cudaError_t launch_g_build(const double *px, const double *py, int L, int N, double *G,
                           cudaStream_t st);
cudaError_t launch_eps_init_random(const DevReplica *d_rep, int N, cudaStream_t st);
cudaError_t launch_pr_random(const DevReplica *d_reps, const int *d_index, int n_ctas,
                             int threads, int smem_bytes, const RunArgs &args, cudaStream_t st);
cudaError_t set_pr_random_smem_limit(int bytes);
// The per-site record of a random-site partner list (16 ints, 64 bytes):
// [0] first pair of the list, [1] one past its last; [2], [3] the list's
// last running weight (lo, hi words); [4 + b/2] holds, in its low (b even)
// or high (b odd) 16 bits, b = 0..15, the offset from [0] of the pair that
// x1 = b 2^28 selects (the smallest m with b 2^28 < C_m; the last pair when
// none); [12..15] unused.  A label with x1 in bucket b = x1 >> 28 finds its
// pair in [start(b), min(start(b + 1), [1] - 1)], start(16) = [1].
// The offsets are 16 bits: the library refuses lists of 2^16 or more pairs.
constexpr int kRandomGuide = 16;
constexpr int kRandomBuckets = 16;
// Sites whose eps a CTA of a C-CTA cluster owns: ceil(N / C) rounded up to a
// multiple of 32 (CTA rank owns [rank Nc, min(N, (rank + 1) Nc))).
__host__ __device__ inline int random_cluster_sites(int N, int C)
{
    return C <= 1 ? N : (((N + C - 1) / C + 31) / 32) * 32;
}
// Dynamic shared memory of a random-site CTA: its eps (binary64) and the
// whole occupation bitmask; with guide = true (one CTA per replica, every
// list below 256 pairs) also each site's guide record compacted to 32 bytes
// (kRandomGuideSmem): first pair, the last running weight (33 bits), the
// list's length (16 bits) and the 16 bucket starts as 8-bit offsets.
constexpr int kRandomGuideSmem = 32;
inline int random_smem_bytes(int N, int C = 1, bool guide = false)
{
    return cg_align16(random_cluster_sites(N, C) * 8) + cg_align16(((N + 31) / 32) * 4) +
           (guide ? N * kRandomGuideSmem : 0);
}
// The random-site chain on clusters of `cluster` (2, 4 or 8) CTAs per replica
// (cg_pr_random_cluster.cu); grid = n_reps * cluster CTAs of 256, 512 or 1024
// threads.
cudaError_t launch_pr_random_cluster(const DevReplica *d_reps, const int *d_index, int n_reps,
                                     int cluster, int threads, int smem_bytes,
                                     const RunArgs &args, cudaStream_t st);

// Launchers (defined in the .cu files).
cudaError_t launch_pr_persistent(int precision, const DevReplica *d_reps,
                                 const int *d_index, int n_ctas, int threads,
                                 int smem_bytes, const RunArgs &args,
                                 cudaStream_t st, int L, int dim);
// The cubic-lattice instances (cg_pr_kernel3d.cu).
cudaError_t launch_pr_persistent3(int precision, const DevReplica *d_reps, const int *d_index,
                                  int n_ctas, int threads, int smem_bytes, const RunArgs &args,
                                  cudaStream_t st, int L);
cudaError_t set_pr3_smem_limit(int precision, int bytes);
// The cubic lattice with two-electron hops (cg_pr_kernel3d_pair.cu).
cudaError_t launch_pr_persistent3_pair(int precision, const DevReplica *d_reps,
                                       const int *d_index, int n_ctas, int threads,
                                       int smem_bytes, const RunArgs &args, cudaStream_t st,
                                       int L);
cudaError_t set_pr3_pair_smem_limit(int precision, int bytes);
// The two-electron-hop instances (cg_pr_kernel_pair.cu): square lattice, one
// CTA per replica.
cudaError_t launch_pr_persistent_pair(int precision, const DevReplica *d_reps,
                                      const int *d_index, int n_ctas, int threads,
                                      int smem_bytes, const RunArgs &args, cudaStream_t st,
                                      int L);
cudaError_t set_pr_pair_smem_limit(int precision, int bytes);
// ... and with the stochastic clock (cg_pr_kernel_pair_time.cu).
cudaError_t launch_pr_persistent_pair_time(int precision, const DevReplica *d_reps,
                                           const int *d_index, int n_ctas, int threads,
                                           int smem_bytes, const RunArgs &args, cudaStream_t st,
                                           int L);
cudaError_t set_pr_pair_time_smem_limit(int precision, int bytes);
// The same chain over a thread-block cluster of `cluster` CTAs per replica
// (eps split by rows, or by z-planes on the cubic lattice, dim = 3);
// grid = n_reps * cluster CTAs.
cudaError_t launch_pr_cluster(int precision, const DevReplica *d_reps, const int *d_index,
                              int n_reps, int cluster, int threads, int smem_bytes,
                              const RunArgs &args, cudaStream_t st, int L, int dim);
// Its two-electron-hop instances (cg_pr_cluster_pair.cu).
cudaError_t launch_pr_cluster_pair(int precision, const DevReplica *d_reps, const int *d_index,
                                   int n_reps, int cluster, int threads, int smem_bytes,
                                   const RunArgs &args, cudaStream_t st, int L, int dim);
cudaError_t launch_eps_init(const DevReplica *d_rep, int N, int tab_entries, int words,
                            int precision, cudaStream_t st);
cudaError_t launch_refresh_fp64(const DevReplica *d_rep, int N, int tab_entries, int words,
                                cudaStream_t st);
cudaError_t launch_debug_philox(const uint32_t *ctr, const uint32_t *key,
                                uint32_t *out, int n, cudaStream_t st);
cudaError_t launch_debug_exp(const double *x, double *out, int n, cudaStream_t st);
cudaError_t launch_debug_gauss(const uint64_t *seed, const uint32_t *rep, const uint64_t *hop,
                               double *z, int n, cudaStream_t st);
cudaError_t launch_debug_tower(const unsigned short *guide, const unsigned *thr, int V,
                               const uint32_t *x1, int *out, int n, cudaStream_t st);
cudaError_t set_pr_smem_limit(int precision, int bytes);
int microbench(int kind, int device, double *result);
// Histogram of eps (binary64 or binary32 by precision) of `count` replicas
// starting at d_reps, added to the nbins counters at out.
cudaError_t launch_eps_histogram(const DevReplica *d_reps, int count, int max_N, int precision,
                                 int nbins, double lo, double scale, unsigned long long *out,
                                 cudaStream_t st);
cudaError_t launch_reset_refresh_err(const DevReplica *d_reps, const int *d_index, int R,
                                     cudaStream_t st);
// log2 of the factor applied to 1/r before its binary16 split (cubic lattice)
constexpr int kTcF16Log2Scale = 10;

// Tensor-core refresh of R <= 512 binary32 replicas of one L and dimension
// (dim 2: N = L^2, dim 3: N = L^3; N % 128 == 0).  d_tab: the folded table's
// two-term split (H1^dim entries; BF16 of 1/r for dim 2, binary16 of
// 2^kTcF16Log2Scale / r for dim 3).  d_scratch: refresh_tc_scratch_bytes(N, R)
// bytes (the S image and the K-split partial sums), 256-byte aligned.
cudaError_t launch_refresh_tc(const DevReplica *d_reps, const int *d_index, int R, int L,
                              int dim, const uint32_t *d_tab, unsigned char *d_scratch,
                              int *d_err, cudaStream_t st);
int refresh_tc_smem_bytes(int R_pad, int tab_entries);
// The FFT refresh of R binary32 replicas of one L = 2^m or 3 2^m (dim 2 or
// 3; cg_refresh_fft.cu): d_ghat holds DFT(g)/N (N floats), d_tw the L
// twiddles exp(-2 pi i k / L), d_buf refresh_fft_buffer_bytes.
cudaError_t launch_refresh_fft(const DevReplica *d_reps, const int *d_index, int R, int L,
                               int dim, const float *d_ghat, const float2 *d_tw, float2 *d_buf,
                               cudaStream_t st);
size_t refresh_fft_buffer_bytes(int N, int R);
bool refresh_fft_size_ok(int L);      // L = 2^m (4..1024) or 3 2^m (6..192)
int refresh_tc_ksplit(int N, int dim);
int refresh_tc_max_replicas(int dim);   // replicas per launch
size_t refresh_tc_scratch_bytes(int N, int dim, int R);

}  // namespace cg
