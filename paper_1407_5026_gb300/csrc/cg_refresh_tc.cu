// cg_refresh_tc.cu -- the periodic eps refresh of the binary32 form as one
// tensor-core contraction over all replicas of one lattice size.
//
// The single-particle energies below Eq. 2 are eps_s = phi_s + sum_t
// G_st (n_t - nu) with G_st = 1/r_st (0 for s = t).  With S_t = 2 n_t - 1 =
// +-1 (exact in BF16) this is
//     eps_s = phi_s + D_s / 2 + (1/2 - nu) C0,   D = G S,   C0 = sum_t G_st,
// and for R replicas of one L the matrix S has R columns, so D = G S is an
// (N x N) x (N x R) product.  G is split as G_hi + G_lo (two BF16 terms,
// residual ~2^-17 |G|) and both products accumulate in FP32 in tensor memory.
// On the cubic lattice, where sum_t G_st^2 is about eight times larger, the
// split is instead two binary16 terms of 2^10 G (residual ~2^-22 |G|), with S
// in binary16 too; the reduction undoes the scale in binary64.
//
// Kernel layout (one CTA per 128 sites, 288 threads):
//   warps 0-7  generate the 128 x 64 tiles of G_hi and G_lo for each K-block
//              from the folded 1/r table into 128B-swizzled shared memory
//              (G is never stored), then run the epilogue; on the cubic
//              lattice (kDim = 3) the table is (L/2+1)^3 and a site decodes
//              to (x, y, z);
//   warp 8     bulk-copies the K-block of S (a pre-swizzled BF16 image built
//              by pack_s_kernel) with cp.async.bulk and, from one lane,
//              issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
//              N = up to 256 per instruction) into the TMEM accumulator.
// Two pipeline stages; every mbarrier wait is bounded in time and on expiry
// sets an error word, stops the CTA's loops, waits for its own MMAs and frees
// its tensor memory before returning.
#include <cmath>

#include "cg_device.cuh"
#include "cg_internal.h"

namespace cg {

namespace tc {

constexpr int kThreads = 288;
constexpr int kGenThreads = 256;
constexpr int kStages = 2;
constexpr int kTileBytes = 128 * 128;   // 128 rows x 64 BF16
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; false when the time limit or the
// CTA's abort flag ends the wait first.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (now_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulator.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte rows swizzled in
// 1024-byte atoms (8 rows), consecutive 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3ffffu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// The same with A and B in binary16 (format 0): FP32 accumulator.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

}  // namespace tc

// S image: for K-block kb (64 sites) and replica row r, 128 bytes holding
// S_t = 2 n_t - 1 (one = the 16-bit pattern of +1: BF16 0x3f80 or binary16
// 0x3c00; -1 adds the sign bit) for t = 64 kb ... 64 kb + 63, 16-byte chunk c
// stored at chunk c ^ (r & 7) (the 128-byte swizzle); rows r >= R are zero.
__global__ void pack_s_kernel(const DevReplica *__restrict__ reps, const int *__restrict__ index,
                              int R, int R_pad, int kblocks, uint32_t one,
                              unsigned char *__restrict__ img)
{
    const long long total = (long long)kblocks * R_pad * 8;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(g & 7);
        const int r = (int)((g >> 3) % R_pad);
        const int kb = (int)((g >> 3) / R_pad);
        uint4 out = make_uint4(0u, 0u, 0u, 0u);
        if (r < R) {
            const DevReplica &Rr = reps[index[r]];
            const int t0 = kb * 64 + c * 8;
            const unsigned bits = (Rr.occ[t0 >> 5] >> (t0 & 31)) & 0xffu;
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t lo = ((bits >> (2 * e)) & 1u) ? one : (one | 0x8000u);
                const uint32_t hi = ((bits >> (2 * e + 1)) & 1u) ? one : (one | 0x8000u);
                w[e] = lo | (hi << 16);
            }
            out = make_uint4(w[0], w[1], w[2], w[3]);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(img + ((size_t)kb * R_pad + r) * 128 +
                                               (size_t)((c ^ (r & 7)) * 16));
        *dst = out;
    }
}

struct TcArgs {
    const DevReplica *reps;
    const int *index;        // the group's replicas
    int R, R_pad, n0, n1;    // n0 + n1 = R_pad, each a multiple of 16, n0 <= 256
    int L, N, H1, kblocks;
    int kb_per;              // K-blocks per CTA (the K range is split over gridDim.y)
    int tab_entries;         // H1^2 (square lattice) or H1^3 (cubic lattice)
    int lo_off;              // TMEM column of the G_lo accumulator (0: shared with G_hi)
    unsigned magicL;
    uint32_t tmem_cols;
    const uint32_t *tab;     // folded table: BF16 hi | BF16 lo << 16 of 1/r
    const unsigned char *img;
    float *part;             // gridDim.y x R_pad x N partial sums of D
    int *err;                // set nonzero when a bounded wait expired
};

template <int kDim>
__global__ void __launch_bounds__(tc::kThreads, 1) refresh_tc_kernel(TcArgs a)
{
    using namespace tc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bars[3 * kStages + 1];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    // 1024-byte aligned stage buffers (the swizzle atom)
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const int b_bytes = a.R_pad * 128;
    const int stage_bytes = 2 * kTileBytes + b_bytes;
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem + kStages * stage_bytes);
    uint64_t *full_a = bars, *full_b = bars + kStages, *empty = bars + 2 * kStages;
    uint64_t *done = bars + 3 * kStages;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full_a[s], kGenThreads);
            mbar_init(&full_b[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        s_abort = 0;
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&s_tmem, a.tmem_cols);
    for (int l = tid; l < a.tab_entries; l += tc::kThreads) tab[l] = a.tab[l];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int *abort_flag = &s_abort;

    const int L = a.L, H1 = a.H1;
    const int m0 = blockIdx.x * 128;
    const int kb0 = blockIdx.y * a.kb_per;

    if (warp < 8) {
        // ---- G tile generators: thread -> row (site s), half of the 8 chunks ----
        const int row = tid & 127, half = tid >> 7;
        const int s = m0 + row;
        int xs, ys, zs = 0;
        if (kDim == 3) {
            const unsigned q = __umulhi((unsigned)s, a.magicL);    // s / L
            xs = s - (int)q * L;
            zs = (int)__umulhi(q, a.magicL);                      // s / L^2
            ys = (int)q - zs * L;
        } else {
            ys = (int)__umulhi((unsigned)s, a.magicL);
            xs = s - ys * L;
        }
        for (int kk = 0; kk < a.kb_per; ++kk) {
            const int kb = kb0 + kk;
            const int st = kk % kStages, use = kk / kStages;
            if (kk >= kStages && !mbar_wait(&empty[st], (use - 1) & 1, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            unsigned char *ahi = smem + st * stage_bytes;
            unsigned char *alo = ahi + kTileBytes;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int c = half * 4 + cc;
                uint32_t whi[4], wlo[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    uint32_t v2[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int t = kb * 64 + c * 8 + 2 * e + h;
                        if (kDim == 3) {
                            const unsigned q = __umulhi((unsigned)t, a.magicL);
                            const int xt = t - (int)q * L, zt = (int)__umulhi(q, a.magicL);
                            const int yt = (int)q - zt * L;
                            v2[h] = tab[(fold_axis(zs - zt, L) * H1 + fold_axis(ys - yt, L)) * H1 +
                                        fold_axis(xs - xt, L)];
                        } else {
                            const int yt = (int)__umulhi((unsigned)t, a.magicL), xt = t - yt * L;
                            v2[h] = tab[fold_axis(ys - yt, L) * H1 + fold_axis(xs - xt, L)];
                        }
                    }
                    whi[e] = (v2[0] & 0xffffu) | (v2[1] << 16);
                    wlo[e] = (v2[0] >> 16) | (v2[1] & 0xffff0000u);
                }
                const int off = row * 128 + ((c ^ (row & 7)) << 4);
                *reinterpret_cast<uint4 *>(ahi + off) = make_uint4(whi[0], whi[1], whi[2], whi[3]);
                *reinterpret_cast<uint4 *>(alo + off) = make_uint4(wlo[0], wlo[1], wlo[2], wlo[3]);
            }
            fence_proxy_async();
            mbar_arrive(&full_a[st]);
        }
    } else if (lane == 0) {
        // ---- S loader and MMA issuer ----
        // both operands in one format: BF16 (square lattice) or binary16 (cubic)
        const uint32_t id0 = kDim == 3 ? idesc_f16(128, a.n0) : idesc_bf16(128, a.n0);
        const uint32_t id1 = a.n1 ? (kDim == 3 ? idesc_f16(128, a.n1) : idesc_bf16(128, a.n1))
                                  : 0u;
        for (int kk = 0; kk < a.kb_per; ++kk) {
            const int kb = kb0 + kk;
            const int st = kk % kStages, use = kk / kStages;
            if (kk >= kStages && !mbar_wait(&empty[st], (use - 1) & 1, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            unsigned char *stage = smem + st * stage_bytes;
            unsigned char *bsm = stage + 2 * kTileBytes;
            mbar_arrive_tx(&full_b[st], (uint32_t)b_bytes);
            bulk_g2s(bsm, a.img + (size_t)kb * b_bytes, (uint32_t)b_bytes, &full_b[st]);
            if (!mbar_wait(&full_a[st], use & 1, abort_flag) ||
                !mbar_wait(&full_b[st], use & 1, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t ahi = smem_u32(stage), alo = ahi + kTileBytes, b = smem_u32(bsm);
#pragma unroll
            // G_lo products go to their own accumulator when lo_off > 0, which
            // halves the adds into each (the accumulation error grows with
            // their count)
            const uint32_t tlo = tmem + (uint32_t)a.lo_off;
            for (int ks = 0; ks < 4; ++ks) {
                const uint32_t koff = ks * 32;    // 16 elements along K
                const uint32_t acc = (kk > 0 || ks > 0) ? 1u : 0u;
                const uint32_t acc_lo = a.lo_off ? acc : 1u;
                mma_bf16(tmem, sw128_desc(ahi + koff), sw128_desc(b + koff), id0, acc);
                mma_bf16(tlo, sw128_desc(alo + koff), sw128_desc(b + koff), id0, acc_lo);
                if (a.n1) {
                    const uint32_t b1 = b + a.n0 * 128;
                    mma_bf16(tmem + a.n0, sw128_desc(ahi + koff), sw128_desc(b1 + koff), id1, acc);
                    mma_bf16(tlo + a.n0, sw128_desc(alo + koff), sw128_desc(b1 + koff), id1, acc_lo);
                }
            }
            mma_commit(&empty[st]);
        }
        mma_commit(done);   // arrives once every MMA issued above has completed
    }
    __syncwarp();

    // ---- epilogue: this CTA's partial D for its 128 sites and every replica ----
    const bool ok = mbar_wait(done, 0, abort_flag) && !*abort_flag;
    tc_fence_after();
    if (warp < 8 && ok) {
        const int lane_base = 32 * (warp & 3);
        const int s = m0 + lane_base + lane;
        float *part = a.part + (size_t)blockIdx.y * a.R_pad * a.N;
        for (int c = (warp >> 2); c * 16 < a.R_pad; c += 2) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(c * 16), v);
            if (a.lo_off) {
                uint32_t w[16];
                tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(a.lo_off + c * 16), w);
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    v[e] = __float_as_uint(__uint_as_float(v[e]) + __uint_as_float(w[e]));
            }
#pragma unroll
            for (int e = 0; e < 16; ++e)
                part[(size_t)(c * 16 + e) * a.N + s] = __uint_as_float(v[e]);
        }
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, a.tmem_cols);
    }
}

// D = sum of the K-split partials in binary64, then eps = phi + D/2 +
// (1/2 - nu) C0 for replica blockIdx.y (half = 1/2, or 2^-11 when the
// contraction ran on 2^10 / r); the largest |eps_old - eps_new| of the replica
// goes to its counters.
__global__ void __launch_bounds__(256) refresh_tc_reduce_kernel(
    const DevReplica *__restrict__ reps, const int *__restrict__ index, int R_pad, int N,
    int ksplit, double half, const float *__restrict__ part)
{
    const int r = blockIdx.y;
    const int s = blockIdx.x * 256 + threadIdx.x;
    const DevReplica &Rr = reps[index[r]];
    double err = 0.0;
    if (s < N) {
        double D = 0.0;
        for (int y = 0; y < ksplit; ++y) D += (double)part[((size_t)y * R_pad + r) * N + s];
        float *eps = reinterpret_cast<float *>(Rr.eps);
        const double enew = Rr.phi[s] + (half * D + (0.5 - Rr.nu) * Rr.C0);
        err = fabs((double)eps[s] - enew);
        eps[s] = __double2float_rn(enew);
    }
    unsigned long long bits = (unsigned long long)__double_as_longlong(err);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = bits > other ? bits : other;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&Rr.ctr->max_err_bits, bits);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&Rr.ctr->refreshes, 1ull);
}

int refresh_tc_smem_bytes(int R_pad, int tab_entries)
{
    return 1024 + tc::kStages * (2 * tc::kTileBytes + R_pad * 128) + tab_entries * 4;
}

// K split of the contraction.  Square lattice: the largest divisor of the
// K-block count that is at most max(8, K-blocks / 32), so each CTA's FP32
// partial sum covers at most an eighth of the lattice and at most 32 K-blocks
// (2048 sites) on large ones.  Cubic lattice (larger sums of G^2, so a
// tighter bound on the accumulation): the smallest divisor that leaves at most
// 16 K-blocks (1024 sites) per CTA.
int refresh_tc_ksplit(int N, int dim)
{
    const int kblocks = N / 64;
    if (dim == 3) {
        for (int k = 1; k <= kblocks; ++k)
            if (kblocks % k == 0 && kblocks / k <= 16) return k;
        return kblocks;
    }
    const int cap = kblocks / 32 > 8 ? kblocks / 32 : 8;
    for (int k = cap; k > 1; --k)
        if (kblocks % k == 0) return k;
    return 1;
}

int refresh_tc_max_replicas(int dim)
{
    return dim == 3 ? 256 : 512;   // TMEM columns: one accumulator, or G_hi and G_lo apart
}

size_t refresh_tc_scratch_bytes(int N, int dim, int R)
{
    const size_t R_pad = (size_t)(R + 15) / 16 * 16;
    const size_t img = 2 * (size_t)N * R_pad;
    const size_t part = (size_t)refresh_tc_ksplit(N, dim) * R_pad * (size_t)N * 4;
    return ((img + 255) & ~(size_t)255) + part;
}

cudaError_t launch_refresh_tc(const DevReplica *d_reps, const int *d_index, int R, int L,
                              int dim, const uint32_t *d_tab, unsigned char *d_scratch,
                              int *d_err, cudaStream_t st)
{
    const int H1 = L / 2 + 1;
    const int N = dim == 3 ? L * L * L : L * L;
    const int tab_entries = dim == 3 ? H1 * H1 * H1 : H1 * H1;
    if (N % 128 != 0 || R < 1) return cudaErrorInvalidValue;
    const int R_pad = (R + 15) / 16 * 16;
    if (R > refresh_tc_max_replicas(dim)) return cudaErrorInvalidValue;
    const int kblocks = N / 64;
    const int ksplit = refresh_tc_ksplit(N, dim);
    unsigned char *d_img = d_scratch;
    float *d_part = reinterpret_cast<float *>(
        d_scratch + ((2 * (size_t)N * R_pad + 255) & ~(size_t)255));
    pack_s_kernel<<<2 * 152, 256, 0, st>>>(d_reps, d_index, R, R_pad, kblocks,
                                           dim == 3 ? 0x3c00u : 0x3f80u, d_img);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    TcArgs a;
    a.reps = d_reps;
    a.index = d_index;
    a.R = R;
    a.R_pad = R_pad;
    a.n0 = R_pad < 256 ? R_pad : 256;
    a.n1 = R_pad - a.n0;
    a.L = L;
    a.N = N;
    a.H1 = H1;
    a.kblocks = kblocks;
    a.kb_per = kblocks / ksplit;
    a.tab_entries = tab_entries;
    a.lo_off = dim == 3 ? R_pad : 0;
    a.part = d_part;
    a.magicL = (unsigned)(4294967296ull / (unsigned long long)L + 1ull);
    uint32_t cols = 32;
    while (cols < (uint32_t)(R_pad + a.lo_off)) cols <<= 1;
    a.tmem_cols = cols;
    a.tab = d_tab;
    a.img = d_img;
    a.err = d_err;
    const int smem = refresh_tc_smem_bytes(R_pad, tab_entries);
    if (dim == 3) {
        e = cudaFuncSetAttribute(refresh_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e) return e;
        refresh_tc_kernel<3><<<dim3(N / 128, ksplit), tc::kThreads, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(refresh_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e) return e;
        refresh_tc_kernel<2><<<dim3(N / 128, ksplit), tc::kThreads, smem, st>>>(a);
    }
    e = cudaGetLastError();
    if (e) return e;
    const double half = dim == 3 ? std::ldexp(0.5, -kTcF16Log2Scale) : 0.5;
    refresh_tc_reduce_kernel<<<dim3((N + 255) / 256, R), 256, 0, st>>>(d_reps, d_index, R_pad,
                                                                     N, ksplit, half, d_part);
    return cudaGetLastError();
}

}  // namespace cg
