// cg_pr_kernel3d.cu -- launches of the persistent parallel-rejection kernel
// (cg_pr_persistent.cuh) on the L x L x L cubic lattice, with L known at run
// time (a power of two or any even L), and binary32 L = 32 fixed at compile
// time (the largest power of two whose eps fits one CTA: the octant update's
// offsets and loop counts become constants).
#include "cg_pr_persistent.cuh"

namespace cg {

template <typename Real, int kThreads, bool kTime>
static void launch3_tt(const DevReplica *d_reps, const int *d_index, int n_ctas, int smem_bytes,
                       const RunArgs &args, cudaStream_t st, int L)
{
    if constexpr (sizeof(Real) == 4) {
        if (L == 32) {
            pr_persistent<Real, kThreads, 5, kTime, 3>
                <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
            return;
        }
    }
    if ((L & (L - 1)) == 0)
        pr_persistent<Real, kThreads, 0, kTime, 3>
            <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
    else
        pr_persistent<Real, kThreads, -1, kTime, 3>
            <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
}

template <typename Real, int kThreads>
static cudaError_t launch3_t(const DevReplica *d_reps, const int *d_index, int n_ctas,
                             int smem_bytes, const RunArgs &args, cudaStream_t st, int L)
{
    if (args.time_mode)
        launch3_tt<Real, kThreads, true>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
    else
        launch3_tt<Real, kThreads, false>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
    return cudaGetLastError();
}

template <typename Real, int kThreads>
static cudaError_t set3_one(int bytes)
{
    const void *k[6] = {(const void *)pr_persistent<Real, kThreads, 0, false, 3>,
                        (const void *)pr_persistent<Real, kThreads, -1, false, 3>,
                        (const void *)pr_persistent<Real, kThreads, 0, true, 3>,
                        (const void *)pr_persistent<Real, kThreads, -1, true, 3>,
                        nullptr, nullptr};
    if constexpr (sizeof(Real) == 4) {
        k[4] = (const void *)pr_persistent<Real, kThreads, 5, false, 3>;
        k[5] = (const void *)pr_persistent<Real, kThreads, 5, true, 3>;
    }
    for (const void *f : k) {
        if (!f) continue;
        const cudaError_t e =
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e) return e;
    }
    return cudaSuccess;
}

cudaError_t set_pr3_smem_limit(int precision, int bytes)
{
    cudaError_t e = set_pr3_pair_smem_limit(precision, bytes);
    if (e) return e;
    if (precision == CG_FP64) {
        if ((e = set3_one<double, 1024>(bytes)) || (e = set3_one<double, 512>(bytes)) ||
            (e = set3_one<double, 384>(bytes)) || (e = set3_one<double, 256>(bytes)))
            return e;
    } else {
        if ((e = set3_one<float, 1024>(bytes)) || (e = set3_one<float, 512>(bytes)) ||
            (e = set3_one<float, 384>(bytes)) || (e = set3_one<float, 256>(bytes)))
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pr_persistent3(int precision, const DevReplica *d_reps, const int *d_index,
                                  int n_ctas, int threads, int smem_bytes, const RunArgs &args,
                                  cudaStream_t st, int L)
{
    if (args.pair)
        return launch_pr_persistent3_pair(precision, d_reps, d_index, n_ctas, threads, smem_bytes,
                                          args, st, L);
    if (precision == CG_FP64) {
        switch (threads) {
        case 1024: return launch3_t<double, 1024>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 512: return launch3_t<double, 512>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 384: return launch3_t<double, 384>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 256: return launch3_t<double, 256>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        }
    } else {
        switch (threads) {
        case 1024: return launch3_t<float, 1024>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 512: return launch3_t<float, 512>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 384: return launch3_t<float, 384>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 256: return launch3_t<float, 256>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace cg
