// cg_pr_kernel_pair_time.cu -- the two-electron-hop instances of the
// persistent parallel-rejection kernel (cg_pr_persistent.cuh) with the
// stochastic clock of step 3c (CG_TIME_GAUSSIAN), square lattice, L known at
// run time.
#include "cg_pr_persistent.cuh"

namespace cg {

template <typename Real, int kThreads>
static cudaError_t launch_pt(const DevReplica *d_reps, const int *d_index, int n_ctas,
                             int smem_bytes, const RunArgs &args, cudaStream_t st, int L)
{
    if ((L & (L - 1)) == 0)
        pr_persistent<Real, kThreads, 0, true, 2, true>
            <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
    else
        pr_persistent<Real, kThreads, -1, true, 2, true>
            <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
    return cudaGetLastError();
}

template <typename Real, int kThreads>
static cudaError_t set_pt_one(int bytes)
{
    const void *k[2] = {(const void *)pr_persistent<Real, kThreads, 0, true, 2, true>,
                        (const void *)pr_persistent<Real, kThreads, -1, true, 2, true>};
    for (const void *f : k) {
        const cudaError_t e =
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e) return e;
    }
    return cudaSuccess;
}

cudaError_t set_pr_pair_time_smem_limit(int precision, int bytes)
{
    cudaError_t e;
    if (precision == CG_FP64) {
        if ((e = set_pt_one<double, 1024>(bytes)) || (e = set_pt_one<double, 512>(bytes)) ||
            (e = set_pt_one<double, 384>(bytes)) || (e = set_pt_one<double, 256>(bytes)))
            return e;
    } else {
        if ((e = set_pt_one<float, 1024>(bytes)) || (e = set_pt_one<float, 512>(bytes)) ||
            (e = set_pt_one<float, 384>(bytes)) || (e = set_pt_one<float, 256>(bytes)))
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pr_persistent_pair_time(int precision, const DevReplica *d_reps,
                                           const int *d_index, int n_ctas, int threads,
                                           int smem_bytes, const RunArgs &args, cudaStream_t st,
                                           int L)
{
    if (precision == CG_FP64) {
        switch (threads) {
        case 1024: return launch_pt<double, 1024>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 512: return launch_pt<double, 512>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 384: return launch_pt<double, 384>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 256: return launch_pt<double, 256>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        }
    } else {
        switch (threads) {
        case 1024: return launch_pt<float, 1024>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 512: return launch_pt<float, 512>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 384: return launch_pt<float, 384>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 256: return launch_pt<float, 256>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace cg
