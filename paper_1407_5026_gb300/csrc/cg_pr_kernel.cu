// cg_pr_kernel.cu -- launches of the persistent parallel-rejection kernel
// (cg_pr_persistent.cuh) on the square lattice, with L = 32, 48, 64, 96 and
// 128 fixed at compile time and any other L at run time; cubic lattices go
// to cg_pr_kernel3d.cu.
#include "cg_pr_persistent.cuh"

namespace cg {

template <typename Real, int kThreads, bool kTime>
static void launch_tt(const DevReplica *d_reps, const int *d_index, int n_ctas, int smem_bytes,
                      const RunArgs &args, cudaStream_t st, int L)
{
    switch (L) {
    case 32:
        pr_persistent<Real, kThreads, 5, kTime>
            <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
        break;
    case 48:
        pr_persistent<Real, kThreads, -48, kTime>
            <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
        break;
    case 96:
        pr_persistent<Real, kThreads, -96, kTime>
            <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
        break;
    case 64:
        pr_persistent<Real, kThreads, 6, kTime>
            <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
        break;
    case 128:
        pr_persistent<Real, kThreads, 7, kTime>
            <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
        break;
    default:
        if ((L & (L - 1)) == 0)
            pr_persistent<Real, kThreads, 0, kTime>
                <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
        else
            pr_persistent<Real, kThreads, -1, kTime>
                <<<n_ctas, kThreads, smem_bytes, st>>>(d_reps, d_index, args);
    }
}

template <typename Real, int kThreads>
static cudaError_t launch_t(const DevReplica *d_reps, const int *d_index, int n_ctas,
                            int smem_bytes, const RunArgs &args, cudaStream_t st, int L)
{
    if (args.time_mode)
        launch_tt<Real, kThreads, true>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
    else
        launch_tt<Real, kThreads, false>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
    return cudaGetLastError();
}

template <typename Real, int kThreads, bool kTime>
static cudaError_t set_smem_tt(int bytes)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(pr_persistent<Real, kThreads, 5, kTime>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) ||
        (e = cudaFuncSetAttribute(pr_persistent<Real, kThreads, -48, kTime>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) ||
        (e = cudaFuncSetAttribute(pr_persistent<Real, kThreads, -96, kTime>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    if ((e = cudaFuncSetAttribute(pr_persistent<Real, kThreads, 6, kTime>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    if ((e = cudaFuncSetAttribute(pr_persistent<Real, kThreads, 7, kTime>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    if ((e = cudaFuncSetAttribute(pr_persistent<Real, kThreads, 0, kTime>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    return cudaFuncSetAttribute(pr_persistent<Real, kThreads, -1, kTime>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename Real, int kThreads>
static cudaError_t set_smem_one(int bytes)
{
    cudaError_t e = set_smem_tt<Real, kThreads, false>(bytes);
    return e ? e : set_smem_tt<Real, kThreads, true>(bytes);
}

template <typename Real>
static cudaError_t set_smem_t(int bytes)
{
    cudaError_t e;
    if ((e = set_smem_one<Real, 1024>(bytes))) return e;
    if ((e = set_smem_one<Real, 512>(bytes))) return e;
    if ((e = set_smem_one<Real, 384>(bytes))) return e;
    return set_smem_one<Real, 256>(bytes);
}

cudaError_t set_pr_smem_limit(int precision, int bytes)
{
    const cudaError_t e =
        precision == CG_FP64 ? set_smem_t<double>(bytes) : set_smem_t<float>(bytes);
    if (e) return e;
    const cudaError_t e3 = set_pr3_smem_limit(precision, bytes);
    return e3 ? e3 : set_pr_pair_smem_limit(precision, bytes);
}

cudaError_t launch_pr_persistent(int precision, const DevReplica *d_reps, const int *d_index,
                                 int n_ctas, int threads, int smem_bytes, const RunArgs &args,
                                 cudaStream_t st, int L, int dim)
{
    // the square lattice's update needs L/2 columns, the cubic one's L
    if (threads < L / 2 || (dim == 3 && threads < L)) return cudaErrorInvalidValue;
    if (dim == 3)
        return launch_pr_persistent3(precision, d_reps, d_index, n_ctas, threads, smem_bytes,
                                     args, st, L);
    if (args.pair)
        return launch_pr_persistent_pair(precision, d_reps, d_index, n_ctas, threads, smem_bytes,
                                         args, st, L);
    if (precision == CG_FP64) {
        switch (threads) {
        case 1024: return launch_t<double, 1024>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 512: return launch_t<double, 512>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 384: return launch_t<double, 384>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 256: return launch_t<double, 256>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        }
    } else {
        switch (threads) {
        case 1024: return launch_t<float, 1024>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 512: return launch_t<float, 512>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 384: return launch_t<float, 384>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        case 256: return launch_t<float, 256>(d_reps, d_index, n_ctas, smem_bytes, args, st, L);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace cg
