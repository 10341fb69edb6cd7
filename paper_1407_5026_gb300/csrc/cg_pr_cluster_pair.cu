// cg_pr_cluster_pair.cu -- launches of the cluster form of the persistent
// parallel-rejection kernel (cg_pr_cluster.cuh) with two-electron hops on the
// square and the cubic lattice.
#include "cg_pr_cluster.cuh"

namespace cg {

template <typename Real, int kThreads, bool kPow2, int kDim>
static cudaError_t launch_cluster_pair_d(const DevReplica *d_reps, const int *d_index,
                                         int n_reps, int cluster, int smem_bytes,
                                         const RunArgs &args, cudaStream_t st)
{
    auto kern = pr_cluster<Real, kThreads, kPow2, kDim, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
    if (e) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_reps * cluster), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, d_reps, d_index, args);
}

template <typename Real, int kThreads, bool kPow2>
static cudaError_t launch_cluster_pair_t(const DevReplica *d_reps, const int *d_index,
                                         int n_reps, int cluster, int smem_bytes,
                                         const RunArgs &args, cudaStream_t st, int dim)
{
    return dim == 3 ? launch_cluster_pair_d<Real, kThreads, kPow2, 3>(d_reps, d_index, n_reps,
                                                                      cluster, smem_bytes, args, st)
                    : launch_cluster_pair_d<Real, kThreads, kPow2, 2>(d_reps, d_index, n_reps,
                                                                      cluster, smem_bytes, args, st);
}

cudaError_t launch_pr_cluster_pair(int precision, const DevReplica *d_reps, const int *d_index,
                                   int n_reps, int cluster, int threads, int smem_bytes,
                                   const RunArgs &args, cudaStream_t st, int L, int dim)
{
    const bool pow2 = (L & (L - 1)) == 0;
    if (precision == CG_FP64) {
        if (threads == 1024)
            return pow2 ? launch_cluster_pair_t<double, 1024, true>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st, dim)
                        : launch_cluster_pair_t<double, 1024, false>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st, dim);
        if (threads == 512)
            return pow2 ? launch_cluster_pair_t<double, 512, true>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st, dim)
                        : launch_cluster_pair_t<double, 512, false>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st, dim);
    } else {
        if (threads == 1024)
            return pow2 ? launch_cluster_pair_t<float, 1024, true>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st, dim)
                        : launch_cluster_pair_t<float, 1024, false>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st, dim);
        if (threads == 512)
            return pow2 ? launch_cluster_pair_t<float, 512, true>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st, dim)
                        : launch_cluster_pair_t<float, 512, false>(d_reps, d_index, n_reps, cluster, smem_bytes, args, st, dim);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cg
