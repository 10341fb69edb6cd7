// cg_pr_cluster.cu -- launches of the cluster form of the persistent
// parallel-rejection kernel (cg_pr_cluster.cuh), single-electron hops.
#include "cg_pr_cluster.cuh"

namespace cg {

template <typename Real, int kThreads, bool kPow2, int kDim>
static cudaError_t launch_cluster_d(const DevReplica *d_reps, const int *d_index, int n_reps,
                                    int cluster, int smem_bytes, const RunArgs &args,
                                    cudaStream_t st)
{
    auto kern = pr_cluster<Real, kThreads, kPow2, kDim>;
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
static cudaError_t launch_cluster_t(const DevReplica *d_reps, const int *d_index, int n_reps,
                                    int cluster, int smem_bytes, const RunArgs &args,
                                    cudaStream_t st, int dim)
{
    return dim == 3 ? launch_cluster_d<Real, kThreads, kPow2, 3>(d_reps, d_index, n_reps, cluster,
                                                                 smem_bytes, args, st)
                    : launch_cluster_d<Real, kThreads, kPow2, 2>(d_reps, d_index, n_reps, cluster,
                                                                 smem_bytes, args, st);
}

template <typename Real>
static cudaError_t launch_cluster_p(const DevReplica *d_reps, const int *d_index, int n_reps,
                                    int cluster, int threads, int smem_bytes,
                                    const RunArgs &args, cudaStream_t st, bool pow2, int dim)
{
    if (threads == 1024)
        return pow2 ? launch_cluster_t<Real, 1024, true>(d_reps, d_index, n_reps, cluster,
                                                         smem_bytes, args, st, dim)
                    : launch_cluster_t<Real, 1024, false>(d_reps, d_index, n_reps, cluster,
                                                          smem_bytes, args, st, dim);
    if (threads == 512)
        return pow2 ? launch_cluster_t<Real, 512, true>(d_reps, d_index, n_reps, cluster,
                                                        smem_bytes, args, st, dim)
                    : launch_cluster_t<Real, 512, false>(d_reps, d_index, n_reps, cluster,
                                                         smem_bytes, args, st, dim);
    return cudaErrorInvalidValue;
}

cudaError_t launch_pr_cluster(int precision, const DevReplica *d_reps, const int *d_index,
                              int n_reps, int cluster, int threads, int smem_bytes,
                              const RunArgs &args, cudaStream_t st, int L, int dim)
{
    // square lattice: L/(2C) base rows and their partners per CTA; cubic
    // lattice: L/C z-planes per CTA
    if (cluster < 2 || cluster > 8 || (L % (dim == 3 ? cluster : 2 * cluster)) != 0 ||
        threads < L)
        return cudaErrorInvalidValue;
    if (args.pair)
        return launch_pr_cluster_pair(precision, d_reps, d_index, n_reps, cluster, threads,
                                      smem_bytes, args, st, L, dim);
    const bool pow2 = (L & (L - 1)) == 0;
    return precision == CG_FP64
               ? launch_cluster_p<double>(d_reps, d_index, n_reps, cluster, threads, smem_bytes,
                                          args, st, pow2, dim)
               : launch_cluster_p<float>(d_reps, d_index, n_reps, cluster, threads, smem_bytes,
                                         args, st, pow2, dim);
}

}  // namespace cg
