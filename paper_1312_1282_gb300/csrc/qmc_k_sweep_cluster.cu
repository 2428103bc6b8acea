// Cluster sweep kernel (one walker over a thread-block cluster): launcher and capacity query.
#include "qmc_cluster.cuh"

namespace qmc {

static cudaError_t prepare_cluster()
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sweep_cluster_kernel<CLUSTER_TPW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return cudaSuccess;
}

static cudaLaunchConfig_t config(int grid, size_t smem, cudaStream_t st, cudaLaunchAttribute *attr, int C)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(CLUSTER_TPW, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t launch_sweep_cluster(int grid, size_t smem, cudaStream_t st, const ClusterArgs &a)
{
    cudaError_t e = prepare_cluster();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = config(grid, smem, st, attr, a.C);
    return cudaLaunchKernelEx(&cfg, sweep_cluster_kernel<CLUSTER_TPW>, a);
}

// clusters of C CTAs with this shared memory that can be resident at once (0: none)
cudaError_t cluster_capacity(int C, size_t smem, int *clusters)
{
    cudaError_t e = prepare_cluster();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = config(C, smem, nullptr, attr, C);
    return cudaOccupancyMaxActiveClusters(clusters, sweep_cluster_kernel<CLUSTER_TPW>, &cfg);
}

}  // namespace qmc
