// Mixed group-size sweep kernels (uneven batches with dominant walkers): float, exponent 5,
// symmetrised u, whole CTAs of MIXED_TPWB threads for the dominant walkers.
#include "qmc_launch.h"

namespace qmc {

template <int TPWS> static cudaError_t prepare_mixed()
{
    auto k = sweep_mixed_kernel<float, 5, true, MIXED_TPWB, TPWS>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        if (e != cudaSuccess) return e;
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        attr = true;
    }
    return cudaSuccess;
}

template <int TPWS>
static cudaError_t go_mixed(int grid, size_t smem, cudaStream_t st, const SweepArgs &a, const SweepArgs &big,
                            unsigned *big_next)
{
    cudaError_t e = prepare_mixed<TPWS>();
    if (e != cudaSuccess) return e;
    sweep_mixed_kernel<float, 5, true, MIXED_TPWB, TPWS><<<grid, MIXED_TPWB, smem, st>>>(a, big, big_next);
    return cudaGetLastError();
}

template <int TPWS> static cudaError_t occ_mixed(size_t smem, int *ctas)
{
    cudaError_t e = prepare_mixed<TPWS>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, sweep_mixed_kernel<float, 5, true, MIXED_TPWB, TPWS>,
                                                         MIXED_TPWB, smem);
}

cudaError_t launch_sweep_mixed(int tpw_small, int grid, size_t smem, cudaStream_t st, const SweepArgs &a,
                               const SweepArgs &big, unsigned *big_next)
{
    switch (tpw_small) {
    case 64: return go_mixed<64>(grid, smem, st, a, big, big_next);
    case 128: return go_mixed<128>(grid, smem, st, a, big, big_next);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_sweep_mixed(int tpw_small, size_t smem, int *ctas)
{
    switch (tpw_small) {
    case 64: return occ_mixed<64>(smem, ctas);
    case 128: return occ_mixed<128>(smem, ctas);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qmc
