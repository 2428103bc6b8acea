// Stand-alone passes (local energy, ln psi, trial ratios, (b, m) gradient) and the start
// configuration kernel, both precisions.
#include "qmc_launch.h"

namespace qmc {

template <typename K> static cudaError_t big_smem(K k)
{
    static_assert(sizeof(K) > 0, "");
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess) cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

template <typename T, int MEXP, bool SYM>
static cudaError_t pass_go(int kind, int grid, size_t smem, cudaStream_t st, const PassArgs &a)
{
    if (kind == 0 || kind == 1) {
        auto k = pass_kernel<T, MEXP, SYM, PASS_TPW>;
        static bool attr = false;
        if (!attr) {
            cudaError_t e = big_smem(k);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        k<<<grid, PASS_TPW, smem, st>>>(a, kind);
    } else if (kind == 2) {
        auto k = trial_kernel<T, MEXP, SYM, TRIAL_TPW>;
        static bool attr = false;
        if (!attr) {
            cudaError_t e = big_smem(k);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        k<<<grid, TRIAL_TPW, smem, st>>>(a);
    } else {
        auto k = grad_kernel<T, SYM, PASS_TPW>;
        static bool attr = false;
        if (!attr) {
            cudaError_t e = big_smem(k);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        k<<<grid, PASS_TPW, smem, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t pass_t(Variant v, int kind, int grid, size_t smem, cudaStream_t st, const PassArgs &a)
{
    switch (v) {
    case V5S: return pass_go<T, 5, true>(kind, grid, smem, st, a);
    case VGS: return pass_go<T, 0, true>(kind, grid, smem, st, a);
    default: return pass_go<T, 0, false>(kind, grid, smem, st, a);
    }
}

cudaError_t launch_pass(int precision, Variant v, int kind, int grid, size_t smem, cudaStream_t st, const PassArgs &a)
{
    return precision == QMC_FP64 ? pass_t<double>(v, kind, grid, smem, st, a)
                                 : pass_t<float>(v, kind, grid, smem, st, a);
}

cudaError_t launch_hist(int precision, int grid, size_t smem, cudaStream_t st, const PassArgs &a, int nbins,
                        double rmax, unsigned long long *hist)
{
    if (precision == QMC_FP64) {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = big_smem(hist_kernel<double, PASS_TPW>);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        hist_kernel<double, PASS_TPW><<<grid, PASS_TPW, smem, st>>>(a, nbins, rmax, hist);
    } else {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = big_smem(hist_kernel<float, PASS_TPW>);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        hist_kernel<float, PASS_TPW><<<grid, PASS_TPW, smem, st>>>(a, nbins, rmax, hist);
    }
    return cudaGetLastError();
}

cudaError_t launch_init(int precision, int grid, size_t smem, cudaStream_t st, const DevWalker *walkers,
                        unsigned long long seed, double sigma, void *pos)
{
    if (precision == QMC_FP64) {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = big_smem(init_kernel<double>);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        init_kernel<double><<<grid, 256, smem, st>>>(walkers, seed, sigma, pos);
    } else {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = big_smem(init_kernel<float>);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        init_kernel<float><<<grid, 256, smem, st>>>(walkers, seed, sigma, pos);
    }
    return cudaGetLastError();
}

// fills the FIFO with the walkers in processing order and clears the chunk counters
__global__ void queue_init_kernel(const int *order, int W, uint2 *slots, int *prog, unsigned *head, unsigned *tail)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < W) {
        slots[i] = make_uint2((unsigned)i + 1u, (unsigned)order[i]);
        prog[order[i]] = 0;
    }
    if (i == 0) {
        *head = 0u;
        *tail = (unsigned)W;
    }
}

cudaError_t launch_queue_init(const int *order, int W, uint2 *slots, int *prog, unsigned *head, unsigned *tail,
                              cudaStream_t st)
{
    queue_init_kernel<<<(W + 255) / 256, 256, 0, st>>>(order, W, slots, prog, head, tail);
    return cudaGetLastError();
}

}  // namespace qmc
