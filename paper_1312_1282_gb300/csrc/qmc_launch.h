// qmc_launch.h -- internal interface between the host API (qmc_api.cu) and the kernel
// translation units (qmc_k_*.cu), which instantiate the templates of qmc_kernels.cuh.
#pragma once

#include <cuda_runtime.h>

#include "qmc_kernels.cuh"
#include "qmc_probe.h"

namespace qmc {

// Jastrow variants compiled: 5 = exponent 5 by multiplication, symmetrised u;
// GS = general exponent, symmetrised; GN = general exponent, plain truncated u.
enum Variant { V5S = 0, VGS = 1, VGN = 2 };

// Each launcher returns the launch error (cudaSuccess if enqueued).
cudaError_t launch_sweep_f32_small(int tpw, Variant v, int grid, int block, size_t smem, cudaStream_t st,
                                   const SweepArgs &a);  // tpw 32, 64, 128
cudaError_t launch_sweep_f32_big(int tpw, Variant v, int grid, int block, size_t smem, cudaStream_t st,
                                 const SweepArgs &a);  // tpw 256, 512, 1024
cudaError_t launch_sweep_f64_small(int tpw, Variant v, int grid, int block, size_t smem, cudaStream_t st,
                                   const SweepArgs &a);
cudaError_t launch_sweep_f64_big(int tpw, Variant v, int grid, int block, size_t smem, cudaStream_t st,
                                 const SweepArgs &a);

// resident CTAs per SM of a sweep kernel instantiation with this block and shared memory
cudaError_t occupancy_sweep_f32_small(int tpw, Variant v, int block, size_t smem, int *ctas);
cudaError_t occupancy_sweep_f32_big(int tpw, Variant v, int block, size_t smem, int *ctas);
cudaError_t occupancy_sweep_f64_small(int tpw, Variant v, int block, size_t smem, int *ctas);
cudaError_t occupancy_sweep_f64_big(int tpw, Variant v, int block, size_t smem, int *ctas);
// uneven batches with dominant walkers: FP32, exponent 5, symmetrised u; dominant walkers on whole
// CTAs of MIXED_TPWB threads, the others on groups of tpw_small (64 or 128) threads
constexpr int MIXED_TPWB = 256;
cudaError_t launch_sweep_mixed(int tpw_small, int grid, size_t smem, cudaStream_t st, const SweepArgs &a,
                               const SweepArgs &big, unsigned *big_next);
cudaError_t occupancy_sweep_mixed(int tpw_small, size_t smem, int *ctas);
cudaError_t launch_queue_init(const int *order, int W, uint2 *slots, int *prog, unsigned *head, unsigned *tail,
                              cudaStream_t st);

constexpr int PASS_TPW = 256;   // threads per walker of the stand-alone passes
constexpr int TRIAL_TPW = 128;  // threads per walker of qmc_trial_delta

// kind 0: local energy, 1: ln psi, 2: trial deltas, 3: energy + (b, m) gradient
cudaError_t launch_pass(int precision, Variant v, int kind, int grid, size_t smem, cudaStream_t st,
                        const PassArgs &a);
cudaError_t launch_hist(int precision, int grid, size_t smem, cudaStream_t st, const PassArgs &a, int nbins,
                        double rmax, unsigned long long *hist);
cudaError_t launch_init(int precision, int grid, size_t smem, cudaStream_t st, const DevWalker *walkers,
                        unsigned long long seed, double sigma, void *pos);

// calibration probes (qmc_probe_rates): launcher, resident CTAs per SM, work per thread and loop
// iteration (lane operations, or pair evaluations for the pair probe)
cudaError_t launch_probe(int kind, int grid, int threads, int iters, float *sink, cudaStream_t st);
cudaError_t probe_occupancy(int kind, int threads, int *blocks);
double probe_ops_per_thread_iter(int kind);

}  // namespace qmc
