// Calibration kernels of qmc_probe_rates (include/qmc_probe.h): loops of one arithmetic operation
// (inline PTX on values that change every iteration, so that nothing can be folded, hoisted or
// dropped) and a loop of the sweep's FP32 partner arithmetic alone.  The host times each launch
// with CUDA events.
#include "qmc_launch.h"

namespace qmc {

constexpr int PROBE_CHAINS = 8;  // independent dependency chains per thread
constexpr int PROBE_UNROLL = 4;  // steps of every chain per loop iteration

__device__ __forceinline__ void op_ffma(float &a, float b, float c)
{
    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a) : "f"(b), "f"(c));
}
__device__ __forceinline__ void op_ffma2(unsigned long long &a, unsigned long long b, unsigned long long c)
{
    asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a) : "l"(b), "l"(c));
}
__device__ __forceinline__ void op_fmin(float &a, float b) { asm volatile("min.f32 %0, %0, %1;" : "+f"(a) : "f"(b)); }
__device__ __forceinline__ void op_rsqrt(float &a) { asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a)); }
__device__ __forceinline__ void op_dfma(double &a, double b, double c)
{
    asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a) : "d"(b), "d"(c));
}

__device__ __forceinline__ unsigned long long pack2(float x, float y)
{
    return (unsigned long long)__float_as_uint(x) | ((unsigned long long)__float_as_uint(y) << 32);
}

// KIND: 0 FFMA, 1 FFMA2, 2 FMNMX, 3 RSQRT, 4 DFMA (QMC_PROBE_* of qmc_probe.h)
template <int KIND> __global__ void __launch_bounds__(1024) op_probe_kernel(int iters, float *sink)
{
    const float s = 1.0f + 1e-3f * (float)(threadIdx.x & 7);
    float f[PROBE_CHAINS];
    unsigned long long p[PROBE_CHAINS];
    double g[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) {
        f[k] = s + 0.01f * k;
        p[k] = pack2(f[k], f[k] + 0.5f);
        g[k] = (double)f[k];
    }
    const float b = 0.999f, c = 1e-3f;
    const unsigned long long b2 = pack2(b, b), c2 = pack2(c, c);
    for (int it = 0; it < iters; ++it) {
        // the min probe's other operand changes every iteration (min with a constant would be
        // idempotent and could be folded)
        const float v = __int_as_float(0x3f800000 + (it & 0xfff));
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) {
                if (KIND == 0) op_ffma(f[k], b, c);
                if (KIND == 1) op_ffma2(p[k], b2, c2);
                if (KIND == 2) op_fmin(f[k], (u & 1) ? v : s);
                if (KIND == 3) op_rsqrt(f[k]);
                if (KIND == 4) op_dfma(g[k], 0.999, 1e-3);
            }
    }
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) r += f[k] + __uint_as_float((unsigned)p[k]) + (float)g[k];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// The partner arithmetic of the FP32 sweep (Packed5::acc5, exponent 5, symmetrised u) for two
// moves at once, old and new position, over PROBE_PAIR_CHUNKS x 4 partners in shared memory:
// 16 pair evaluations per chunk, four chunks per thread per iteration, no reduction or barrier.
constexpr int PROBE_PAIR_CHUNKS_PER_THREAD = 4;
__global__ void __launch_bounds__(512) pair_probe_kernel(int iters, float *sink)
{
    extern __shared__ __align__(16) float4 part[];  // x | y | z chunks
    const int nv = PROBE_PAIR_CHUNKS_PER_THREAD * blockDim.x;
    const float L = 44.697f;
    for (int c = threadIdx.x; c < nv; c += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            const unsigned h = (unsigned)(c * 4 + k) * 2654435761u;
            const float v0 = L * (float)(h >> 8) * 0x1p-24f, v1 = L * (float)((h * 7u) >> 8) * 0x1p-24f;
            const float v2 = L * (float)((h * 13u) >> 8) * 0x1p-24f, v3 = L * (float)((h * 29u) >> 8) * 0x1p-24f;
            part[k * nv + c] = make_float4(v0, v1, v2, v3);
        }
    Jas<float, 5, true> J;
    J.c = -0.5f * 3.07f * 3.07f * 3.07f * 3.07f * 3.07f;
    J.L = L;
    J.hL2 = 0.25f * L * L;
    J.K = 0.f;
    J.m = 5.f;
    Packed5 P;
    P.init(J);
    const float a0 = 0.37f * L + 1e-3f * (threadIdx.x & 31), a1 = 0.61f * L;
    float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
        // the moved positions (all three coordinates) and the partners a thread reads change with
        // the iteration, so no part of the loop body is invariant; as in the sweep, each move packs
        // its old and new position in one f32x2 and every partner is duplicated into both lanes
        const float e = 1e-3f * (float)(it & 15);
        const float2 px0 = make_float2(a0 + e, a0 + 0.5f), px1 = make_float2(a1 - e, a1 - 0.4f);
        const float2 py0 = make_float2(0.5f * L + e, 0.5f * L - e), py1 = make_float2(0.3f * L - e, 0.3f * L + e);
        const float2 pz0 = make_float2(0.25f * L - e, 0.25f * L), pz1 = make_float2(0.75f * L, 0.75f * L + e);
        const int rot = it % nv;
        for (int c0 = threadIdx.x; c0 < nv; c0 += blockDim.x) {
            const int c = c0 + rot < nv ? c0 + rot : c0 + rot - nv;
            const float4 X = part[c], Y = part[nv + c], Z = part[2 * nv + c];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float xe = Vec<float>::get(X, k), ye = Vec<float>::get(Y, k), ze = Vec<float>::get(Z, k);
                const float2 xj = make_float2(xe, xe), yj = make_float2(ye, ye), zj = make_float2(ze, ze);
                P.acc5(__ffma2_rn(px0, P.m1, xj), __ffma2_rn(py0, P.m1, yj), __ffma2_rn(pz0, P.m1, zj), acc0);
                P.acc5(__ffma2_rn(px1, P.m1, xj), __ffma2_rn(py1, P.m1, yj), __ffma2_rn(pz1, P.m1, zj), acc1);
            }
        }
    }
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc0.x + acc0.y + acc1.x + acc1.y;
}

size_t probe_smem(int kind, int threads);

// lane operations (pair probe: pair evaluations) one thread performs per loop iteration
double probe_ops_per_thread_iter(int kind)
{
    if (kind == QMC_PROBE_PAIR) return 16.0 * PROBE_PAIR_CHUNKS_PER_THREAD;
    const double per = (double)PROBE_CHAINS * PROBE_UNROLL;
    return kind == QMC_PROBE_FFMA2 ? 2.0 * per : per;
}

cudaError_t probe_occupancy(int kind, int threads, int *blocks)
{
    const size_t smem = probe_smem(kind, threads);
    switch (kind) {
    case QMC_PROBE_FFMA: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, op_probe_kernel<0>, threads, 0);
    case QMC_PROBE_FFMA2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, op_probe_kernel<1>, threads, 0);
    case QMC_PROBE_FMNMX: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, op_probe_kernel<2>, threads, 0);
    case QMC_PROBE_RSQRT: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, op_probe_kernel<3>, threads, 0);
    case QMC_PROBE_DFMA: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, op_probe_kernel<4>, threads, 0);
    case QMC_PROBE_PAIR: {
        cudaError_t e = cudaFuncSetAttribute(pair_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pair_probe_kernel, threads, smem);
    }
    default: return cudaErrorInvalidValue;
    }
}

size_t probe_smem(int kind, int threads)
{
    return kind == QMC_PROBE_PAIR ? (size_t)3 * PROBE_PAIR_CHUNKS_PER_THREAD * threads * sizeof(float4) : 0;
}

cudaError_t launch_probe(int kind, int grid, int threads, int iters, float *sink, cudaStream_t st)
{
    const size_t smem = probe_smem(kind, threads);
    switch (kind) {
    case QMC_PROBE_FFMA: op_probe_kernel<0><<<grid, threads, 0, st>>>(iters, sink); break;
    case QMC_PROBE_FFMA2: op_probe_kernel<1><<<grid, threads, 0, st>>>(iters, sink); break;
    case QMC_PROBE_FMNMX: op_probe_kernel<2><<<grid, threads, 0, st>>>(iters, sink); break;
    case QMC_PROBE_RSQRT: op_probe_kernel<3><<<grid, threads, 0, st>>>(iters, sink); break;
    case QMC_PROBE_DFMA: op_probe_kernel<4><<<grid, threads, 0, st>>>(iters, sink); break;
    case QMC_PROBE_PAIR: {
        cudaError_t e = cudaFuncSetAttribute(pair_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        if (e != cudaSuccess) return e;
        pair_probe_kernel<<<grid, threads, smem, st>>>(iters, sink);
        break;
    }
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace qmc
