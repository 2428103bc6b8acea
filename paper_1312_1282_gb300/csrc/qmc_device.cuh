// qmc_device.cuh -- device building blocks of libqmc: the counter-based random numbers, the
// Jastrow pair function, the Aziz II potential, the minimum-image distance and the per-walker
// thread-group primitives (reduction, barrier).  Everything here runs on the GPU; the
// host-side API is in qmc_api.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qmc.h"

namespace qmc {

// ----------------------------------------------------------------------------------------------
// Walker table entry (built on the host from qmc_walker_desc, resolved and validated).
// ----------------------------------------------------------------------------------------------
struct DevWalker {
    int32_t n;     // atoms
    int32_t pad;   // SoA block stride (elements), multiple of 4
    int64_t off;   // element offset of the x block
    uint32_t wid;  // walker id in the Philox counter
    int32_t slot;  // index of this walker's logpsi / sweep / accum entries
    double L;      // box side
    double b, m;   // Jastrow parameters
    double step;   // trial step
    double c;      // f prefactor -b^m / 2  (Eq. fifthPower)
    double K;      // 2 f(L/2): the shift of the symmetrised u (Eq. uFunction)
};

constexpr unsigned FULL = 0xffffffffu;

// ----------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round multiplies counter
// words 0 and 2 by fixed odd constants, splits the 64-bit products into hi/lo halves and xors the
// hi halves with the other counter words and the round key; the key advances by two Weyl
// constants between rounds.
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed)
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

enum : uint32_t { ST_STEP = 0, ST_INDEX = 1, ST_SHUFFLE = 2, ST_JITTER = 3, ST_DICE = 4 };

__device__ __forceinline__ uint32_t word(const uint4 &v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// integer in [0, n): floor(x n / 2^32)
__device__ __forceinline__ uint32_t index_of(uint32_t x, uint32_t n) { return __umulhi(x, n); }

// Uniform numbers from 32-bit words.  Double: (x + 1/2) 2^-32 and 2u - 1, both exact.
// Float: the top 24 bits, (x' + 1/2) 2^-24 and 2u - 1, both exact.
template <typename T> struct Rng;
template <> struct Rng<double> {
    static __device__ __forceinline__ double unif(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }
    static __device__ __forceinline__ double sunif(uint32_t x)
    {
        return (double)(2LL * (long long)x + 1LL - 4294967296LL) * 0x1p-32;
    }
};
template <> struct Rng<float> {
    static __device__ __forceinline__ float unif(uint32_t x) { return ((float)(x >> 8) + 0.5f) * 0x1p-24f; }
    static __device__ __forceinline__ float sunif(uint32_t x)
    {
        return (float)(2 * (int)(x >> 8) + 1 - 16777216) * 0x1p-24f;
    }
};

// ----------------------------------------------------------------------------------------------
// Fast single-precision special functions: the PTX approximate instructions (SFU).
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ float rsqrt_a(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_a(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_a(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_a(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename T> struct Fn;
template <> struct Fn<float> {
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrt_a(x); }
    static __device__ __forceinline__ float rcp(float x) { return rcp_a(x); }
    static __device__ __forceinline__ float exp(float x) { return ex2_a(x * 1.4426950408889634f); }
    static __device__ __forceinline__ float exp2(float x) { return ex2_a(x); }
    static __device__ __forceinline__ float log(float x) { return lg2_a(x) * 0.6931471805599453f; }
    // x^(-m) for x > 0
    static __device__ __forceinline__ float powneg(float x, float m) { return ex2_a(-m * lg2_a(x)); }
    static __device__ __forceinline__ float rint(float x) { return rintf(x); }
};
template <> struct Fn<double> {
    static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / sqrt(x); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
    static __device__ __forceinline__ double exp2(double x) { return ::exp2(x); }
    static __device__ __forceinline__ double log(double x) { return ::log(x); }
    static __device__ __forceinline__ double powneg(double x, double m) { return ::pow(x, -m); }
    static __device__ __forceinline__ double rint(double x) { return ::rint(x); }
};

// ----------------------------------------------------------------------------------------------
// Jastrow exponent u(r) of Eqs. (uFunction) and (fifthPower): f(r) = c r^-m with c = -b^m/2;
// symmetrised u(r) = f(r) + f(L-r) - 2 f(L/2) for r < L/2 (SYM), else u(r) = f(r); u = 0 for
// r >= L/2.  MEXP = 5 evaluates the powers by multiplication; MEXP = 0 takes m at run time.
//
// u(r2) with SYM clamps r^2 at (L/2)^2 instead of branching: the clamped value gives
// u(L/2) = 0 analytically, and two clamped pairs give bit-identical values, so far partners
// cancel exactly in the old/new difference of a move.  Padding entries (far coordinates, whose
// r^2 is infinite or above the clamp) and the NaN that marks the moved atom clamp the same way.
// ----------------------------------------------------------------------------------------------
template <typename T, int MEXP, bool SYM> struct Jas {
    T c, K, L, hL2, m;

    __device__ __forceinline__ void init(const DevWalker &d)
    {
        c = (T)d.c;
        K = (T)d.K;
        L = (T)d.L;
        hL2 = (T)(0.25 * d.L * d.L);
        m = (T)d.m;
    }

    // c r^-m from q = 1/r (MEXP = 5) or from r (general m)
    __device__ __forceinline__ T fq(T q, T r) const
    {
        if (MEXP == 5) {
            const T q2 = q * q;
            return c * (q2 * q2 * q);
        } else {
            return c * Fn<T>::powneg(r, m);
        }
    }

    __device__ __forceinline__ T u(T r2) const
    {
        if (SYM) {
            const T rc = fmin(r2, hL2);
            const T q = Fn<T>::rsqrt(rc);
            const T r = rc * q;
            const T w = L - r;
            const T iw = Fn<T>::rcp(w);
            if (MEXP == 5) {
                const T q2 = q * q, w2 = iw * iw;
                const T q5 = q2 * q2 * q, w5 = w2 * w2 * iw;
                return fma(c, q5, fma(c, w5, -K));
            } else {
                return fq(q, r) + fq(iw, w) - K;
            }
        } else {
            const T q = Fn<T>::rsqrt(r2);
            const T v = fq(q, r2 * q);
            return r2 < hL2 ? v : (T)0;
        }
    }

    // q = 1/r, u' and u'' at r^2 (meaningful for 0 < r < L/2; the caller masks the rest)
    __device__ __forceinline__ void d12(T r2, T &q, T &u1, T &u2) const
    {
        q = Fn<T>::rsqrt(r2);
        const T r = r2 * q;
        T f0;
        if (MEXP == 5) {
            const T q2 = q * q;
            f0 = c * (q2 * q2 * q);
        } else {
            f0 = c * Fn<T>::powneg(r, m);
        }
        u1 = -m * f0 * q;                    // f'(r)  = -m f / r
        u2 = m * (m + (T)1) * f0 * (q * q);  // f''(r) = m(m+1) f / r^2
        if (SYM) {
            const T w = L - r;
            const T iw = Fn<T>::rcp(w);
            T g0;
            if (MEXP == 5) {
                const T w2 = iw * iw;
                g0 = c * (w2 * w2 * iw);
            } else {
                g0 = c * Fn<T>::powneg(w, m);
            }
            u1 += m * g0 * iw;                   // d/dr f(L-r) = -f'(L-r) = +m f(L-r)/(L-r)
            u2 += m * (m + (T)1) * g0 * (iw * iw);
        }
    }
};

// ----------------------------------------------------------------------------------------------
// HFD-B(HE) (Aziz II) pair potential (published 1987 constants)
// ----------------------------------------------------------------------------------------------
// Aziz II (HFD-B(HE)) potential in K, r in Angstrom (the paper's Sec. 7 potential), with the
// constants folded in double and rounded once: with x = r/rm, q = 1/r and A = q^6,
//   eps C_2k / x^2k = A q^(2k-6) (eps C_2k rm^2k)      (k = 3, 4, 5)
//   eps A* exp(-alpha x + beta x^2) = 2^(e0 + ea r + eb r^2),  e0 = log2(eps A*),
// and the damping F(x) = exp(-(D/x - 1)^2) for x < D, i.e. r < D rm, where D/x = D rm q.
// A* = 1.8443101e5 enters only through e0.
template <typename T> struct Aziz {
    T k6, k8, k10, e0, ea, eb, Drm;
    __device__ __forceinline__ Aziz()
    {
        const double eps = 10.948, rm = 2.963, alpha = 10.43329537, beta = -2.27965105,
                     C6 = 1.36745214, C8 = 0.42123807, C10 = 0.17473318, D = 1.4826, log2e = 1.4426950408889634;
        const double rm2 = rm * rm, rm6 = rm2 * rm2 * rm2;
        k6 = (T)(eps * C6 * rm6);
        k8 = (T)(eps * C8 * rm6 * rm2);
        k10 = (T)(eps * C10 * rm6 * rm2 * rm2);
        e0 = (T)20.94531715824703;  // log2(eps As) = log2(2.01914469e6), a literal so it stays an immediate
        ea = (T)(-alpha * log2e / rm);
        eb = (T)(beta * log2e / rm2);
        Drm = (T)(D * rm);
    }
    // V from r, r^2, q = 1/r, q^2 and A = q^6
    __device__ __forceinline__ T operator()(T r, T r2, T q, T q2, T A) const
    {
        const T disp = A * fma(fma(k10, q2, k8), q2, k6);
        const T rep = Fn<T>::exp2(fma(eb, r2, fma(ea, r, e0)));
        const T t = fma(Drm, q, (T)-1);
        const T F = r < Drm ? Fn<T>::exp(-(t * t)) : (T)1;
        return fma(-F, disp, rep);
    }
    __device__ __forceinline__ T operator()(T r, T r2, T q) const
    {
        const T q2 = q * q;
        return (*this)(r, r2, q, q2, q2 * q2 * q2);
    }
};

// ----------------------------------------------------------------------------------------------
// Periodic cube
// ----------------------------------------------------------------------------------------------
// |d| folded to the nearest image, for |d| <= L
template <typename T> __device__ __forceinline__ T mi_abs(T d, T L)
{
    const T a = fabs(d);
    return fmin(a, L - a);
}
// signed nearest-image difference; the rounding to an integer uses the add/subtract of
// 1.5 * 2^(mantissa bits), which stays on the FMA pipe (valid for |d / L| < 2^22)
template <typename T> __device__ __forceinline__ T round_magic(T x);
template <> __device__ __forceinline__ float round_magic<float>(float x)
{
    return __fadd_rn(__fadd_rn(x, 12582912.0f), -12582912.0f);
}
template <> __device__ __forceinline__ double round_magic<double>(double x)
{
    return __dadd_rn(__dadd_rn(x, 6755399441055744.0), -6755399441055744.0);
}
template <typename T> __device__ __forceinline__ T mi_signed(T d, T L, T iL)
{
    return fma(-L, round_magic<T>(d * iL), d);
}
// a coordinate displaced by less than one box length, put back into [0, L]
template <typename T> __device__ __forceinline__ T wrap(T x, T L)
{
    return x < (T)0 ? x + L : (x >= L ? x - L : x);
}

// ----------------------------------------------------------------------------------------------
// Per-walker thread group: TPW consecutive threads of a CTA (TPW a multiple of 32).
// bar_id = 1 + group index; groups of one warp synchronise with __syncwarp.
// ----------------------------------------------------------------------------------------------
template <int TPW> __device__ __forceinline__ void group_sync(int bar_id)
{
    if (TPW == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(TPW) : "memory");
    }
}

template <typename T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Sum over the group, identical (bit for bit) in every thread: a butterfly within each warp
// (IEEE addition commutes, so all lanes get the same tree), then every thread adds the per-warp
// values in the same order.  red holds 2 * (TPW/32) slots; `ph` alternates them so that one
// barrier per call suffices.
template <int TPW, typename T> __device__ __forceinline__ T group_sum(T v, T *red, int &ph, int bar_id, int gtid)
{
    v = warp_sum(v);
    if (TPW == 32) return v;
    constexpr int NW = TPW / 32;
    if ((gtid & 31) == 0) red[ph * NW + (gtid >> 5)] = v;
    group_sync<TPW>(bar_id);
    T s;
    if constexpr (sizeof(T) == 4 && NW % 4 == 0) {
        const float4 *r4 = reinterpret_cast<const float4 *>(red + ph * NW);
        float4 a = r4[0];
        s = ((a.x + a.y) + a.z) + a.w;
#pragma unroll
        for (int w = 1; w < NW / 4; ++w) {
            a = r4[w];
            s = (((s + a.x) + a.y) + a.z) + a.w;
        }
    } else {
        s = red[ph * NW];
#pragma unroll
        for (int w = 1; w < NW; ++w) s += red[ph * NW + w];
    }
    ph ^= 1;
    return s;
}

}  // namespace qmc
