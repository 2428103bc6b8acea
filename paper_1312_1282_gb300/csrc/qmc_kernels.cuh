// qmc_kernels.cuh -- the kernels of libqmc, as templates instantiated by the qmc_k_*.cu files.
//
// Layout in shared memory: each walker's coordinates stay resident for a whole call as three
// blocks x[pad] | y[pad] | z[pad] of T (structure of arrays, as in HBM), read as 16-byte vectors
// (float4 / double2).  Entries n .. pad-1 hold NaN, which the clamped pair function turns into an
// exact zero contribution, so the partner loops need no bound checks.
//
// Work split: a CTA holds G walkers, each served by a group of TPW threads (TPW a multiple of
// 32).  For one move every thread of the group evaluates the old and new pair terms of its
// partner chunks j = 4c..4c+3, c = gtid, gtid + TPW, ...; the group sums them (warp butterfly,
// then one named barrier), and every thread takes the same accept/reject decision.  The owner of
// the moved atom's chunk writes its new coordinates; all other threads keep a register copy of
// the last accepted move, so a move needs exactly one group barrier (none for TPW = 32).
#pragma once

#include "qmc_device.cuh"

namespace qmc {

template <typename T> struct Vec;
template <> struct Vec<float> {
    using type = float4;
    static constexpr int N = 4;
    static __device__ __forceinline__ float get(const float4 &v, int e)
    {
        return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
    }
    static __device__ __forceinline__ void set(float4 &v, int e, float a)
    {
        v.x = e == 0 ? a : v.x;
        v.y = e == 1 ? a : v.y;
        v.z = e == 2 ? a : v.z;
        v.w = e == 3 ? a : v.w;
    }
};
template <> struct Vec<double> {
    using type = double2;
    static constexpr int N = 2;
    static __device__ __forceinline__ double get(const double2 &v, int e) { return e == 0 ? v.x : v.y; }
    static __device__ __forceinline__ void set(double2 &v, int e, double a)
    {
        v.x = e == 0 ? a : v.x;
        v.y = e == 1 ? a : v.y;
    }
};

template <typename T> __device__ __forceinline__ T qnan();
template <> __device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }

struct SweepArgs {
    const DevWalker *walkers;  // [W] table
    const int *order;          // [W] processing order (longest walkers first)
    int W;
    int G;                     // walkers per CTA
    int stride;                // shared-memory block stride (elements) = largest pad in the batch
    void *pos;
    double *logpsi;
    unsigned long long *sweep;
    double *accum;
    unsigned long long seed;
    int nsweeps, energy_every, recompute_every;
    int proposal, sequential;
    double h2m;
    unsigned *err;
};

// shared-memory bytes of one group: positions + reduction slots (T and double, 2 phases each)
template <typename T> __host__ __device__ constexpr size_t group_smem(int stride, int tpw)
{
    return (size_t)3 * stride * sizeof(T) + (size_t)2 * (tpw / 32) * (sizeof(T) + sizeof(double)) * 2;
}

// ----------------------------------------------------------------------------------------------
// Load / store one walker
// ----------------------------------------------------------------------------------------------
// Copy walker coordinates to shared memory (NaN past n).  Returns false (in every thread of the
// group) if a coordinate is non-finite or outside [0, L].
template <typename T, int TPW>
__device__ bool load_walker(const T *gx, int n, int pad, T L, T *sx, T *sy, T *sz, T *red, int &ph, int bar_id,
                            int gtid)
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    const int nv = pad / VN;
    int bad = 0;
    for (int c = gtid; c < nv; c += TPW) {
        V v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            v[k] = reinterpret_cast<const V *>(gx + (size_t)k * pad)[c];
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const int j = c * VN + e;
                const T a = Vec<T>::get(v[k], e);
                if (j < n) {
                    bad |= !(a >= (T)0 && a <= L);  // false for NaN
                } else {
                    Vec<T>::set(v[k], e, qnan<T>());
                }
            }
        }
        reinterpret_cast<V *>(sx)[c] = v[0];
        reinterpret_cast<V *>(sy)[c] = v[1];
        reinterpret_cast<V *>(sz)[c] = v[2];
    }
    const T nbad = group_sum<TPW>((T)bad, red, ph, bar_id, gtid);
    group_sync<TPW>(bar_id);
    return nbad == (T)0;
}

template <typename T, int TPW>
__device__ void store_walker(T *gx, int n, int pad, const T *sx, const T *sy, const T *sz, int gtid)
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    const int nfull = n / VN;
    for (int c = gtid; c < nfull; c += TPW) {
        reinterpret_cast<V *>(gx)[c] = reinterpret_cast<const V *>(sx)[c];
        reinterpret_cast<V *>(gx + pad)[c] = reinterpret_cast<const V *>(sy)[c];
        reinterpret_cast<V *>(gx + 2 * (size_t)pad)[c] = reinterpret_cast<const V *>(sz)[c];
    }
    for (int j = nfull * VN + gtid; j < n; j += TPW) {
        gx[j] = sx[j];
        gx[pad + j] = sy[j];
        gx[2 * (size_t)pad + j] = sz[j];
    }
}

// ----------------------------------------------------------------------------------------------
// Eq. (JastrowUpdate): this thread's share of sum_{j != s} [u(|r' - r_j|) - u(|r_s - r_j|)]
// ----------------------------------------------------------------------------------------------
template <typename T, int MEXP, bool SYM, int TPW>
__device__ __forceinline__ T partner_delta(const Jas<T, MEXP, SYM> &J, const T *sx, const T *sy, const T *sz,
                                           int nv, int s, T xs, T ys, T zs, T xn, T yn, T zn, int gtid)
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    const int cs = s / VN;
    const T L = J.L;
    T acc = (T)0;
#pragma unroll 2
    for (int c = gtid; c < nv; c += TPW) {
        V X = reinterpret_cast<const V *>(sx)[c];
        V Y = reinterpret_cast<const V *>(sy)[c];
        V Z = reinterpret_cast<const V *>(sz)[c];
        if (c == cs) {  // the moved atom is not its own partner
            const int e = s - cs * VN;
            Vec<T>::set(X, e, qnan<T>());
            Vec<T>::set(Y, e, qnan<T>());
            Vec<T>::set(Z, e, qnan<T>());
        }
#pragma unroll
        for (int e = 0; e < VN; ++e) {
            const T xj = Vec<T>::get(X, e), yj = Vec<T>::get(Y, e), zj = Vec<T>::get(Z, e);
            const T ax = mi_abs(xs - xj, L), ay = mi_abs(ys - yj, L), az = mi_abs(zs - zj, L);
            const T bx = mi_abs(xn - xj, L), by = mi_abs(yn - yj, L), bz = mi_abs(zn - zj, L);
            const T ro = fma(ax, ax, fma(ay, ay, az * az));
            const T rn = fma(bx, bx, fma(by, by, bz * bz));
            acc += J.u(rn) - J.u(ro);
        }
    }
    return acc;
}

// ----------------------------------------------------------------------------------------------
// Group-wide O(N^2) passes over the resident configuration
// ----------------------------------------------------------------------------------------------
// ln psi = sum_{i<j} u(r_ij) (Eq. Jastrow): full rows, halved.  FP32 row sums, double totals.
template <typename T, int MEXP, bool SYM, int TPW>
__device__ double group_log_psi(const Jas<T, MEXP, SYM> &J, const T *sx, const T *sy, const T *sz, int n, int nv,
                                double *redD, int &phD, int bar_id, int gtid)
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    const T L = J.L, hL2 = J.hL2;
    double tot = 0.0;
    for (int i = gtid; i < n; i += TPW) {
        const T xi = sx[i], yi = sy[i], zi = sz[i];
        T row = (T)0;
        for (int c = 0; c < nv; ++c) {
            const V X = reinterpret_cast<const V *>(sx)[c];
            const V Y = reinterpret_cast<const V *>(sy)[c];
            const V Z = reinterpret_cast<const V *>(sz)[c];
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const T ax = mi_abs(xi - Vec<T>::get(X, e), L), ay = mi_abs(yi - Vec<T>::get(Y, e), L),
                        az = mi_abs(zi - Vec<T>::get(Z, e), L);
                const T r2 = fma(ax, ax, fma(ay, ay, az * az));
                const T uu = J.u(r2);
                row += (r2 < hL2 && c * VN + e != i) ? uu : (T)0;
            }
        }
        tot += (double)row;
    }
    return 0.5 * group_sum<TPW>(tot, redD, phD, bar_id, gtid);
}

// Local energy pieces (Sec. 2 Hamiltonian): sums over i of V_i (full rows), lap_i and |F_i|^2.
// out = {V, T_L, T_PB, T_F, E_L}, valid in every thread of the group.
template <typename T, int MEXP, bool SYM, int TPW>
__device__ void group_energy(const Jas<T, MEXP, SYM> &J, const T *sx, const T *sy, const T *sz, int n, int nv,
                             double h2m, double *redD, int &phD, int bar_id, int gtid, double out[5])
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    const T L = J.L, iL = (T)1 / J.L, hL2 = J.hL2;
    double sV = 0.0, sLap = 0.0, sF2 = 0.0;
    for (int i = gtid; i < n; i += TPW) {
        const T xi = sx[i], yi = sy[i], zi = sz[i];
        T v = 0, lap = 0, fx = 0, fy = 0, fz = 0;
        for (int c = 0; c < nv; ++c) {
            const V X = reinterpret_cast<const V *>(sx)[c];
            const V Y = reinterpret_cast<const V *>(sy)[c];
            const V Z = reinterpret_cast<const V *>(sz)[c];
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const T dx = mi_signed(xi - Vec<T>::get(X, e), L, iL);
                const T dy = mi_signed(yi - Vec<T>::get(Y, e), L, iL);
                const T dz = mi_signed(zi - Vec<T>::get(Z, e), L, iL);
                const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                const bool ok = (r2 < hL2) && (c * VN + e != i);
                T q, u1, u2;
                J.d12(r2, q, u1, u2);
                const T vv = aziz(r2 * q, q);
                const T g = u1 * q;
                v += ok ? vv : (T)0;
                lap += ok ? fma((T)2 * u1, q, u2) : (T)0;
                fx += ok ? g * dx : (T)0;
                fy += ok ? g * dy : (T)0;
                fz += ok ? g * dz : (T)0;
            }
        }
        sV += (double)v;
        sLap += (double)lap;
        sF2 += (double)fx * fx + (double)fy * fy + (double)fz * fz;
    }
    sV = group_sum<TPW>(sV, redD, phD, bar_id, gtid);
    sLap = group_sum<TPW>(sLap, redD, phD, bar_id, gtid);
    sF2 = group_sum<TPW>(sF2, redD, phD, bar_id, gtid);
    const double k = 0.5 * h2m;
    out[0] = 0.5 * sV;
    out[1] = -k * (sLap + sF2);
    out[2] = -0.5 * k * sLap;
    out[3] = k * sF2;
    out[4] = out[0] + out[1];
}

// ----------------------------------------------------------------------------------------------
// The sweep: one group runs one walker's chain for a whole call.
// ----------------------------------------------------------------------------------------------
template <typename T, int MEXP, bool SYM, int TPW>
__device__ void run_walker(const SweepArgs &a, const DevWalker &d, T *sx, T *sy, T *sz, T *redT, double *redD,
                           int gtid, int bar_id)
{
    constexpr int VN = Vec<T>::N;
    const int n = d.n, pad = d.pad, nv = (n + VN - 1) / VN;
    const int slot = d.slot;
    const T L = (T)d.L, step = (T)d.step;
    int phT = 0, phD = 0;
    T *gx = reinterpret_cast<T *>(a.pos) + d.off;

    if (!load_walker<T, TPW>(gx, n, pad, L, sx, sy, sz, redT, phT, bar_id, gtid)) {
        if (gtid == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_POS);
        return;
    }
    Jas<T, MEXP, SYM> J;
    J.init(d);

    double lp = a.logpsi[slot];
    const unsigned long long k0 = a.sweep[slot];
    double *A = a.accum + 8 * (size_t)slot;
    int nacc = 0;
    int last_s = -1;
    T lx = 0, ly = 0, lz = 0;
    const int lane = gtid & 31;
    const uint32_t wid = d.wid;

    for (int it = 0; it < a.nsweeps; ++it) {
        const unsigned long long kk = k0 + (unsigned long long)it;
        const uint32_t k = (uint32_t)kk;
        for (int t0 = 0; t0 < n; t0 += 32) {
            // random numbers of moves t0 .. t0+31, one move per lane (Sec. 5.2: 5 numbers per move)
            const uint32_t t = (uint32_t)(t0 + lane);
            const uint4 rw = philox(t, k, wid, ST_STEP, a.seed);
            int my_s;
            if (a.sequential) {
                my_s = (int)t;
            } else {
                const uint4 ri = philox(((uint32_t)t0 >> 2) + (uint32_t)(lane >> 2), k, wid, ST_INDEX, a.seed);
                my_s = (int)index_of(word(ri, lane & 3), (uint32_t)n);
            }
            T mdx, mdy, mdz, mxi;
            if (a.proposal == QMC_CUBE) {
                mdx = step * Rng<T>::sunif(rw.x);
                mdy = step * Rng<T>::sunif(rw.y);
                mdz = step * Rng<T>::sunif(rw.z);
                mxi = Rng<T>::unif(rw.w);
            } else {
                const T two_pi = (T)6.283185307179586;
                const T r0 = sqrt((T)-2 * log(Rng<T>::unif(rw.x)));
                const T r1 = sqrt((T)-2 * log(Rng<T>::unif(rw.z)));
                mdx = step * (r0 * cos(two_pi * Rng<T>::unif(rw.y)));
                mdy = step * (r0 * sin(two_pi * Rng<T>::unif(rw.y)));
                mdz = step * (r1 * cos(two_pi * Rng<T>::unif(rw.w)));
                const uint4 rd = philox(((uint32_t)t0 >> 2) + (uint32_t)(lane >> 2), k, wid, ST_DICE, a.seed);
                mxi = Rng<T>::unif(word(rd, lane & 3));
            }
            const int cnt = min(32, n - t0);
            for (int tt = 0; tt < cnt; ++tt) {
                const int s = __shfl_sync(FULL, my_s, tt);
                const T dx = __shfl_sync(FULL, mdx, tt);
                const T dy = __shfl_sync(FULL, mdy, tt);
                const T dz = __shfl_sync(FULL, mdz, tt);
                const T xi = __shfl_sync(FULL, mxi, tt);
                T xs = sx[s], ys = sy[s], zs = sz[s];
                if (s == last_s) {
                    xs = lx;
                    ys = ly;
                    zs = lz;
                }
                const T xn = wrap(xs + dx, L), yn = wrap(ys + dy, L), zn = wrap(zs + dz, L);
                const T part = partner_delta<T, MEXP, SYM, TPW>(J, sx, sy, sz, nv, s, xs, ys, zs, xn, yn, zn, gtid);
                const T delta = group_sum<TPW>(part, redT, phT, bar_id, gtid);
                if (delta != delta) {  // identical in every thread of the group
                    if (gtid == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_RATIO);
                    return;
                }
                // Eq. (Decision): accept iff |psi'|^2 / |psi|^2 = exp(2 Delta) > xi
                if (exp((T)2 * delta) > xi) {
                    if (gtid == (s / VN) % TPW) {
                        sx[s] = xn;
                        sy[s] = yn;
                        sz[s] = zn;
                    }
                    last_s = s;
                    lx = xn;
                    ly = yn;
                    lz = zn;
                    lp += (double)delta;
                    ++nacc;
                } else {
                    last_s = -1;
                }
                if (TPW == 32) __syncwarp();
            }
        }
        group_sync<TPW>(bar_id);
        last_s = -1;
        if (a.recompute_every > 0 && (kk + 1) % (unsigned long long)a.recompute_every == 0)
            lp = group_log_psi<T, MEXP, SYM, TPW>(J, sx, sy, sz, n, nv, redD, phD, bar_id, gtid);
        if (a.energy_every > 0 && (kk + 1) % (unsigned long long)a.energy_every == 0) {
            double e[5];
            group_energy<T, MEXP, SYM, TPW>(J, sx, sy, sz, n, nv, a.h2m, redD, phD, bar_id, gtid, e);
            // added sample by sample, so a run split over several calls sums in the same order
            if (gtid == 0) {
                A[0] += e[4];
                A[1] += e[4] * e[4];
                A[2] += e[0];
                A[3] += e[1];
                A[4] += e[2];
                A[5] += e[3];
                A[6] += 1.0;
            }
        }
    }
    group_sync<TPW>(bar_id);
    store_walker<T, TPW>(gx, n, pad, sx, sy, sz, gtid);
    if (gtid == 0) {
        A[7] += (double)nacc;  // integer-valued: exact in any order
        a.logpsi[slot] = lp;
        a.sweep[slot] = k0 + (unsigned long long)a.nsweeps;
    }
}

// CTAs hold up to 256 threads (TPW <= 256) or exactly one group; at least 1024 resident threads
// per SM, i.e. at most 64 registers per thread.
template <int TPW> constexpr int cta_bound() { return TPW > 256 ? TPW : 256; }

template <typename T, int MEXP, bool SYM, int TPW>
__global__ void __launch_bounds__(cta_bound<TPW>(), 1024 / cta_bound<TPW>()) sweep_kernel(SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = threadIdx.x / TPW, gtid = threadIdx.x % TPW;
    const int item = blockIdx.x * a.G + g;
    if (item >= a.W) return;  // only group barriers follow, so whole groups may leave
    constexpr int NW = TPW / 32;
    unsigned char *base = smem + (size_t)g * group_smem<T>(a.stride, TPW);
    T *sx = reinterpret_cast<T *>(base);
    T *sy = sx + a.stride;
    T *sz = sy + a.stride;
    double *redD = reinterpret_cast<double *>(sz + a.stride);
    T *redT = reinterpret_cast<T *>(redD + 2 * NW);
    const DevWalker d = a.walkers[a.order[item]];
    run_walker<T, MEXP, SYM, TPW>(a, d, sx, sy, sz, redT, redD, gtid, 1 + g);
}

// ----------------------------------------------------------------------------------------------
// Stand-alone passes: one CTA (TPW threads) per walker
// ----------------------------------------------------------------------------------------------
struct PassArgs {
    const DevWalker *walkers;
    int W;
    int stride;
    const void *pos;
    double *out;
    double h2m;
    // qmc_trial_delta
    const int32_t *s;
    const double *delta;
    int M;
    unsigned *err;
};

template <typename T, int TPW>
__device__ __forceinline__ void pass_smem(unsigned char *smem, int stride, T *&sx, T *&sy, T *&sz, T *&redT,
                                          double *&redD)
{
    constexpr int NW = TPW / 32;
    sx = reinterpret_cast<T *>(smem);
    sy = sx + stride;
    sz = sy + stride;
    redD = reinterpret_cast<double *>(sz + stride);
    redT = reinterpret_cast<T *>(redD + 2 * NW);
}

// kind: 0 = local energy (5 outputs), 1 = ln psi (1 output)
template <typename T, int MEXP, bool SYM, int TPW>
__global__ void __launch_bounds__(TPW) pass_kernel(PassArgs a, int kind)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *sx, *sy, *sz, *redT;
    double *redD;
    pass_smem<T, TPW>(smem, a.stride, sx, sy, sz, redT, redD);
    const DevWalker d = a.walkers[blockIdx.x];
    const int gtid = threadIdx.x;
    int phT = 0, phD = 0;
    constexpr int VN = Vec<T>::N;
    const T *gx = reinterpret_cast<const T *>(a.pos) + d.off;
    if (!load_walker<T, TPW>(gx, d.n, d.pad, (T)d.L, sx, sy, sz, redT, phT, 1, gtid)) {
        if (gtid == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_POS);
        return;
    }
    Jas<T, MEXP, SYM> J;
    J.init(d);
    const int nv = (d.n + VN - 1) / VN;
    if (kind == 0) {
        double e[5];
        group_energy<T, MEXP, SYM, TPW>(J, sx, sy, sz, d.n, nv, a.h2m, redD, phD, 1, gtid, e);
        if (gtid == 0)
            for (int q = 0; q < 5; ++q) a.out[5 * (size_t)d.slot + q] = e[q];
    } else {
        const double lp = group_log_psi<T, MEXP, SYM, TPW>(J, sx, sy, sz, d.n, nv, redD, phD, 1, gtid);
        if (gtid == 0) a.out[d.slot] = lp;
    }
}

// Eq. (JastrowUpdate) for M given trial moves from the unchanged configuration.
template <typename T, int MEXP, bool SYM, int TPW>
__global__ void __launch_bounds__(TPW) trial_kernel(PassArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *sx, *sy, *sz, *redT;
    double *redD;
    pass_smem<T, TPW>(smem, a.stride, sx, sy, sz, redT, redD);
    const DevWalker d = a.walkers[blockIdx.x];
    const int gtid = threadIdx.x;
    int phT = 0;
    constexpr int VN = Vec<T>::N;
    const T *gx = reinterpret_cast<const T *>(a.pos) + d.off;
    const T L = (T)d.L;
    if (!load_walker<T, TPW>(gx, d.n, d.pad, L, sx, sy, sz, redT, phT, 1, gtid)) {
        if (gtid == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_POS);
        return;
    }
    Jas<T, MEXP, SYM> J;
    J.init(d);
    const int nv = (d.n + VN - 1) / VN;
    for (int q = 0; q < a.M; ++q) {
        const size_t mi = (size_t)d.slot * a.M + q;
        const int s = a.s[mi];
        if (s < 0 || s >= d.n) {  // uniform across the group: skip the move, flag it
            if (gtid == 0) {
                a.out[mi] = qnan<double>();
                atomicOr(a.err, QMC_DEVERR_BAD_INDEX);
            }
            continue;
        }
        const T xs = sx[s], ys = sy[s], zs = sz[s];
        const T xn = wrap(xs + (T)a.delta[3 * mi], L), yn = wrap(ys + (T)a.delta[3 * mi + 1], L),
                zn = wrap(zs + (T)a.delta[3 * mi + 2], L);
        const T part = partner_delta<T, MEXP, SYM, TPW>(J, sx, sy, sz, nv, s, xs, ys, zs, xn, yn, zn, gtid);
        const T delta = group_sum<TPW>(part, redT, phT, 1, gtid);
        if (gtid == 0) a.out[mi] = (double)delta;
    }
}

// ----------------------------------------------------------------------------------------------
// ln psi, E_L and their (b, m) derivatives.  u depends on b only through c = -b^m/2, so
// d/db of ln psi, u', u'' is (dc/db)/c = m/b times the quantity; the m-derivatives use
// d f/dm = f ln(b/r) (and the matching forms for f', f'').
// ----------------------------------------------------------------------------------------------
template <typename T, bool SYM, int TPW>
__global__ void __launch_bounds__(TPW) grad_kernel(PassArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *sx, *sy, *sz, *redT;
    double *redD;
    pass_smem<T, TPW>(smem, a.stride, sx, sy, sz, redT, redD);
    const DevWalker d = a.walkers[blockIdx.x];
    const int gtid = threadIdx.x;
    int phT = 0, phD = 0;
    constexpr int VN = Vec<T>::N;
    using V = typename Vec<T>::type;
    const T *gx = reinterpret_cast<const T *>(a.pos) + d.off;
    const T L = (T)d.L, iL = (T)1 / L, hL2 = (T)(0.25 * d.L * d.L);
    if (!load_walker<T, TPW>(gx, d.n, d.pad, L, sx, sy, sz, redT, phT, 1, gtid)) {
        if (gtid == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_POS);
        return;
    }
    const int n = d.n, nv = (n + VN - 1) / VN;
    const T c = (T)d.c, m = (T)d.m, lnb = (T)::log(d.b > 0 ? d.b : 1.0);
    const T K = (T)d.K;
    // m-derivative of the shift 2 f(L/2): 2 f(L/2) ln(2b/L)
    const T Km = (T)(d.K * ::log(d.b > 0 ? 2.0 * d.b / d.L : 1.0));
    const T c1 = (T)1 / m, c2 = (T)(2.0 * d.m + 1.0) / (m * (m + (T)1));
    double sLp = 0, sLpm = 0, sV = 0, sLap = 0, sLapm = 0, sF2 = 0, sFFm = 0;
    for (int i = gtid; i < n; i += TPW) {
        const T xi = sx[i], yi = sy[i], zi = sz[i];
        T lp = 0, lpm = 0, v = 0, lap = 0, lapm = 0, fx = 0, fy = 0, fz = 0, gx_ = 0, gy_ = 0, gz_ = 0;
        for (int cc = 0; cc < nv; ++cc) {
            const V X = reinterpret_cast<const V *>(sx)[cc];
            const V Y = reinterpret_cast<const V *>(sy)[cc];
            const V Z = reinterpret_cast<const V *>(sz)[cc];
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const T dx = mi_signed(xi - Vec<T>::get(X, e), L, iL);
                const T dy = mi_signed(yi - Vec<T>::get(Y, e), L, iL);
                const T dz = mi_signed(zi - Vec<T>::get(Z, e), L, iL);
                const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                const bool ok = (r2 < hL2) && (cc * VN + e != i);
                const T q = Fn<T>::rsqrt(r2);
                const T r = r2 * q;
                const T lbr = lnb + Fn<T>::log(q);  // ln(b/r)
                const T f = c * Fn<T>::powneg(r, m);
                const T f1 = -m * f * q, f2 = m * (m + (T)1) * f * (q * q);
                T uu = f, u1 = f1, u2 = f2, um = f * lbr, u1m = f1 * (c1 + lbr), u2m = f2 * (c2 + lbr);
                if (SYM) {
                    const T w = L - r, iw = Fn<T>::rcp(w);
                    const T lbw = lnb + Fn<T>::log(iw);
                    const T g = c * Fn<T>::powneg(w, m);
                    const T g1 = -m * g * iw, g2 = m * (m + (T)1) * g * (iw * iw);
                    uu += g - K;
                    u1 -= g1;
                    u2 += g2;
                    um += g * lbw - Km;
                    u1m -= g1 * (c1 + lbw);
                    u2m += g2 * (c2 + lbw);
                }
                const T vv = aziz(r, q);
                lp += ok ? uu : (T)0;
                lpm += ok ? um : (T)0;
                v += ok ? vv : (T)0;
                lap += ok ? fma((T)2 * u1, q, u2) : (T)0;
                lapm += ok ? fma((T)2 * u1m, q, u2m) : (T)0;
                const T g0 = u1 * q, gm = u1m * q;
                fx += ok ? g0 * dx : (T)0;
                fy += ok ? g0 * dy : (T)0;
                fz += ok ? g0 * dz : (T)0;
                gx_ += ok ? gm * dx : (T)0;
                gy_ += ok ? gm * dy : (T)0;
                gz_ += ok ? gm * dz : (T)0;
            }
        }
        sLp += (double)lp;
        sLpm += (double)lpm;
        sV += (double)v;
        sLap += (double)lap;
        sLapm += (double)lapm;
        sF2 += (double)fx * fx + (double)fy * fy + (double)fz * fz;
        sFFm += (double)fx * gx_ + (double)fy * gy_ + (double)fz * gz_;
    }
    sLp = group_sum<TPW>(sLp, redD, phD, 1, gtid);
    sLpm = group_sum<TPW>(sLpm, redD, phD, 1, gtid);
    sV = group_sum<TPW>(sV, redD, phD, 1, gtid);
    sLap = group_sum<TPW>(sLap, redD, phD, 1, gtid);
    sLapm = group_sum<TPW>(sLapm, redD, phD, 1, gtid);
    sF2 = group_sum<TPW>(sF2, redD, phD, 1, gtid);
    sFFm = group_sum<TPW>(sFFm, redD, phD, 1, gtid);
    if (gtid == 0) {
        const double k = 0.5 * a.h2m;
        const double mb = d.b > 0 ? d.m / d.b : 0.0;  // (dc/db)/c
        double *o = a.out + 6 * (size_t)d.slot;
        o[0] = 0.5 * sLp;
        o[1] = 0.5 * sV - k * (sLap + sF2);
        o[2] = mb * 0.5 * sLp;
        o[3] = 0.5 * sLpm;
        o[4] = -k * mb * (sLap + 2.0 * sF2);
        o[5] = -k * (sLapm + 2.0 * sFFm);
    }
}

// ----------------------------------------------------------------------------------------------
// Start configurations: fcc sites chosen by a Philox Fisher-Yates shuffle, Gaussian jitter.
// One CTA per walker; the shuffle is sequential in thread 0 over a shared-memory permutation.
// ----------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) init_kernel(const DevWalker *walkers, unsigned long long seed, double sigma,
                                                   void *pos)
{
    extern __shared__ __align__(16) int perm[];
    const DevWalker d = walkers[blockIdx.x];
    const int n = d.n;
    int nc = 1;
    while (4LL * nc * nc * nc < n) ++nc;
    const int M = 4 * nc * nc * nc;
    for (int q = threadIdx.x; q < M; q += blockDim.x) perm[q] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) {
            const uint4 w = philox((uint32_t)i >> 2, 0u, d.wid, ST_SHUFFLE, seed);
            const int j = i + (int)index_of(word(w, i & 3), (uint32_t)(M - i));
            const int tmp = perm[i];
            perm[i] = perm[j];
            perm[j] = tmp;
        }
    }
    __syncthreads();
    const double L = d.L, a = L / nc;
    const double two_pi = 6.283185307179586;
    T *gx = reinterpret_cast<T *>(pos) + d.off;
    for (int i = threadIdx.x; i < d.pad; i += blockDim.x) {
        if (i >= n) {
            gx[i] = (T)0;
            gx[d.pad + i] = (T)0;
            gx[2 * (size_t)d.pad + i] = (T)0;
            continue;
        }
        const int q = perm[i];
        const int basis = q & 3, cell = q >> 2;
        const int iz = cell % nc, iy = (cell / nc) % nc, ix = cell / (nc * nc);
        const uint4 w = philox((uint32_t)i, 0u, d.wid, ST_JITTER, seed);
        const double r0 = sqrt(-2.0 * log(Rng<double>::unif(w.x)));
        const double r1 = sqrt(-2.0 * log(Rng<double>::unif(w.z)));
        const double gxx = r0 * cos(two_pi * Rng<double>::unif(w.y));
        const double gyy = r0 * sin(two_pi * Rng<double>::unif(w.y));
        const double gzz = r1 * cos(two_pi * Rng<double>::unif(w.w));
        const double bx = (basis == 1 || basis == 2) ? 0.5 : 0.0;
        const double by = (basis == 1 || basis == 3) ? 0.5 : 0.0;
        const double bz = (basis == 2 || basis == 3) ? 0.5 : 0.0;
        // no contraction: the site and the jitter are rounded separately, then added
        const double px = __dadd_rn(__dmul_rn((double)ix + bx, a), __dmul_rn(sigma, gxx));
        const double py = __dadd_rn(__dmul_rn((double)iy + by, a), __dmul_rn(sigma, gyy));
        const double pz = __dadd_rn(__dmul_rn((double)iz + bz, a), __dmul_rn(sigma, gzz));
        gx[i] = (T)wrap(px, L);
        gx[d.pad + i] = (T)wrap(py, L);
        gx[2 * (size_t)d.pad + i] = (T)wrap(pz, L);
    }
}

}  // namespace qmc
