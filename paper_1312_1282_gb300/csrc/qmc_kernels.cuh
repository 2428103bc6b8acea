// qmc_kernels.cuh -- the kernels of libqmc, as templates instantiated by the qmc_k_*.cu files.
//
// Layout in shared memory: each walker's coordinates stay resident for a whole call as three
// blocks x[pad] | y[pad] | z[pad] of T (structure of arrays, as in HBM), read as 16-byte vectors
// (float4 / double2).  Entries n .. stride-1 hold distinct far coordinates: their squared
// distances overflow to infinity (FP32) or exceed (L/2)^2, which the clamped pair function turns
// into an exact zero contribution and the energy passes mask, so the loops need no bound checks.
//
// Work split: a CTA holds G walkers, each served by a group of TPW threads (TPW a multiple of
// 32).  For one move every thread of the group evaluates the old and new pair terms of its
// partner chunks j = 4c..4c+3, c = gtid, gtid + TPW, ...; the group sums them (warp butterfly,
// then one named barrier), and every thread takes the same accept/reject decision.  The owner of
// the moved atom's chunk writes its new coordinates; all other threads keep a private copy of
// the last batch's accepted moves, so a batch of moves (two in FP32 for groups of 64 threads or
// more, one otherwise) needs exactly one group barrier (none for TPW = 32).
#pragma once

#include <cuda/atomic>
#include <type_traits>

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

// Running sum carried in two floats (Kahan compensation): keeps the ln psi and energy sums of the
// FP32 path off the FP64 pipe (1/64 of the FP32 rate on this part) inside the hot loops; the
// total goes to double once per chunk or pass.
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Sum of one row of pair terms (one atom against all partners) in the row-wise passes.  In FP32
// the partners go in blocks of ROW_BLOCK 4-atom chunks summed in float, and the block sums are
// added with compensation: a long row of tiny far-partner terms (u, u', u'' fall off as powers of
// 1/r) is not lost below the rounding of a large running sum.  In FP64 one block is the row.
template <typename T> struct RowSum;
template <> struct RowSum<float> {
    KahanF k;
    __device__ __forceinline__ void add(float x) { k.add(x); }
    __device__ __forceinline__ double value() const { return k.value(); }
};
template <> struct RowSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <typename T> constexpr int row_block() { return std::is_same<T, float>::value ? 16 : (1 << 30); }

// the ln psi carried along a chain: double in FP64 mode, compensated floats in FP32 mode
template <typename T> struct LogPsiAcc {
    double base;
    KahanF inc;
    __device__ __forceinline__ void add(T d)
    {
        if constexpr (std::is_same<T, float>::value)
            inc.add(d);
        else
            base += d;
    }
    __device__ __forceinline__ double value() const
    {
        if constexpr (std::is_same<T, float>::value)
            return base + inc.value();
        else
            return base;
    }
    __device__ __forceinline__ void set(double v)
    {
        base = v;
        inc = KahanF();
    }
};

struct SweepArgs {
    const DevWalker *walkers;  // [W] table
    const int *order;          // [W] processing order (longest walkers first)
    int W;
    int G;                     // walkers per CTA
    int stride;                // shared-memory block stride (elements): largest pad, rounded up to 32
    int tile;                  // local energy by the tiled pass: 1 drift arrays in smem, 2 in fscr
    float *fscr;               // tile 2: 3 x stride floats of drift per resident group (L2-resident)
    int gmem;                  // 1: walkers too large for shared memory stay in HBM (updated in place)
    void *pos;
    double *logpsi;
    unsigned long long *sweep;
    double *accum;
    unsigned long long seed;
    int nsweeps, energy_every, recompute_every;
    int proposal, sequential;
    double h2m;
    unsigned *err;
    // persistent mode: walkers circulate through a FIFO of ready walkers in chunks of moves
    int dynamic;             // 0: one walker per thread group for the whole call
    int chunk_moves;         // moves per chunk (a multiple of 32)
    unsigned q_total;        // chunks of all walkers: sum over w of ceil(nsweeps n_w / chunk_moves)
    unsigned *q_head, *q_tail;
    uint2 *q_slots;          // [W] {sequence, walker table index}
    int *q_prog;             // [W] chunks done (bit 30: walker faulted, its chunks are skipped)
    unsigned long long wait_ns;  // limit of every wait on the queue (global-timer nanoseconds)
    int drop_push;           // failure test only: the first walker of the order is never pushed back
                             // after its first chunk, so pops that wait for it run out (0 normally)
};

// Moves per batch of the FP32 sweep: the partner loop serves KB trial moves at once and the
// group reduces their KB sums with one barrier (see move_batch); the FP64 sweep (registers twice
// as wide) and groups of one warp (no barrier to save; measured slower with KB = 2 at N = 128)
// take one move at a time.  Measured on GB300 at N = 1952, 528 walkers,
// 128 threads per walker, 5 sweeps without / with one energy sample: KB = 1 18.7 / 21.6 ms,
// KB = 2 17.8 / 20.7 ms (the batch loop unrolled once; unrolled twice it spilled registers and
// took 22.3 ms with the energy), so KB = 2 is the default.
#ifndef QMC_KB
#define QMC_KB 2
#endif
constexpr int KB = QMC_KB;
template <typename T, int TPW> constexpr int kb_of() { return std::is_same<T, float>::value && TPW >= 64 ? KB : 1; }

// Shared memory of one group, in this order: positions x | y | z (stride elements of T each),
// reduction slots (2 phases of TPW/32 doubles, 2 phases of KB x TPW/32 T's), the cross terms of
// a batch (2 phases of KB x KB T's), a broadcast word, and with the tiled energy pass the drift
// components Fx | Fy | Fz (stride floats each).
struct GroupLayout {
    size_t red, redT, dsm, bc, F, bytes;
};
template <typename T> __host__ __device__ constexpr GroupLayout group_layout(int stride, int tpw, bool tile)
{
    GroupLayout g{};
    g.red = (size_t)3 * stride * sizeof(T);
    g.redT = g.red + (size_t)2 * (tpw / 32) * sizeof(double);
    g.dsm = g.redT + (size_t)2 * KB * (tpw / 32) * sizeof(T);
    g.bc = (g.dsm + (size_t)2 * KB * KB * sizeof(T) + 15) / 16 * 16;
    g.F = g.bc + 16;
    g.bytes = g.F + (tile ? (size_t)3 * stride * sizeof(float) : 0);
    return g;
}
template <typename T> __host__ __device__ constexpr size_t group_smem(int stride, int tpw, bool tile = false)
{
    return group_layout<T>(stride, tpw, tile).bytes;
}
__host__ __device__ constexpr int stride_of(int maxpad) { return (maxpad + 31) / 32 * 32; }

template <typename T> struct GroupMem {
    T *sx, *sy, *sz, *redT, *dsm;
    double *redD;
    float *fx, *fy, *fz;
    int *bc;  // one int broadcast from the group's thread 0
    __device__ __forceinline__ void bind(unsigned char *base, int stride, int tpw, bool tile)
    {
        const GroupLayout g = group_layout<T>(stride, tpw, tile);
        bc = reinterpret_cast<int *>(base + g.bc);
        sx = reinterpret_cast<T *>(base);
        sy = sx + stride;
        sz = sy + stride;
        redD = reinterpret_cast<double *>(base + g.red);
        redT = reinterpret_cast<T *>(base + g.redT);
        dsm = reinterpret_cast<T *>(base + g.dsm);
        fx = reinterpret_cast<float *>(base + g.F);
        fy = fx + stride;
        fz = fy + stride;
    }
    // drift arrays of the tiled energy pass in a group's own block of global scratch
    __device__ __forceinline__ void use_global_drift(float *f, int stride)
    {
        fx = f;
        fy = f + stride;
        fz = f + 2 * (size_t)stride;
    }
    // positions of a walker too large for shared memory: its own blocks in HBM, used in place
    __device__ __forceinline__ void use_global(T *gx, int pad)
    {
        sx = gx;
        sy = gx + pad;
        sz = gx + 2 * (size_t)pad;
    }
};

// Validation of a walker used in place (no copy): false in every thread of the group if a
// coordinate is non-finite or outside [0, L].
template <typename T, int TPW>
__device__ bool check_walker(const T *gx, int n, int pad, T L, T *red, int &ph, int bar_id, int gtid)
{
    int bad = 0;
    for (int j = gtid; j < n; j += TPW)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T a = gx[(size_t)k * pad + j];
            bad |= !(a >= (T)0 && a <= L);
        }
    const T nbad = group_sum<TPW>((T)bad, red, ph, bar_id, gtid);
    group_sync<TPW>(bar_id);
    return nbad == (T)0;
}

// ----------------------------------------------------------------------------------------------
// Load / store one walker
// ----------------------------------------------------------------------------------------------
// Copy walker coordinates to shared memory.  Entries n .. stride-1 get distinct far coordinates
// 1e30 (1 + j - n): any squared distance to them is infinite (FP32) or far above (L/2)^2, so the
// pair loops treat them as absent without index checks.  Returns false (in every thread of the
// group) if a coordinate is non-finite or outside [0, L].
template <typename T, int TPW>
__device__ bool load_walker(const T *gx, int n, int pad, int stride, T L, T *sx, T *sy, T *sz, T *red, int &ph,
                            int bar_id, int gtid)
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    const int nvp = pad / VN, nvs = stride / VN;
    int bad = 0;
    for (int c = gtid; c < nvs; c += TPW) {
        V v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (c < nvp) v[k] = reinterpret_cast<const V *>(gx + (size_t)k * pad)[c];
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const int j = c * VN + e;
                if (j < n) {
                    const T a = Vec<T>::get(v[k], e);
                    bad |= !(a >= (T)0 && a <= L);  // false for NaN
                } else {
                    Vec<T>::set(v[k], e, (T)1e30 * (T)(1 + j - n));
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
// Partner sums of Eq. (JastrowUpdate), FP32, exponent 5, symmetrised u: with q = 1/r and
// w = 1/(L - r), r clamped at L/2, u(r) = c (q^5 + w^5) - K (Eqs. uFunction, fifthPower), so
// sum_j [u(r'_j) - u(r_j)] = c (sum_j [q'^5 + w'^5] - sum_j [q^5 + w^5]).  Two partners per
// packed f32x2 instruction (FFMA2/FADD2/FMUL2 issue once for two lanes of work; min/max and the
// SFU stay scalar).
struct Packed5 {
    float2 L, hL2, m1;  // (L, L), ((L/2)^2, ...), (-1, -1)
    __device__ __forceinline__ void init(const Jas<float, 5, true> &J)
    {
        L = make_float2(J.L, J.L);
        hL2 = make_float2(J.hL2, J.hL2);
        m1 = make_float2(-1.f, -1.f);
    }
    // |d| folded to the nearest image: min(|d|, L - |d|), for two differences at once
    __device__ __forceinline__ float2 fold(float2 d) const
    {
        const float2 a = make_float2(fabsf(d.x), fabsf(d.y));
        const float2 b = __ffma2_rn(a, m1, L);
        return make_float2(fminf(a.x, b.x), fminf(a.y, b.y));
    }
    // acc += q^5 + w^5 of two partners, i.e. (u(r) + K) / c: the constant and the factor c are
    // applied once per partner sum, and the last power of each term is fused into the add
    __device__ __forceinline__ void acc5(float2 dx, float2 dy, float2 dz, float2 &acc) const
    {
        const float2 mx = fold(dx), my = fold(dy), mz = fold(dz);
        float2 r2 = __fmul2_rn(mx, mx);
        r2 = __ffma2_rn(my, my, r2);
        r2 = __ffma2_rn(mz, mz, r2);
        r2 = make_float2(fminf(r2.x, hL2.x), fminf(r2.y, hL2.y));
        const float2 q = make_float2(rsqrt_a(r2.x), rsqrt_a(r2.y));
        const float2 r = __fmul2_rn(r2, q);
        const float2 w = __ffma2_rn(r, m1, L);
        const float2 iw = make_float2(rcp_a(w.x), rcp_a(w.y));
        const float2 q2 = __fmul2_rn(q, q), w2 = __fmul2_rn(iw, iw);
        acc = __ffma2_rn(__fmul2_rn(q2, q2), q, acc);
        acc = __ffma2_rn(__fmul2_rn(w2, w2), iw, acc);
    }
};

// ----------------------------------------------------------------------------------------------
// Group-wide O(N^2) passes over the resident configuration
// ----------------------------------------------------------------------------------------------
// ln psi = sum_{i<j} u(r_ij) (Eq. Jastrow): full rows, halved.  FP32 row sums, double totals.
template <typename T, int MEXP, bool SYM, int TPW>
__device__ double group_log_psi(const Jas<T, MEXP, SYM> &J, const T *sx, const T *sy, const T *sz, int n, int nv,
                                double *redD, int &phD, int bar_id, int gtid, int part = 0, int parts = 1)
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    const T L = J.L, hL2 = J.hL2;
    double tot = 0.0;
    for (int i = part * TPW + gtid; i < n; i += parts * TPW) {  // this CTA's share of the rows
        const T xi = sx[i], yi = sy[i], zi = sz[i];
        RowSum<T> row;
        for (int c0 = 0; c0 < nv; c0 += row_block<T>()) {
            const int c1 = min(nv, c0 + row_block<T>());
            T blk = (T)0;
            for (int c = c0; c < c1; ++c) {
                const V X = reinterpret_cast<const V *>(sx)[c];
                const V Y = reinterpret_cast<const V *>(sy)[c];
                const V Z = reinterpret_cast<const V *>(sz)[c];
#pragma unroll
                for (int e = 0; e < VN; ++e) {
                    const T ax = mi_abs(xi - Vec<T>::get(X, e), L), ay = mi_abs(yi - Vec<T>::get(Y, e), L),
                            az = mi_abs(zi - Vec<T>::get(Z, e), L);
                    const T r2 = fma(ax, ax, fma(ay, ay, az * az));
                    const T uu = J.u(r2);
                    const int j = c * VN + e;
                    blk += (r2 < hL2 && j != i && j < n) ? uu : (T)0;
                }
            }
            row.add(blk);
        }
        tot += row.value();
    }
    return 0.5 * group_sum<TPW>(tot, redD, phD, bar_id, gtid);
}

// Local energy, tiled (FP32).  Each unordered pair is evaluated once.  Atoms form blocks of 32;
// a warp takes a tile of two blocks (a, b): lane l holds atom 32a + l, and at step t meets atom
// 32b + ((l + t) mod 32), so the 32 lanes see 32 distinct partners.  The drift of the row atom
// accumulates in a register; the opposite drift of the partner accumulates in a register that
// is passed to the neighbouring lane after every step, so that after 32 steps lane l holds the
// total for atom 32b + l.  Tiles are scheduled in the rounds of a round-robin tournament between
// blocks: in one round every block is in at most one tile, so the warps add their tile totals
// to the shared drift arrays without conflicts, in an order fixed by the schedule (the result
// is bit-reproducible).  Diagonal tiles (pairs inside one block) form a last round.
template <int MEXP, bool SYM> struct TilePair {
    const Jas<float, MEXP, SYM> &J;
    Aziz<float> AZ;
    float L, iL, hL2, m, mm1;
    __device__ __forceinline__ TilePair(const Jas<float, MEXP, SYM> &j)
        : J(j), L(j.L), iL(1.f / j.L), hL2(j.hL2), m(j.m), mm1(j.m * (j.m + 1.f))
    {
    }
    // drift contribution g (r_i - r_j) of the pair, its Laplacian term u'' + 2u'/r and V(r)
    __device__ __forceinline__ void operator()(float xi, float yi, float zi, float xj, float yj, float zj, bool take,
                                               float &gx, float &gy, float &gz, float &lap, float &v) const
    {
        const float dx = mi_signed(xi - xj, L, iL), dy = mi_signed(yi - yj, L, iL), dz = mi_signed(zi - zj, L, iL);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool ok = take && r2 < hL2;
        const float q = rsqrt_a(r2);
        const float r = r2 * q;
        const float f0 = J.fq(q, r);
        float u1 = -m * f0 * q, u2 = mm1 * f0 * (q * q);
        if (SYM) {
            const float w = L - r, iw = rcp_a(w);
            const float g0 = J.fq(iw, w);
            u1 += m * g0 * iw;
            u2 += mm1 * g0 * (iw * iw);
        }
        const float g = ok ? u1 * q : 0.f;
        gx = g * dx;
        gy = g * dy;
        gz = g * dz;
        lap = ok ? fmaf(2.f * u1, q, u2) : 0.f;
        // Aziz II; the damping exp(-(D/x - 1)^2) only matters for x < D: skipped when no lane needs it
        const float q2 = q * q, A6 = q2 * q2 * q2;
        const float disp = A6 * fmaf(fmaf(AZ.k10, q2, AZ.k8), q2, AZ.k6);
        const float rep = Fn<float>::exp2(fmaf(AZ.eb, r2, fmaf(AZ.ea, r, AZ.e0)));
        float F = 1.f;
        const bool damp = ok && r < AZ.Drm;
        if (__any_sync(FULL, damp)) {
            const float t = fmaf(AZ.Drm, q, -1.f);
            F = damp ? Fn<float>::exp(-(t * t)) : 1.f;
        }
        v = ok ? fmaf(-F, disp, rep) : 0.f;
    }
};

// Two tile steps at once (partners j0 and j1 of the same row atom), packed f32x2 arithmetic for
// exponent 5 and the symmetrised u; the general case evaluates the scalar form twice.
// In the packed form the Jastrow terms come out divided by constants that the caller applies
// once per walker: with A = q^6, B = w^6 (q = 1/r, w = 1/(L - r)), u'(r) = 5c (B - A) and
// u''(r) = 30c (A q + B w), so the drift g (r_i - r_j) is returned over GSCALE = 5c and the
// Laplacian term u'' + 2u'/r = 10c [q (B + 2A) + 3 B w] over LSCALE = 10c.  The Aziz II
// potential (the folded constants of Aziz) reuses the powers: its dispersion is
// F A (k6 + k8 q^2 + k10 q^4) and its repulsion 2^(e0 + ea r + eb r^2).
template <int MEXP, bool SYM> struct TilePair2 {
    static constexpr bool PACKED = MEXP == 5 && SYM;
    TilePair<MEXP, SYM> P;
    float GSCALE, LSCALE;
    float2 L2, iL2, nL2, M2, nM2, m1, two2, three2, k6, k8, k10, e0, ea, eb;
    __device__ __forceinline__ TilePair2(const Jas<float, MEXP, SYM> &j) : P(j)
    {
        GSCALE = PACKED ? 5.f * j.c : 1.f;
        LSCALE = PACKED ? 10.f * j.c : 1.f;
        L2 = make_float2(j.L, j.L);
        iL2 = make_float2(1.f / j.L, 1.f / j.L);
        nL2 = make_float2(-j.L, -j.L);
        M2 = make_float2(12582912.f, 12582912.f);
        nM2 = make_float2(-12582912.f, -12582912.f);
        m1 = make_float2(-1.f, -1.f);
        two2 = make_float2(2.f, 2.f);
        three2 = make_float2(3.f, 3.f);
        const Aziz<float> &az = P.AZ;  // the folded Aziz II constants, in both lanes
        k6 = make_float2(az.k6, az.k6);
        k8 = make_float2(az.k8, az.k8);
        k10 = make_float2(az.k10, az.k10);
        e0 = make_float2(az.e0, az.e0);
        ea = make_float2(az.ea, az.ea);
        eb = make_float2(az.eb, az.eb);
    }
    __device__ __forceinline__ float2 mi(float2 d) const
    {
        const float2 t = __fadd2_rn(__ffma2_rn(d, iL2, M2), nM2);  // round(d / L)
        return __ffma2_rn(nL2, t, d);
    }
    __device__ __forceinline__ void operator()(float xi, float yi, float zi, float2 xj, float2 yj, float2 zj,
                                               bool take0, bool take1, float2 &gx, float2 &gy, float2 &gz,
                                               float2 &lap, float2 &v) const
    {
        if constexpr (PACKED) {
            const float2 dx = mi(__ffma2_rn(xj, m1, make_float2(xi, xi)));
            const float2 dy = mi(__ffma2_rn(yj, m1, make_float2(yi, yi)));
            const float2 dz = mi(__ffma2_rn(zj, m1, make_float2(zi, zi)));
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            const bool ok0 = take0 && r2.x < P.hL2, ok1 = take1 && r2.y < P.hL2;
            const float2 q = make_float2(rsqrt_a(r2.x), rsqrt_a(r2.y));
            const float2 r = __fmul2_rn(r2, q);
            const float2 q2 = __fmul2_rn(q, q);
            const float2 q4 = __fmul2_rn(q2, q2);
            const float2 A = __fmul2_rn(q4, q2);
            const float2 w = __ffma2_rn(r, m1, L2);
            const float2 iw = make_float2(rcp_a(w.x), rcp_a(w.y));
            const float2 w2 = __fmul2_rn(iw, iw);
            const float2 B = __fmul2_rn(__fmul2_rn(w2, w2), w2);
            float2 g = __fmul2_rn(__ffma2_rn(A, m1, B), q);  // u'/r over 5c
            g = make_float2(ok0 ? g.x : 0.f, ok1 ? g.y : 0.f);
            gx = __fmul2_rn(g, dx);
            gy = __fmul2_rn(g, dy);
            gz = __fmul2_rn(g, dz);
            const float2 lp = __ffma2_rn(__ffma2_rn(A, two2, B), q, __fmul2_rn(B, __fmul2_rn(iw, three2)));
            lap = make_float2(ok0 ? lp.x : 0.f, ok1 ? lp.y : 0.f);
            // Aziz II; the damping factor F = exp(-(D/x - 1)^2) only where some lane has x < D
            const float2 disp = __fmul2_rn(A, __ffma2_rn(__ffma2_rn(k10, q2, k8), q2, k6));
            const float2 ex = __ffma2_rn(eb, r2, __ffma2_rn(ea, r, e0));
            const float2 rep = make_float2(ex2_a(ex.x), ex2_a(ex.y));
            float2 nF = m1;
            const float Drm = P.AZ.Drm;  // x < D is r < D rm
            const bool d0 = ok0 && r.x < Drm, d1 = ok1 && r.y < Drm;
            if (__any_sync(FULL, d0 || d1)) {
                const float t0 = fmaf(Drm, q.x, -1.f), t1 = fmaf(Drm, q.y, -1.f);
                nF.x = d0 ? -Fn<float>::exp(-(t0 * t0)) : -1.f;
                nF.y = d1 ? -Fn<float>::exp(-(t1 * t1)) : -1.f;
            }
            const float2 vv = __ffma2_rn(nF, disp, rep);
            v = make_float2(ok0 ? vv.x : 0.f, ok1 ? vv.y : 0.f);
        } else {
            P(xi, yi, zi, xj.x, yj.x, zj.x, take0, gx.x, gy.x, gz.x, lap.x, v.x);
            P(xi, yi, zi, xj.y, yj.y, zj.y, take1, gx.y, gy.y, gz.y, lap.y, v.y);
        }
    }
};

template <int MEXP, bool SYM, int TPW>
__device__ void group_energy_tiled(const Jas<float, MEXP, SYM> &J, const float *sx, const float *sy, const float *sz,
                                   float *Fx, float *Fy, float *Fz, int n, double h2m, double *redD, int &phD,
                                   int bar_id, int gtid, double out[5])
{
    constexpr int NW = TPW / 32;
    const int lane = gtid & 31, warp = gtid >> 5;
    const int NB = (n + 31) >> 5;
    const TilePair2<MEXP, SYM> P2(J);
    const float2 z2 = make_float2(0.f, 0.f);
    for (int i = gtid; i < NB * 32; i += TPW) {
        Fx[i] = 0.f;
        Fy[i] = 0.f;
        Fz[i] = 0.f;
    }
    group_sync<TPW>(bar_id);
    KahanF kV, kLap;
    const int NBp = NB + (NB & 1);  // an even number of teams: a dummy block when NB is odd
    for (int r = 0; r < NBp - 1; ++r) {
        for (int k = warp; k < NBp / 2; k += NW) {
            const int a = k == 0 ? r : (r + k) % (NBp - 1);
            const int b = k == 0 ? NBp - 1 : (r - k + NBp - 1) % (NBp - 1);
            if (a >= NB || b >= NB) continue;  // the dummy block
            const int i = 32 * a + lane;
            const float xi = sx[i], yi = sy[i], zi = sz[i];
            float2 rx = z2, ry = z2, rz = z2, lap = z2, v = z2;
            float cx = 0.f, cy = 0.f, cz = 0.f;
            const int src = (lane + 1) & 31;
            for (int t = 0; t < 32; t += 2) {
                const int j0 = 32 * b + ((lane + t) & 31), j1 = 32 * b + ((lane + t + 1) & 31);
                float2 gx, gy, gz, l2, v2;
                P2(xi, yi, zi, make_float2(sx[j0], sx[j1]), make_float2(sy[j0], sy[j1]), make_float2(sz[j0], sz[j1]),
                   true, true, gx, gy, gz, l2, v2);
                rx = __fadd2_rn(rx, gx);
                ry = __fadd2_rn(ry, gy);
                rz = __fadd2_rn(rz, gz);
                lap = __fadd2_rn(lap, l2);
                v = __fadd2_rn(v, v2);
                // partner drift: step t belongs to the register now here, step t+1 to the next one
                cx = __shfl_sync(FULL, cx - gx.x, src) - gx.y;
                cy = __shfl_sync(FULL, cy - gy.x, src) - gy.y;
                cz = __shfl_sync(FULL, cz - gz.x, src) - gz.y;
                cx = __shfl_sync(FULL, cx, src);
                cy = __shfl_sync(FULL, cy, src);
                cz = __shfl_sync(FULL, cz, src);
            }
            Fx[i] += rx.x + rx.y;
            Fy[i] += ry.x + ry.y;
            Fz[i] += rz.x + rz.y;
            const int jb = 32 * b + lane;
            Fx[jb] += cx;
            Fy[jb] += cy;
            Fz[jb] += cz;
            kV.add(v.x + v.y);
            kLap.add(lap.x + lap.y);
        }
        group_sync<TPW>(bar_id);
    }
    for (int b = warp; b < NB; b += NW) {  // pairs inside one block: steps 1..15, and 16 for half the lanes
        const int i = 32 * b + lane;
        const float xi = sx[i], yi = sy[i], zi = sz[i];
        float2 rx = z2, ry = z2, rz = z2, lap = z2, v = z2;
        float cx = 0.f, cy = 0.f, cz = 0.f;
        const int src1 = (lane + 1) & 31;
        for (int t = 1; t <= 16; t += 2) {
            const int j0 = 32 * b + ((lane + t) & 31), j1 = 32 * b + ((lane + t + 1) & 31);
            float2 gx, gy, gz, l2, v2;
            P2(xi, yi, zi, make_float2(sx[j0], sx[j1]), make_float2(sy[j0], sy[j1]), make_float2(sz[j0], sz[j1]),
               true, t + 1 < 16 || lane < 16, gx, gy, gz, l2, v2);
            rx = __fadd2_rn(rx, gx);
            ry = __fadd2_rn(ry, gy);
            rz = __fadd2_rn(rz, gz);
            lap = __fadd2_rn(lap, l2);
            v = __fadd2_rn(v, v2);
            cx = __shfl_sync(FULL, cx - gx.x, src1) - gx.y;  // step t, then step t+1
            cy = __shfl_sync(FULL, cy - gy.x, src1) - gy.y;
            cz = __shfl_sync(FULL, cz - gz.x, src1) - gz.y;
            if (t + 1 < 16) {
                cx = __shfl_sync(FULL, cx, src1);
                cy = __shfl_sync(FULL, cy, src1);
                cz = __shfl_sync(FULL, cz, src1);
            }
        }
        // after step 16 lane l holds the partner total of atom 32b + ((l + 16) mod 32)
        const int src = (lane + 16) & 31;
        cx = __shfl_sync(FULL, cx, src);
        cy = __shfl_sync(FULL, cy, src);
        cz = __shfl_sync(FULL, cz, src);
        Fx[i] += (rx.x + rx.y) + cx;
        Fy[i] += (ry.x + ry.y) + cy;
        Fz[i] += (rz.x + rz.y) + cz;
        kV.add(v.x + v.y);
        kLap.add(lap.x + lap.y);
    }
    group_sync<TPW>(bar_id);
    double sF2 = 0.0;
    for (int i = gtid; i < n; i += TPW) sF2 += (double)Fx[i] * Fx[i] + (double)Fy[i] * Fy[i] + (double)Fz[i] * Fz[i];
    double sV = group_sum<TPW>(kV.value(), redD, phD, bar_id, gtid);
    // each pair's term belongs to both atoms; the packed pair form leaves the constant factors out
    double sLap = 2.0 * (double)P2.LSCALE * group_sum<TPW>(kLap.value(), redD, phD, bar_id, gtid);
    sF2 = (double)P2.GSCALE * (double)P2.GSCALE * group_sum<TPW>(sF2, redD, phD, bar_id, gtid);
    const double k = 0.5 * h2m;
    out[0] = sV;
    out[1] = -k * (sLap + sF2);
    out[2] = -0.5 * k * sLap;
    out[3] = k * sF2;
    out[4] = out[0] + out[1];
}

// Local energy pieces (Sec. 2 Hamiltonian).  Rows i are spread over the group one warp-block of
// 32 consecutive rows at a time; partners j are read as broadcast 16-byte chunks.  The drift
// F_i = sum_j u'(r) (r_i - r_j)/r needs every ordered pair; V and the Laplacian term
// u'' + 2u'/r are symmetric, so they are taken once per pair (j > i) and the warp skips them
// for chunks that lie wholly at or below its block's first row.
// out = {V, T_L, T_PB, T_F, E_L}, valid in every thread of the group.  With parts > 1 the group
// takes rows part*TPW .. of every parts*TPW and out holds that share (every output is linear in
// the row sums, so the shares of all parts add up to the walker's values).
template <typename T, int MEXP, bool SYM, int TPW>
__device__ void group_energy(const Jas<T, MEXP, SYM> &J, const T *sx, const T *sy, const T *sz, int n, int nv,
                             double h2m, double *redD, int &phD, int bar_id, int gtid, double out[5], int part = 0,
                             int parts = 1)
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    const T L = J.L, iL = (T)1 / J.L, hL2 = J.hL2, m = J.m, mm1 = J.m * (J.m + (T)1);
    // exponent 5 with the symmetrised u: the Jastrow terms without their constant factors, which
    // are applied to the row sums (drift times 5c, Laplacian term times 10c)
    constexpr bool FOLD = MEXP == 5 && SYM;
    const double gs = FOLD ? 5.0 * (double)J.c : 1.0, ls = FOLD ? 10.0 * (double)J.c : 1.0;
    const Aziz<T> AZ;
    const int lane = gtid & 31;
    double sV = 0.0, sLap = 0.0, sF2 = 0.0;
    for (int i0 = part * TPW + gtid - lane; i0 < n; i0 += parts * TPW) {  // warp-uniform; this CTA's rows
        const int i = i0 + lane;
        const bool row = i < n;
        const int ii = row ? i : n - 1;
        const T xi = sx[ii], yi = sy[ii], zi = sz[ii];
        RowSum<T> sv, slap, sfx, sfy, sfz;
        for (int c0 = 0; c0 < nv; c0 += row_block<T>()) {
            const int c1 = min(nv, c0 + row_block<T>());
            T v = 0, lap = 0, fx = 0, fy = 0, fz = 0;
            for (int c = c0; c < c1; ++c) {
                const V X = reinterpret_cast<const V *>(sx)[c];
                const V Y = reinterpret_cast<const V *>(sy)[c];
                const V Z = reinterpret_cast<const V *>(sz)[c];
                const bool upper = c * VN + VN - 1 > i0;  // some lane of the warp has j > i here
#pragma unroll
                for (int e = 0; e < VN; ++e) {
                    const int j = c * VN + e;
                    const T dx = mi_signed(xi - Vec<T>::get(X, e), L, iL);
                    const T dy = mi_signed(yi - Vec<T>::get(Y, e), L, iL);
                    const T dz = mi_signed(zi - Vec<T>::get(Z, e), L, iL);
                    const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    const bool ok = (r2 < hL2) && (j != i) && (j < n);
                    const T q = Fn<T>::rsqrt(r2);
                    const T r = r2 * q;
                    if constexpr (FOLD) {
                        // A = q^6, B = w^6: u'/r = 5c (B - A) q, u'' + 2u'/r = 10c [q (B + 2A) + 3 B w]
                        const T q2 = q * q, A6 = q2 * q2 * q2;
                        const T iw = Fn<T>::rcp(L - r), w2 = iw * iw, B6 = w2 * w2 * w2;
                        const T g = (B6 - A6) * q;
                        fx += ok ? g * dx : (T)0;
                        fy += ok ? g * dy : (T)0;
                        fz += ok ? g * dz : (T)0;
                        if (upper) {
                            const bool half = ok && j > i;
                            lap += half ? fma(fma((T)2, A6, B6), q, B6 * ((T)3 * iw)) : (T)0;
                            v += half ? AZ(r, r2, q, q2, A6) : (T)0;
                        }
                    } else {
                        const T f0 = J.fq(q, r);  // f(r) = c r^-m
                        T u1 = -m * f0 * q, u2 = mm1 * f0 * (q * q);
                        if (SYM) {
                            const T w = L - r, iw = Fn<T>::rcp(w);
                            const T g0 = J.fq(iw, w);  // f(L - r)
                            u1 += m * g0 * iw;
                            u2 += mm1 * g0 * (iw * iw);
                        }
                        const T g = u1 * q;
                        fx += ok ? g * dx : (T)0;
                        fy += ok ? g * dy : (T)0;
                        fz += ok ? g * dz : (T)0;
                        if (upper) {
                            const bool half = ok && j > i;
                            lap += half ? fma((T)2 * u1, q, u2) : (T)0;
                            v += half ? AZ(r, r2, q) : (T)0;
                        }
                    }
                }
            }
            sv.add(v);
            slap.add(lap);
            sfx.add(fx);
            sfy.add(fy);
            sfz.add(fz);
        }
        if (row) {
            const double fx = gs * sfx.value(), fy = gs * sfy.value(), fz = gs * sfz.value();
            sV += sv.value();
            sLap += 2.0 * ls * slap.value();  // each pair's Laplacian term belongs to both atoms
            sF2 += fx * fx + fy * fy + fz * fz;
        }
    }
    sV = group_sum<TPW>(sV, redD, phD, bar_id, gtid);
    sLap = group_sum<TPW>(sLap, redD, phD, bar_id, gtid);
    sF2 = group_sum<TPW>(sF2, redD, phD, bar_id, gtid);
    const double k = 0.5 * h2m;
    out[0] = sV;
    out[1] = -k * (sLap + sF2);
    out[2] = -0.5 * k * sLap;
    out[3] = k * sF2;
    out[4] = out[0] + out[1];
}

// ----------------------------------------------------------------------------------------------
// Batched moves.  A batch of K consecutive trial moves (distinct atoms s_0..s_{K-1}) is
// evaluated against the configuration X at the start of the batch: for every partner j the
// partner loop adds u(|b_i - r_j|) - u(|a_i - r_j|) to S_i, where a_i = r_{s_i} and
// b_i = wrap(a_i + delta_i).  The decisions are then taken in order; if move k < i was accepted,
// atom s_k sits at b_k instead of a_k when move i is tried, which changes exactly one term of
// Delta_i by
//     D_ik = [u(|b_i - b_k|) - u(|a_i - b_k|)] - [u(|b_i - a_k|) - u(|a_i - a_k|)],
// computed during the same loop by the thread that owns atom s_k's chunk.  So
// Delta_i = S_i + sum_{k < i, accepted} D_ik is Eq. (JastrowUpdate) for the true configuration.
// A batch that draws the same atom twice is done one move at a time.
// ----------------------------------------------------------------------------------------------
// Accepted moves of the previous batch (a private copy per thread), appended in batch order.
// With two or more moves per batch the entries are addressed by the running count, so the
// compiler keeps them in local memory (L1): measured faster at N = 1952, 128 threads per walker
// (20.9 against 21.7 ms per step) than entries held in registers across the partner loop.
template <typename T, int KM> struct Recent {
    int s[KM];
    T x[KM], y[KM], z[KM];
    int cnt;
    __device__ __forceinline__ void clear() { cnt = 0; }
    __device__ __forceinline__ void add(int a, T px, T py, T pz)
    {
        s[cnt] = a;
        x[cnt] = px;
        y[cnt] = py;
        z[cnt] = pz;
        ++cnt;
    }
    __device__ __forceinline__ void lookup(int a, T &px, T &py, T &pz) const
    {
#pragma unroll
        for (int q = 0; q < KM; ++q)
            if (q < cnt && s[q] == a) {
                px = x[q];
                py = y[q];
                pz = z[q];
            }
    }
};

template <typename T, int MEXP, bool SYM>
__device__ __forceinline__ T pair_du(const Jas<T, MEXP, SYM> &J, T xj, T yj, T zj, T ax, T ay, T az, T bx, T by,
                                     T bz)
{
    const T L = J.L;
    const T px = mi_abs(ax - xj, L), py = mi_abs(ay - yj, L), pz = mi_abs(az - zj, L);
    const T qx = mi_abs(bx - xj, L), qy = mi_abs(by - yj, L), qz = mi_abs(bz - zj, L);
    return J.u(fma(qx, qx, fma(qy, qy, qz * qz))) - J.u(fma(px, px, fma(py, py, pz * pz)));
}

// The FP32 sweep with exponent 5 and the symmetrised u runs the packed partner loop (Packed5)
template <typename T, int MEXP, bool SYM> constexpr bool packed5()
{
    return std::is_same<T, float>::value && MEXP == 5 && SYM;
}

// This thread's partner sums S[0..K-1] of one batch; the owners of the moved atoms' chunks
// also write the cross terms D_ik (i > k) to dsm[i * K + k].  In the partner loop every moved
// atom is replaced by NaN, which contributes exactly zero to every sum (the clamp), so the loop
// has a single fast path; afterwards the owner of atom s_k adds its terms as a partner of the
// other moves, u(|b_i - a_k|) - u(|a_i - a_k|), and the cross terms.
template <typename T, int MEXP, bool SYM, int TPW, int K, bool GM = false>
__device__ __forceinline__ void batch_partners(const Jas<T, MEXP, SYM> &J, const T *sx, const T *sy, const T *sz,
                                               int n, int nv, const int (&s)[K], const T (&ax)[K], const T (&ay)[K],
                                               const T (&az)[K], const T (&bx)[K], const T (&by)[K],
                                               const T (&bz)[K], T (&S)[K], T *dsm, int gtid)
{
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::N;
    int cs[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        cs[i] = s[i] / VN;
        S[i] = (T)0;
    }
    if constexpr (packed5<T, MEXP, SYM>()) {
        Packed5 P;
        P.init(J);
        // one f32x2 lane pair per move: (old, new) position, and acc = (sum at a_i, sum at b_i);
        // the difference r_j - p is taken as fma(p, -1, r_j), the exactly rounded r_j - p
        float2 px[K], py[K], pz[K], acc[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            px[i] = make_float2(ax[i], bx[i]);
            py[i] = make_float2(ay[i], by[i]);
            pz[i] = make_float2(az[i], bz[i]);
            acc[i] = make_float2(0.f, 0.f);
        }
#pragma unroll (K == 1 ? 2 : 1)
        for (int c = gtid; c < nv; c += TPW) {
            float4 X = reinterpret_cast<const float4 *>(sx)[c];
            float4 Y = reinterpret_cast<const float4 *>(sy)[c];
            float4 Z = reinterpret_cast<const float4 *>(sz)[c];
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (c == cs[k]) {
                    const int e = s[k] - 4 * c;
                    Vec<float>::set(X, e, qnan<float>());
                    Vec<float>::set(Y, e, qnan<float>());
                    Vec<float>::set(Z, e, qnan<float>());
                }
            if (GM && c == nv - 1)  // entries past n (HBM padding of a walker used in place)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * c + e >= n) {
                        Vec<float>::set(X, e, qnan<float>());
                        Vec<float>::set(Y, e, qnan<float>());
                        Vec<float>::set(Z, e, qnan<float>());
                    }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float xe = Vec<float>::get(X, e), ye = Vec<float>::get(Y, e), ze = Vec<float>::get(Z, e);
                const float2 xj = make_float2(xe, xe), yj = make_float2(ye, ye), zj = make_float2(ze, ze);
#pragma unroll
                for (int i = 0; i < K; ++i)
                    P.acc5(__ffma2_rn(px[i], P.m1, xj), __ffma2_rn(py[i], P.m1, yj), __ffma2_rn(pz[i], P.m1, zj),
                           acc[i]);
            }
        }
        if constexpr (K > 1) {
            // the owner of moved atom s_k adds it as a partner of the other moves at a_k and, for
            // the later moves, writes D_ik = [u(|b_i - b_k|) - u(|a_i - b_k|)] - [u(|b_i - a_k|) - u(|a_i - a_k|)]
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (gtid == cs[k] % TPW) {
                    const float2 akx = make_float2(ax[k], ax[k]), aky = make_float2(ay[k], ay[k]),
                                 akz = make_float2(az[k], az[k]);
                    const float2 bkx = make_float2(bx[k], bx[k]), bky = make_float2(by[k], by[k]),
                                 bkz = make_float2(bz[k], bz[k]);
#pragma unroll
                    for (int i = 0; i < K; ++i) {
                        if (i == k) continue;
                        float2 ta = make_float2(0.f, 0.f);
                        P.acc5(__ffma2_rn(px[i], P.m1, akx), __ffma2_rn(py[i], P.m1, aky),
                               __ffma2_rn(pz[i], P.m1, akz), ta);
                        acc[i] = __fadd2_rn(acc[i], ta);
                        if (i > k) {
                            float2 tb = make_float2(0.f, 0.f);
                            P.acc5(__ffma2_rn(px[i], P.m1, bkx), __ffma2_rn(py[i], P.m1, bky),
                                   __ffma2_rn(pz[i], P.m1, bkz), tb);
                            dsm[i * K + k] = J.c * ((tb.y - tb.x) - (ta.y - ta.x));
                        }
                    }
                }
        }
        // every partner (the masked ones at the clamp included) is in both sums, so the constants
        // K cancel: S = c (sum_new - sum_old)
#pragma unroll
        for (int i = 0; i < K; ++i) S[i] = J.c * (acc[i].y - acc[i].x);
    } else {
#pragma unroll 2
        for (int c = gtid; c < nv; c += TPW) {
            V X = reinterpret_cast<const V *>(sx)[c];
            V Y = reinterpret_cast<const V *>(sy)[c];
            V Z = reinterpret_cast<const V *>(sz)[c];
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (c == cs[k]) {
                    const int e = s[k] - VN * c;
                    Vec<T>::set(X, e, qnan<T>());
                    Vec<T>::set(Y, e, qnan<T>());
                    Vec<T>::set(Z, e, qnan<T>());
                }
            if (GM && c == nv - 1)  // entries past n (HBM padding of a walker used in place)
#pragma unroll
                for (int e = 0; e < VN; ++e)
                    if (VN * c + e >= n) {
                        Vec<T>::set(X, e, qnan<T>());
                        Vec<T>::set(Y, e, qnan<T>());
                        Vec<T>::set(Z, e, qnan<T>());
                    }
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const T xj = Vec<T>::get(X, e), yj = Vec<T>::get(Y, e), zj = Vec<T>::get(Z, e);
#pragma unroll
                for (int i = 0; i < K; ++i) S[i] += pair_du(J, xj, yj, zj, ax[i], ay[i], az[i], bx[i], by[i], bz[i]);
            }
        }
    }
    if constexpr (K > 1 && !packed5<T, MEXP, SYM>()) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (gtid == cs[k] % TPW) {
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    if (i == k) continue;
                    const T t = pair_du(J, ax[k], ay[k], az[k], ax[i], ay[i], az[i], bx[i], by[i], bz[i]);
                    S[i] += t;
                    if (i > k) dsm[i * K + k] = pair_du(J, bx[k], by[k], bz[k], ax[i], ay[i], az[i], bx[i], by[i], bz[i]) - t;
                }
            }
    }
}

// Sum K <= KB values over the group with one barrier (identical in every thread).  red holds
// 2 phases x KB x (TPW/32) slots.  The phases are KB x (TPW/32) slots apart for every K, so that a
// batch of K moves and a following single move (ph alternates) never share a slot: a thread that
// is already writing the next batch's partials cannot overwrite ones another thread still reads.
template <int TPW, int K, typename T> __device__ __forceinline__ void group_sum_k(T (&v)[K], T *red, int ph, int bar_id, int gtid)
{
    if constexpr (K == 2 && TPW == 128 && std::is_same<T, float>::value) {
        // two sums in one butterfly: after the first exchange lanes 0-15 carry the first sum and
        // lanes 16-31 the second (5 shuffles instead of 10: 20.02 against 20.19 ms per step at
        // N = 1952, 528 walkers); the four warps' partials of a sum are one 16-byte load
        const int lane = gtid & 31;
        const bool lo = lane < 16;
        float keep = lo ? v[0] : v[1];
        const float send = lo ? v[1] : v[0];
        keep += __shfl_xor_sync(FULL, send, 16);
        keep += __shfl_xor_sync(FULL, keep, 8);
        keep += __shfl_xor_sync(FULL, keep, 4);
        keep += __shfl_xor_sync(FULL, keep, 2);
        keep += __shfl_xor_sync(FULL, keep, 1);
        float *r = red + ph * (KB * 4);  // 16-byte aligned: the slots start on a 16-byte boundary
        if ((lane & 15) == 0) r[(lane >> 4) * 4 + (gtid >> 5)] = keep;
        group_sync<TPW>(bar_id);
        const float4 a = reinterpret_cast<const float4 *>(r)[0], b = reinterpret_cast<const float4 *>(r)[1];
        v[0] = ((a.x + a.y) + a.z) + a.w;
        v[1] = ((b.x + b.y) + b.z) + b.w;
        return;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = warp_sum(v[i]);
    if (TPW == 32) {
        __syncwarp();
        return;
    }
    constexpr int NW = TPW / 32;
    T *r = red + ph * KB * NW;  // phases KB x NW apart whatever K: batches of any size alternate safely
    if ((gtid & 31) == 0) {
#pragma unroll
        for (int i = 0; i < K; ++i) r[i * NW + (gtid >> 5)] = v[i];
    }
    group_sync<TPW>(bar_id);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        T t = r[i * NW];
#pragma unroll
        for (int w = 1; w < NW; ++w) t += r[i * NW + w];
        v[i] = t;
    }
}

// One batch of K moves.  Returns false on a non-finite ratio (identically in every thread).
template <typename T, int MEXP, bool SYM, int TPW, int K, int KM, bool GM>
__device__ __forceinline__ bool move_batch(const Jas<T, MEXP, SYM> &J, T *sx, T *sy, T *sz, int n, int nv,
                                           const int (&s)[K], const T (&dx)[K], const T (&dy)[K], const T (&dz)[K],
                                           const T (&xi)[K], Recent<T, KM> &rec, LogPsiAcc<T> &lp, int &nacc, T *red,
                                           T *dsm_base, int &ph, int bar_id, int gtid)
{
    constexpr int VN = Vec<T>::N;
    const T L = J.L;
    T ax[K], ay[K], az[K], bx[K], by[K], bz[K], S[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        ax[i] = sx[s[i]];
        ay[i] = sy[s[i]];
        az[i] = sz[s[i]];
        rec.lookup(s[i], ax[i], ay[i], az[i]);
        bx[i] = wrap(ax[i] + dx[i], L);
        by[i] = wrap(ay[i] + dy[i], L);
        bz[i] = wrap(az[i] + dz[i], L);
    }
    T *dsm = dsm_base + ph * KM * KM;
    batch_partners<T, MEXP, SYM, TPW, K, GM>(J, sx, sy, sz, n, nv, s, ax, ay, az, bx, by, bz, S, dsm, gtid);
    group_sum_k<TPW, K>(S, red, ph, bar_id, gtid);
    ph ^= 1;
    bool acc[K];
    rec.clear();
#pragma unroll
    for (int i = 0; i < K; ++i) {
        T delta = S[i];
#pragma unroll
        for (int k = 0; k < i; ++k)
            if (acc[k]) delta += dsm[i * K + k];
        if (delta != delta) return false;
        // Eq. (Decision): accept iff |psi'|^2 / |psi|^2 = exp(2 Delta) > xi
        if constexpr (std::is_same<T, float>::value)
            acc[i] = 2.f * delta > xi[i];  // xi holds ln xi for FP32
        else
            acc[i] = exp(2.0 * delta) > xi[i];
        if (acc[i]) {
            if (gtid == 0) lp.add(delta);
            ++nacc;
        }
    }
    // Only the owner of an accepted atom's chunk writes its new position; every thread keeps the
    // batch's accepted moves in its private copy, which the next batch reads for the atoms it moves
    // (the owner's writes are visible to the other threads only after the next barrier).
    // Measured at N = 1952, 528 walkers: 20.95 ms per step, against 21.49 when every thread wrote
    // every accepted position itself and read it back from shared memory.
#pragma unroll
    for (int i = 0; i < K; ++i)
        if (acc[i]) {
            if (gtid == (s[i] / VN) % TPW) {
                sx[s[i]] = bx[i];
                sy[s[i]] = by[i];
                sz[s[i]] = bz[i];
            }
            rec.add(s[i], bx[i], by[i], bz[i]);
        }
    if (TPW == 32) __syncwarp();
    return true;
}

// ----------------------------------------------------------------------------------------------
// Helpers of the bounded waits and of the cluster sweep
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(unsigned long long *mb, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}

// u(|b - r|) - u(|a - r|) of one partner at r, in the same arithmetic as the partner loop
__device__ __forceinline__ float cross5(const Jas<float, 5, true> &J, float ax, float ay, float az, float bx,
                                        float by, float bz, float rx, float ry, float rz)
{
    Packed5 P;
    P.init(J);
    float2 acc = make_float2(0.f, 0.f);
    P.acc5(make_float2(ax - rx, bx - rx), make_float2(ay - ry, by - ry), make_float2(az - rz, bz - rz), acc);
    return J.c * (acc.y - acc.x);
}

// ----------------------------------------------------------------------------------------------
// The sweep: one group advances one walker through moves [m_begin, m_end) of the call (move m is
// move m mod n of sweep k0 + m / n), doing the after-sweep work (ln psi recompute, energy sample)
// at every sweep it completes.  The walker is loaded from HBM at the start and written back at the
// end; `last` marks the range that ends the call (the walker's sweep counter advances then).
// Returns false if the walker faulted (nothing of it is written back).
// ----------------------------------------------------------------------------------------------
template <typename T, int MEXP, bool SYM, int TPW, bool GM>
__device__ bool run_range(const SweepArgs &a, const DevWalker &d, GroupMem<T> mem, int gtid, int bar_id,
                          long long m_begin, long long m_end, bool last)
{
    // GM: the walker is used in place in HBM; otherwise it is copied to shared memory (the
    // address space is a compile-time property so that shared loads stay shared loads)
    T *const gx = reinterpret_cast<T *>(a.pos) + d.off;
    if constexpr (GM) mem.use_global(gx, d.pad);
    T *sx = mem.sx, *sy = mem.sy, *sz = mem.sz, *redT = mem.redT;
    double *redD = mem.redD;
    constexpr int VN = Vec<T>::N;
    const int n = d.n, pad = d.pad, nv = (n + VN - 1) / VN;
    const int slot = d.slot;
    const T L = (T)d.L, step = (T)d.step;
    int phT = 0, phD = 0;
    bool loaded;
    if constexpr (GM)
        loaded = check_walker<T, TPW>(gx, n, pad, L, redT, phT, bar_id, gtid);
    else
        loaded = load_walker<T, TPW>(gx, n, pad, a.stride, L, sx, sy, sz, redT, phT, bar_id, gtid);
    if (!loaded) {
        if (gtid == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_POS);
        return false;
    }
    Jas<T, MEXP, SYM> J;
    J.init(d);

    LogPsiAcc<T> lp;
    lp.set(a.logpsi[slot]);
    const unsigned long long k0 = a.sweep[slot];
    double *A = a.accum + QMC_ACCUM_FIELDS * (size_t)slot;
    int nacc = 0;
    constexpr int K = kb_of<T, TPW>();  // moves per batch
    Recent<T, K> rec;
    rec.clear();
    const int lane = gtid & 31;
    const uint32_t wid = d.wid;
    T *dsm = mem.dsm;  // cross terms of a batch

    for (long long m = m_begin; m < m_end;) {
        const long long it = m / n;
        const int t_start = (int)(m - it * n);
        const int t_stop = (int)min((long long)n, (long long)t_start + (m_end - m));
        m += t_stop - t_start;
        const unsigned long long kk = k0 + (unsigned long long)it;
        const uint32_t k = (uint32_t)kk;
        for (int t0 = t_start & ~31; t0 < t_stop; t0 += 32) {
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
            // FP32: the decision is taken as 2 Delta > ln xi, with ln xi computed here once per move
            if constexpr (std::is_same<T, float>::value) mxi = logf(mxi);
            const int cnt = min(32, t_stop - t0);
            int tt = max(0, t_start - t0);
            for (; tt + K <= cnt; tt += K) {
                int bs[K];
                T bdx[K], bdy[K], bdz[K], bxi[K];
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    bs[i] = __shfl_sync(FULL, my_s, tt + i);
                    bdx[i] = __shfl_sync(FULL, mdx, tt + i);
                    bdy[i] = __shfl_sync(FULL, mdy, tt + i);
                    bdz[i] = __shfl_sync(FULL, mdz, tt + i);
                    bxi[i] = __shfl_sync(FULL, mxi, tt + i);
                }
                bool distinct = true;
#pragma unroll
                for (int i = 0; i < K; ++i)
#pragma unroll
                    for (int q = i + 1; q < K; ++q) distinct &= bs[i] != bs[q];
                bool ok = true;
                if (distinct) {
                    ok = move_batch<T, MEXP, SYM, TPW, K, K, GM>(J, sx, sy, sz, n, nv, bs, bdx, bdy, bdz, bxi, rec, lp,
                                                               nacc, redT, dsm, phT, bar_id, gtid);
                } else {
                    for (int i = 0; i < K && ok; ++i) {
                        const int s1[1] = {bs[i]};
                        const T x1[1] = {bdx[i]}, y1[1] = {bdy[i]}, z1[1] = {bdz[i]}, c1[1] = {bxi[i]};
                        ok = move_batch<T, MEXP, SYM, TPW, 1, K, GM>(J, sx, sy, sz, n, nv, s1, x1, y1, z1, c1, rec, lp,
                                                                  nacc, redT, dsm, phT, bar_id, gtid);
                    }
                }
                if (!ok) {
                    if (gtid == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_RATIO);
                    return false;
                }
            }
            for (; tt < cnt; ++tt) {
                const int s1[1] = {__shfl_sync(FULL, my_s, tt)};
                const T x1[1] = {__shfl_sync(FULL, mdx, tt)}, y1[1] = {__shfl_sync(FULL, mdy, tt)},
                        z1[1] = {__shfl_sync(FULL, mdz, tt)}, c1[1] = {__shfl_sync(FULL, mxi, tt)};
                if (!move_batch<T, MEXP, SYM, TPW, 1, K, GM>(J, sx, sy, sz, n, nv, s1, x1, y1, z1, c1, rec, lp, nacc, redT,
                                                          dsm, phT, bar_id, gtid)) {
                    if (gtid == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_RATIO);
                    return false;
                }
            }
        }
        if (t_stop < n) break;  // the range ends inside this sweep
        group_sync<TPW>(bar_id);
        rec.clear();
        if (a.recompute_every > 0 && (kk + 1) % (unsigned long long)a.recompute_every == 0) {
            // Eq. (Jastrow) from scratch; the drift of the carried sum (thread 0 carries it) is
            // recorded before it is replaced
            const double fresh = group_log_psi<T, MEXP, SYM, TPW>(J, sx, sy, sz, n, nv, redD, phD, bar_id, gtid);
            if (gtid == 0) {
                const double drift = fabs(lp.value() - fresh);
                A[8] += drift;
                A[9] = fmax(A[9], drift);
            }
            lp.set(fresh);
        }
        if (a.energy_every > 0 && (kk + 1) % (unsigned long long)a.energy_every == 0) {
            double e[5];
            if constexpr (std::is_same<T, float>::value && !GM) {
                if (a.tile)
                    group_energy_tiled<MEXP, SYM, TPW>(J, sx, sy, sz, mem.fx, mem.fy, mem.fz, n, a.h2m, redD, phD,
                                                       bar_id, gtid, e);
                else
                    group_energy<T, MEXP, SYM, TPW>(J, sx, sy, sz, n, nv, a.h2m, redD, phD, bar_id, gtid, e);
            } else {
                group_energy<T, MEXP, SYM, TPW>(J, sx, sy, sz, n, nv, a.h2m, redD, phD, bar_id, gtid, e);
            }
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
    if constexpr (!GM) store_walker<T, TPW>(gx, n, pad, sx, sy, sz, gtid);
    if (gtid == 0) {
        A[7] += (double)nacc;  // integer-valued: exact in any order
        a.logpsi[slot] = lp.value();
        if (last) a.sweep[slot] = k0 + (unsigned long long)a.nsweeps;
    }
    return true;
}

// ----------------------------------------------------------------------------------------------
// FIFO of ready walkers (persistent mode).  A bounded multi-producer multi-consumer ring with a
// sequence number per slot: the pop of ticket p waits for sequence p + 1, takes the walker and
// frees the slot (sequence p + W); the push of ticket p waits for sequence p, stores the walker
// and publishes it (sequence p + 1).  It starts full (all W walkers) and exactly W walkers
// circulate, so a push finds its slot free as soon as the matching pop has left it.  Every wait
// is bounded (the call's limit, 10 s of global time unless a failure test shortens it); on expiry
// the error word gets QMC_DEVERR_TIMEOUT.
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ bool wait_seq(unsigned *seq_word, unsigned want, unsigned long long limit_ns,
                                         unsigned *err)
{
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> seq(*seq_word);
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < (1u << 30); ++it) {
        if (seq.load(cuda::memory_order_acquire) == want) return true;
        if ((it & 63) == 63 && global_ns() - t0 > limit_ns) break;
        __nanosleep(128);
    }
    atomicOr(err, QMC_DEVERR_TIMEOUT);
    return false;
}

// next walker table index, or -1 when all chunks have been handed out (or on a timeout)
__device__ __forceinline__ int queue_pop(const SweepArgs &a, unsigned total)
{
    const unsigned pos = atomicAdd(a.q_head, 1u);
    if (pos >= total) return -1;
    uint2 *sl = a.q_slots + pos % (unsigned)a.W;
    if (!wait_seq(&sl->x, pos + 1, a.wait_ns, a.err)) return -1;
    const int w = (int)*reinterpret_cast<volatile unsigned *>(&sl->y);
    cuda::atomic_ref<unsigned, cuda::thread_scope_device>(sl->x).store(pos + (unsigned)a.W,
                                                                       cuda::memory_order_release);
    return w;
}

__device__ __forceinline__ void queue_push(const SweepArgs &a, int w)
{
    const unsigned pos = atomicAdd(a.q_tail, 1u);
    uint2 *sl = a.q_slots + pos % (unsigned)a.W;
    if (!wait_seq(&sl->x, pos, a.wait_ns, a.err)) return;
    *reinterpret_cast<volatile unsigned *>(&sl->y) = (unsigned)w;
    cuda::atomic_ref<unsigned, cuda::thread_scope_device>(sl->x).store(pos + 1, cuda::memory_order_release);
}



// Persistent mode: take ready walkers from the FIFO, advance each by one chunk, put it back.
template <typename T, int MEXP, bool SYM, int TPW>
__device__ __forceinline__ void persistent_loop(const SweepArgs &a, GroupMem<T> mem, int g, int gtid)
{
    constexpr int DEAD = 1 << 30;
    for (;;) {
        if (gtid == 0) *mem.bc = queue_pop(a, a.q_total);
        group_sync<TPW>(1 + g);
        const int w = *mem.bc;
        group_sync<TPW>(1 + g);
        if (w < 0) return;
        // the walker was last written by another SM: acquire its state (positions, ln psi, sums)
        cuda::atomic_thread_fence(cuda::memory_order_acquire, cuda::thread_scope_device);
        const DevWalker d = a.walkers[w];
        const long long total = (long long)a.nsweeps * d.n;
        const int c = a.q_prog[w];
        const long long m0 = (long long)(c & (DEAD - 1)) * a.chunk_moves;
        const long long m1 = min(total, m0 + a.chunk_moves);
        bool ok = true;
        if (!(c & DEAD))
            ok = a.gmem ? run_range<T, MEXP, SYM, TPW, true>(a, d, mem, gtid, 1 + g, m0, m1, m1 == total)
                        : run_range<T, MEXP, SYM, TPW, false>(a, d, mem, gtid, 1 + g, m0, m1, m1 == total);
        __threadfence();  // this thread's stores of the walker state, before it is handed on
        group_sync<TPW>(1 + g);
        if (gtid == 0) {
            a.q_prog[w] = (c + 1) | (ok ? 0 : DEAD);
            __threadfence();
            // (a failure test drops one push: the pops that wait for it run out, bounded)
            const bool dropped = a.drop_push && c == 0 && w == a.order[0];
            if (m1 < total && !dropped) queue_push(a, w);
        }
    }
}

// CTAs hold up to 256 threads (TPW <= 256) or exactly one group.  Launch bounds: at least 512
// resident threads per SM, i.e. up to 128 registers per thread, except for groups of 1024
// threads, which keep 64.
template <int TPW> constexpr int cta_bound() { return TPW > 256 ? TPW : 256; }
template <int TPW> constexpr int min_blocks() { return TPW <= 256 ? 2 : 1; }

template <typename T, int MEXP, bool SYM, int TPW>
__global__ void __launch_bounds__(cta_bound<TPW>(), min_blocks<TPW>()) sweep_kernel(SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = threadIdx.x / TPW, gtid = threadIdx.x % TPW;
    const int item = blockIdx.x * a.G + g;
    if (!a.dynamic && item >= a.W) return;  // only group barriers follow, so whole groups may leave
    GroupMem<T> mem;
    mem.bind(smem + (size_t)g * group_smem<T>(a.stride, TPW, a.tile == 1), a.stride, TPW, a.tile == 1);
    if (a.tile == 2) mem.use_global_drift(a.fscr + (size_t)3 * a.stride * (blockIdx.x * a.G + g), a.stride);
    if (!a.dynamic) {
        const DevWalker d = a.walkers[a.order[item]];
        const long long total = (long long)a.nsweeps * d.n;
        if (a.gmem)
            run_range<T, MEXP, SYM, TPW, true>(a, d, mem, gtid, 1 + g, 0, total, true);
        else
            run_range<T, MEXP, SYM, TPW, false>(a, d, mem, gtid, 1 + g, 0, total, true);
        return;
    }
    persistent_loop<T, MEXP, SYM, TPW>(a, mem, g, gtid);
}

// ----------------------------------------------------------------------------------------------
// Uneven batches with dominant walkers (FP32, exponent 5, symmetrised u): one CTA of TPWB threads
// per SM.  First the whole CTA serves the dominant walkers (`big`, the first big.W entries of the
// processing order), one whole call each, taken from a counter; then it splits into TPWB / TPWS
// groups that take the other walkers (`a`) from the queue in chunks.  The dominant walkers' moves
// are the longest sequential work of the call, so they get the most threads per move; the others
// keep the group size that suits them.
// ----------------------------------------------------------------------------------------------
template <typename T, int MEXP, bool SYM, int TPWB, int TPWS>
__global__ void __launch_bounds__(TPWB, TPWB <= 256 ? 2 : 1) sweep_mixed_kernel(SweepArgs a, SweepArgs big,
                                                                                unsigned *big_next)
{
    static_assert(TPWB % TPWS == 0 && TPWB / TPWS <= 15, "groups of the second phase");
    extern __shared__ __align__(16) unsigned char smem[];
    {
        GroupMem<T> mem;
        mem.bind(smem, big.stride, TPWB, big.tile == 1);
        if (big.tile == 2) mem.use_global_drift(big.fscr + (size_t)3 * big.stride * blockIdx.x, big.stride);
        const int gtid = threadIdx.x;
        for (;;) {
            if (gtid == 0) *mem.bc = (int)atomicAdd(big_next, 1u);
            group_sync<TPWB>(1);
            const int i = *mem.bc;
            group_sync<TPWB>(1);
            if (i >= big.W) break;
            const DevWalker d = big.walkers[big.order[i]];
            run_range<T, MEXP, SYM, TPWB, false>(big, d, mem, gtid, 1, 0, (long long)big.nsweeps * d.n, true);
            group_sync<TPWB>(1);
        }
    }
    __syncthreads();
    const int g = threadIdx.x / TPWS, gtid = threadIdx.x % TPWS;
    GroupMem<T> mem;
    mem.bind(smem + (size_t)g * group_smem<T>(a.stride, TPWS, a.tile == 1), a.stride, TPWS, a.tile == 1);
    if (a.tile == 2) mem.use_global_drift(a.fscr + (size_t)3 * a.stride * (blockIdx.x * a.G + g), a.stride);
    persistent_loop<T, MEXP, SYM, TPWS>(a, mem, g, gtid);
}

// ----------------------------------------------------------------------------------------------
// Stand-alone passes: one CTA (TPW threads) per walker
// ----------------------------------------------------------------------------------------------
struct PassArgs {
    const DevWalker *walkers;
    int W;
    int stride;
    int tile;
    int gmem;
    const void *pos;
    double *out;
    double h2m;
    // qmc_trial_delta
    const int32_t *s;
    const double *delta;
    int M;
    unsigned *err;
    // a walker's rows split over `parts` CTAs (row-wise passes of few walkers): CTA part of walker
    // w stores its share of the outputs in part_out[(w * parts + part) * 8 ..], and the last CTA
    // of the walker (part_ctr[w]) adds the shares in part order and writes the outputs
    int parts;
    double *part_out;
    unsigned *part_ctr;
};

// Called by thread 0 of every CTA of a split pass with its share v of the walker's NF outputs
// (failed: this CTA could not load the walker).  Returns true in the last CTA of the walker to
// finish, with v holding the sum of all shares in part order, unless some CTA failed; the
// counter is reset for the next launch.  With one part it returns !failed at once.
template <int NF>
__device__ bool combine_parts(const PassArgs &a, int w, int part, double (&v)[NF], bool failed)
{
    static_assert(NF <= 7, "eight slots per part: NF outputs and a failure flag");
    if (a.parts == 1) return !failed;
    double *base = a.part_out + (size_t)w * a.parts * 8;
    double *slot = base + (size_t)part * 8;
#pragma unroll
    for (int f = 0; f < NF; ++f) slot[f] = v[f];
    slot[7] = failed ? 1.0 : 0.0;
    __threadfence();
    const unsigned prev = atomicAdd(a.part_ctr + w, 1u);
    if (prev != (unsigned)(a.parts - 1)) return false;
    __threadfence();
    bool bad = false;
#pragma unroll
    for (int f = 0; f < NF; ++f) v[f] = 0.0;
    for (int p = 0; p < a.parts; ++p) {
        const volatile double *q = base + (size_t)p * 8;
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f] += q[f];
        bad |= q[7] != 0.0;
    }
    a.part_ctr[w] = 0u;
    return !bad;
}

// kind: 0 = local energy (5 outputs), 1 = ln psi (1 output)
template <typename T, int MEXP, bool SYM, int TPW>
__global__ void __launch_bounds__(TPW) pass_kernel(PassArgs a, int kind)
{
    extern __shared__ __align__(16) unsigned char smem[];
    GroupMem<T> mem;
    mem.bind(smem, a.stride, TPW, a.tile && kind == 0);
    T *sx = mem.sx, *sy = mem.sy, *sz = mem.sz, *redT = mem.redT;
    double *redD = mem.redD;
    const int w = blockIdx.x / a.parts, part = blockIdx.x % a.parts;  // walker, share of its rows
    const DevWalker d = a.walkers[w];
    const int gtid = threadIdx.x;
    int phT = 0, phD = 0;
    constexpr int VN = Vec<T>::N;
    const T *gx = reinterpret_cast<const T *>(a.pos) + d.off;
    if (a.gmem) {
        mem.use_global(const_cast<T *>(gx), d.pad);
        sx = mem.sx;
        sy = mem.sy;
        sz = mem.sz;
    }
    if (!(a.gmem ? check_walker<T, TPW>(gx, d.n, d.pad, (T)d.L, redT, phT, 1, gtid)
                 : load_walker<T, TPW>(gx, d.n, d.pad, a.stride, (T)d.L, sx, sy, sz, redT, phT, 1, gtid))) {
        if (gtid == 0) {
            atomicOr(a.err, QMC_DEVERR_NONFINITE_POS);
            double none[5] = {};
            combine_parts<5>(a, w, part, none, true);  // the walker's other parts must not wait for it
        }
        return;
    }
    Jas<T, MEXP, SYM> J;
    J.init(d);
    const int nv = (d.n + VN - 1) / VN;
    if (kind == 0) {
        double e[5];
        if constexpr (std::is_same<T, float>::value) {
            if (a.tile)  // the tiled pass is never split (parts == 1)
                group_energy_tiled<MEXP, SYM, TPW>(J, sx, sy, sz, mem.fx, mem.fy, mem.fz, d.n, a.h2m, redD, phD, 1,
                                                   gtid, e);
            else
                group_energy<T, MEXP, SYM, TPW>(J, sx, sy, sz, d.n, nv, a.h2m, redD, phD, 1, gtid, e, part, a.parts);
        } else {
            group_energy<T, MEXP, SYM, TPW>(J, sx, sy, sz, d.n, nv, a.h2m, redD, phD, 1, gtid, e, part, a.parts);
        }
        if (gtid == 0 && combine_parts<5>(a, w, part, e, false))
            for (int q = 0; q < 5; ++q) a.out[5 * (size_t)d.slot + q] = e[q];
    } else {
        double lp[1] = {group_log_psi<T, MEXP, SYM, TPW>(J, sx, sy, sz, d.n, nv, redD, phD, 1, gtid, part, a.parts)};
        if (gtid == 0 && combine_parts<1>(a, w, part, lp, false)) a.out[d.slot] = lp[0];
    }
}

// Eq. (JastrowUpdate) for M given trial moves from the unchanged configuration.
template <typename T, int MEXP, bool SYM, int TPW>
__global__ void __launch_bounds__(TPW) trial_kernel(PassArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    GroupMem<T> mem;
    mem.bind(smem, a.stride, TPW, false);
    T *sx = mem.sx, *sy = mem.sy, *sz = mem.sz, *redT = mem.redT;
    double *redD = mem.redD;
    const DevWalker d = a.walkers[blockIdx.x];
    const int gtid = threadIdx.x;
    int phT = 0;
    constexpr int VN = Vec<T>::N;
    const T *gx = reinterpret_cast<const T *>(a.pos) + d.off;
    const T L = (T)d.L;
    if (a.gmem) {
        mem.use_global(const_cast<T *>(gx), d.pad);
        sx = mem.sx;
        sy = mem.sy;
        sz = mem.sz;
    }
    if (!(a.gmem ? check_walker<T, TPW>(gx, d.n, d.pad, L, redT, phT, 1, gtid)
                 : load_walker<T, TPW>(gx, d.n, d.pad, a.stride, L, sx, sy, sz, redT, phT, 1, gtid))) {
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
        const int s1[1] = {s};
        const T ax[1] = {sx[s]}, ay[1] = {sy[s]}, az[1] = {sz[s]};
        const T bx[1] = {wrap(ax[0] + (T)a.delta[3 * mi], L)}, by[1] = {wrap(ay[0] + (T)a.delta[3 * mi + 1], L)},
                bz[1] = {wrap(az[0] + (T)a.delta[3 * mi + 2], L)};
        T S[1];
        batch_partners<T, MEXP, SYM, TPW, 1, true>(J, sx, sy, sz, d.n, nv, s1, ax, ay, az, bx, by, bz, S, nullptr,
                                                  gtid);
        const T delta = group_sum<TPW>(S[0], redT, phT, 1, gtid);
        if (gtid == 0) a.out[mi] = (double)delta;
    }
}

// ----------------------------------------------------------------------------------------------
// Pair-distance histogram (the paper's g(r) analysis, Sec. 5.4 and Sec. 7.1): counts of pairs
// i < j with r < rmax in nbins equal bins, bin = floor(r nbins / rmax), added to hist[walker].
// Counts are integers (the shared-memory atomics commute), so the result is exact.  In FP64
// the squared distance is summed unfused in x, y, z order, as the oracle does.
// ----------------------------------------------------------------------------------------------
template <typename T, int TPW>
__global__ void __launch_bounds__(TPW) hist_kernel(PassArgs a, int nbins, double rmax, unsigned long long *hist)
{
    extern __shared__ __align__(16) unsigned char smem[];
    GroupMem<T> mem;
    mem.bind(smem, a.stride, TPW, false);
    unsigned *counts = reinterpret_cast<unsigned *>(smem + group_smem<T>(a.stride, TPW, false));
    T *sx = mem.sx, *sy = mem.sy, *sz = mem.sz, *redT = mem.redT;
    const int part = blockIdx.x % a.parts;  // share of the walker's rows (counts add exactly)
    const DevWalker d = a.walkers[blockIdx.x / a.parts];
    const int gtid = threadIdx.x;
    int phT = 0;
    constexpr int VN = Vec<T>::N;
    using V = typename Vec<T>::type;
    const T *gx = reinterpret_cast<const T *>(a.pos) + d.off;
    const T L = (T)d.L, iL = (T)1 / L;
    if (a.gmem) {
        mem.use_global(const_cast<T *>(gx), d.pad);
        sx = mem.sx;
        sy = mem.sy;
        sz = mem.sz;
    }
    if (!(a.gmem ? check_walker<T, TPW>(gx, d.n, d.pad, L, redT, phT, 1, gtid)
                 : load_walker<T, TPW>(gx, d.n, d.pad, a.stride, L, sx, sy, sz, redT, phT, 1, gtid))) {
        if (gtid == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_POS);
        return;
    }
    for (int b = gtid; b < nbins; b += TPW) counts[b] = 0u;
    __syncthreads();
    const int n = d.n, nv = (n + VN - 1) / VN;
    const T r2max = (T)(rmax * rmax), scale = (T)((double)nbins / rmax);
    for (int i = part * TPW + gtid; i < n; i += a.parts * TPW) {
        const T xi = sx[i], yi = sy[i], zi = sz[i];
        for (int c = 0; c < nv; ++c) {
            const V X = reinterpret_cast<const V *>(sx)[c];
            const V Y = reinterpret_cast<const V *>(sy)[c];
            const V Z = reinterpret_cast<const V *>(sz)[c];
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const int j = c * VN + e;
                const T dx = mi_signed(xi - Vec<T>::get(X, e), L, iL);
                const T dy = mi_signed(yi - Vec<T>::get(Y, e), L, iL);
                const T dz = mi_signed(zi - Vec<T>::get(Z, e), L, iL);
                T r2;
                if constexpr (std::is_same<T, double>::value)
                    r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                else
                    r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (j > i && j < n && r2 < r2max) {
                    const int bin = min(nbins - 1, (int)(sqrt(r2) * scale));
                    atomicAdd(&counts[bin], 1u);
                }
            }
        }
    }
    __syncthreads();
    unsigned long long *h = hist + (size_t)d.slot * nbins;
    if (a.parts == 1) {
        for (int b = gtid; b < nbins; b += TPW) h[b] += counts[b];
    } else {  // several CTAs add to the walker's row: integer atomics, exact in any order
        for (int b = gtid; b < nbins; b += TPW)
            if (counts[b]) atomicAdd(h + b, (unsigned long long)counts[b]);
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
    GroupMem<T> mem;
    mem.bind(smem, a.stride, TPW, false);
    T *sx = mem.sx, *sy = mem.sy, *sz = mem.sz, *redT = mem.redT;
    double *redD = mem.redD;
    const int w = blockIdx.x / a.parts, part = blockIdx.x % a.parts;  // walker, share of its rows
    const DevWalker d = a.walkers[w];
    const int gtid = threadIdx.x;
    int phT = 0, phD = 0;
    constexpr int VN = Vec<T>::N;
    using V = typename Vec<T>::type;
    const T *gx = reinterpret_cast<const T *>(a.pos) + d.off;
    const T L = (T)d.L, iL = (T)1 / L, hL2 = (T)(0.25 * d.L * d.L);
    if (a.gmem) {
        mem.use_global(const_cast<T *>(gx), d.pad);
        sx = mem.sx;
        sy = mem.sy;
        sz = mem.sz;
    }
    if (!(a.gmem ? check_walker<T, TPW>(gx, d.n, d.pad, L, redT, phT, 1, gtid)
                 : load_walker<T, TPW>(gx, d.n, d.pad, a.stride, L, sx, sy, sz, redT, phT, 1, gtid))) {
        if (gtid == 0) {
            atomicOr(a.err, QMC_DEVERR_NONFINITE_POS);
            double none[6] = {};
            combine_parts<6>(a, w, part, none, true);  // the walker's other parts must not wait for it
        }
        return;
    }
    const int n = d.n, nv = (n + VN - 1) / VN;
    const T c = (T)d.c, m = (T)d.m, lnb = (T)::log(d.b > 0 ? d.b : 1.0);
    const T K = (T)d.K;
    // m-derivative of the shift 2 f(L/2): 2 f(L/2) ln(2b/L)
    const T Km = (T)(d.K * ::log(d.b > 0 ? 2.0 * d.b / d.L : 1.0));
    const T c1 = (T)1 / m, c2 = (T)(2.0 * d.m + 1.0) / (m * (m + (T)1));
    const Aziz<T> AZ;
    double sLp = 0, sLpm = 0, sV = 0, sLap = 0, sLapm = 0, sF2 = 0, sFFm = 0;
    for (int i = part * TPW + gtid; i < n; i += a.parts * TPW) {  // this CTA's share of the rows
        const T xi = sx[i], yi = sy[i], zi = sz[i];
        RowSum<T> a_lp, a_lpm, a_v, a_lap, a_lapm, a_fx, a_fy, a_fz, a_gx, a_gy, a_gz;
        for (int c0 = 0; c0 < nv; c0 += row_block<T>()) {
            const int cend = min(nv, c0 + row_block<T>());
            T lp = 0, lpm = 0, v = 0, lap = 0, lapm = 0, fx = 0, fy = 0, fz = 0, gx_ = 0, gy_ = 0, gz_ = 0;
            for (int cc = c0; cc < cend; ++cc) {
                const V X = reinterpret_cast<const V *>(sx)[cc];
                const V Y = reinterpret_cast<const V *>(sy)[cc];
                const V Z = reinterpret_cast<const V *>(sz)[cc];
#pragma unroll
                for (int e = 0; e < VN; ++e) {
                    const T dx = mi_signed(xi - Vec<T>::get(X, e), L, iL);
                    const T dy = mi_signed(yi - Vec<T>::get(Y, e), L, iL);
                    const T dz = mi_signed(zi - Vec<T>::get(Z, e), L, iL);
                    const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    const bool ok = (r2 < hL2) && (cc * VN + e != i) && (cc * VN + e < n);
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
                    const T vv = AZ(r, r2, q);
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
            a_lp.add(lp);
            a_lpm.add(lpm);
            a_v.add(v);
            a_lap.add(lap);
            a_lapm.add(lapm);
            a_fx.add(fx);
            a_fy.add(fy);
            a_fz.add(fz);
            a_gx.add(gx_);
            a_gy.add(gy_);
            a_gz.add(gz_);
        }
        const double fx = a_fx.value(), fy = a_fy.value(), fz = a_fz.value();
        sLp += a_lp.value();
        sLpm += a_lpm.value();
        sV += a_v.value();
        sLap += a_lap.value();
        sLapm += a_lapm.value();
        sF2 += fx * fx + fy * fy + fz * fz;
        sFFm += fx * a_gx.value() + fy * a_gy.value() + fz * a_gz.value();
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
        // every output is linear in the row sums, so the shares of a split walker add up
        double o[6] = {0.5 * sLp, 0.5 * sV - k * (sLap + sF2), mb * 0.5 * sLp, 0.5 * sLpm, -k * mb * (sLap + 2.0 * sF2),
                       -k * (sLapm + 2.0 * sFFm)};
        if (combine_parts<6>(a, w, part, o, false))
            for (int q = 0; q < 6; ++q) a.out[6 * (size_t)d.slot + q] = o[q];
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
