// qmc_cluster.cuh -- one walker split over a thread-block cluster: few walkers of very large N.
//
// With fewer walkers than SMs, one CTA per walker leaves most of the GPU idle (the paper's own
// 40 960-atom run used 13 walkers).  Here each walker is served by a cluster of C CTAs (C = 2, 4
// or 8, one per SM): CTA r holds atoms [rS, rS + S) of the walker in its shared memory.  For a
// move every CTA draws the same random numbers (the counters of Sec. 5.2, as in the one-CTA
// sweep), reads the moved atom's position from its owner's shared memory through distributed
// shared memory (DSMEM), evaluates the partner terms of Eq. (JastrowUpdate) over its slice, and
// the C partial sums are exchanged: every CTA's thread 0 stores its partial into each CTA's slot
// and arrives on each CTA's mbarrier (release at cluster scope); every thread waits on its own
// CTA's mbarrier (acquire, bounded) and adds the C partials in rank order, so all CTAs take the
// same decision (Eq. Decision).  The owner of the moved atom writes its new position; all threads
// keep a copy of the last accepted move for the one read that may precede that write's
// visibility.  FP32, exponent 5, symmetrised u; calls without energy samples or ln psi
// recomputes (those run as separate passes).
#pragma once

#include "qmc_kernels.cuh"

namespace qmc {

struct ClusterArgs {
    const DevWalker *walkers;
    int W;
    int C;          // CTAs per walker (the cluster size)
    int slice;      // shared-memory slice length (atoms, a multiple of 4) of the largest walker
    void *pos;
    double *logpsi;
    unsigned long long *sweep;
    double *accum;
    unsigned long long seed;
    int nsweeps;
    int proposal, sequential;
    unsigned *err;
};

constexpr int CLUSTER_TPW = 512;  // threads per CTA (one CTA per SM: 512 x 128 registers)
constexpr int CLUSTER_MAX = 8;    // portable cluster size

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// address in the shared::cluster window of CTA `rank` of the object at local shared address p
__device__ __forceinline__ unsigned map_rank(const void *p, unsigned rank)
{
    unsigned out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
    return out;
}

__device__ __forceinline__ float ld_cluster(unsigned addr)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ void st_cluster(unsigned addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void mb_arrive_remote(unsigned addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ bool mb_test_cluster(unsigned addr, unsigned parity)
{
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(addr), "r"(parity)
                 : "memory");
    return done != 0;
}

// bounded like every other wait: 10 s of global time, then QMC_DEVERR_TIMEOUT; once that bit is
// set, later waits fail at once
__device__ __forceinline__ bool mb_wait_cluster(unsigned long long *mb, unsigned parity, unsigned *err)
{
    const unsigned addr = smem_u32(mb);
    unsigned long long t0 = 0;
    for (unsigned it = 0; it < (1u << 30); ++it) {
        if (mb_test_cluster(addr, parity)) return true;
        if ((it & 255) == 255) {
            if (*reinterpret_cast<volatile unsigned *>(err) & QMC_DEVERR_TIMEOUT) return false;
            const unsigned long long now = global_ns();
            if (t0 == 0)
                t0 = now;
            else if (now - t0 > 10000000000ull)
                break;
        }
    }
    atomicOr(err, QMC_DEVERR_TIMEOUT);
    return false;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared memory of one CTA: x | y | z slices (slice floats each), 32 warp partials, 2 x 8
// exchange slots, 2 mbarriers
__host__ __device__ constexpr size_t cluster_smem(int slice) { return (size_t)3 * slice * 4 + 128 + 64 + 16; }

template <int TPW>
__global__ void __launch_bounds__(TPW, 1) sweep_cluster_kernel(ClusterArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NW = TPW / 32;
    const int gtid = threadIdx.x, lane = gtid & 31, warp = gtid >> 5;
    const unsigned rank = cluster_rank();
    const int C = a.C;
    float *sx = reinterpret_cast<float *>(smem), *sy = sx + a.slice, *sz = sy + a.slice;
    float *red = sz + a.slice;
    float *part = red + 32;
    unsigned long long *mb = reinterpret_cast<unsigned long long *>(part + 16);
    if (gtid == 0) {
        mb_init(mb, (unsigned)C);
        mb_init(mb + 1, (unsigned)C);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    cluster_sync_all();  // every CTA's mbarriers exist before the first remote arrive

    const DevWalker d = a.walkers[blockIdx.x / C];
    const int n = d.n;
    const int S = ((n + C - 1) / C + 3) & ~3;  // this walker's slice (multiple of 4, <= a.slice)
    const int j0 = (int)rank * S;
    const int ns = max(0, min(S, n - j0));
    const int nv = S / 4;
    float *gx = reinterpret_cast<float *>(a.pos) + d.off;
    const float L = (float)d.L, step = (float)d.step;
    Jas<float, 5, true> J;
    J.init(d);

    unsigned jx = 0;  // exchanges so far: slot set jx & 1, phase parity (jx >> 1) & 1
    // the sum over the cluster of one value per thread, identical in every CTA (rank order)
    auto exchange = [&](float v, float &total) -> bool {
        v = warp_sum(v);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        const unsigned ph = jx & 1u, par = (jx >> 1) & 1u;
        ++jx;
        if (gtid == 0) {
            float s = red[0];
#pragma unroll
            for (int w = 1; w < NW; ++w) s += red[w];
            for (int r = 0; r < C; ++r) {
                st_cluster(map_rank(&part[ph * 8 + rank], (unsigned)r), s);
                mb_arrive_remote(map_rank(&mb[ph], (unsigned)r));
            }
        }
        if (!mb_wait_cluster(&mb[ph], par, a.err)) return false;
        float t = part[ph * 8];
        for (int r = 1; r < C; ++r) t += part[ph * 8 + r];
        total = t;
        return true;
    };

    // load this CTA's slice; entries past the walker get distinct far coordinates (1e30 scale:
    // their squared distances overflow, which the clamp of the pair function turns into zero)
    int bad = 0;
    for (int i = gtid; i < S; i += TPW) {
        float x, y, z;
        if (i < ns) {
            x = gx[j0 + i];
            y = gx[d.pad + j0 + i];
            z = gx[2 * (size_t)d.pad + j0 + i];
            bad |= !(x >= 0.f && x <= L) || !(y >= 0.f && y <= L) || !(z >= 0.f && z <= L);
        } else {
            x = y = z = 1e30f * (float)(1 + i - ns);
        }
        sx[i] = x;
        sy[i] = y;
        sz[i] = z;
    }
    float nbad = 0.f;
    bool ok = exchange((float)bad, nbad);
    if (ok && nbad != 0.f) {
        if (gtid == 0 && rank == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_POS);
        ok = false;
    }

    LogPsiAcc<float> lp;
    lp.set(a.logpsi[d.slot]);
    const unsigned long long k0 = a.sweep[d.slot];
    int nacc = 0;
    int rs = -1;  // the last accepted move: atom and new position (register copy)
    float rx = 0.f, ry = 0.f, rz = 0.f;
    Packed5 P;
    P.init(J);
    for (int it = 0; ok && it < a.nsweeps; ++it) {
        const uint32_t k = (uint32_t)(k0 + (unsigned long long)it);
        for (int t0 = 0; ok && t0 < n; t0 += 32) {
            // random numbers of moves t0 .. t0+31, one move per lane, as in the one-CTA sweep
            const uint32_t t = (uint32_t)(t0 + lane);
            const uint4 rw = philox(t, k, d.wid, ST_STEP, a.seed);
            int my_s;
            if (a.sequential) {
                my_s = (int)t;
            } else {
                const uint4 ri = philox(((uint32_t)t0 >> 2) + (uint32_t)(lane >> 2), k, d.wid, ST_INDEX, a.seed);
                my_s = (int)index_of(word(ri, lane & 3), (uint32_t)n);
            }
            float mdx, mdy, mdz, mxi;
            if (a.proposal == QMC_CUBE) {
                mdx = step * Rng<float>::sunif(rw.x);
                mdy = step * Rng<float>::sunif(rw.y);
                mdz = step * Rng<float>::sunif(rw.z);
                mxi = Rng<float>::unif(rw.w);
            } else {
                const float two_pi = 6.283185307179586f;
                const float r0 = sqrtf(-2.f * logf(Rng<float>::unif(rw.x)));
                const float r1 = sqrtf(-2.f * logf(Rng<float>::unif(rw.z)));
                mdx = step * (r0 * cosf(two_pi * Rng<float>::unif(rw.y)));
                mdy = step * (r0 * sinf(two_pi * Rng<float>::unif(rw.y)));
                mdz = step * (r1 * cosf(two_pi * Rng<float>::unif(rw.w)));
                const uint4 rd = philox(((uint32_t)t0 >> 2) + (uint32_t)(lane >> 2), k, d.wid, ST_DICE, a.seed);
                mxi = Rng<float>::unif(word(rd, lane & 3));
            }
            mxi = logf(mxi);  // the decision is taken as 2 Delta > ln xi
            const int cnt = min(32, n - t0);
            for (int tt = 0; tt < cnt; ++tt) {
                const int s = __shfl_sync(FULL, my_s, tt);
                const float dx = __shfl_sync(FULL, mdx, tt), dy = __shfl_sync(FULL, mdy, tt),
                            dz = __shfl_sync(FULL, mdz, tt), lxi = __shfl_sync(FULL, mxi, tt);
                const int owner = s / S, ls = s - owner * S;
                float ax, ay, az;
                if (owner == (int)rank) {
                    ax = sx[ls];
                    ay = sy[ls];
                    az = sz[ls];
                } else {
                    ax = ld_cluster(map_rank(&sx[ls], (unsigned)owner));
                    ay = ld_cluster(map_rank(&sy[ls], (unsigned)owner));
                    az = ld_cluster(map_rank(&sz[ls], (unsigned)owner));
                }
                if (s == rs) {
                    ax = rx;
                    ay = ry;
                    az = rz;
                }
                const float bx = wrap(ax + dx, L), by = wrap(ay + dy, L), bz = wrap(az + dz, L);
                // partner terms over this slice, the moved atom masked (it adds zero)
                const int cs = owner == (int)rank ? ls >> 2 : -1;
                const float2 nax = make_float2(-ax, -ax), nay = make_float2(-ay, -ay), naz = make_float2(-az, -az);
                const float2 nbx = make_float2(-bx, -bx), nby = make_float2(-by, -by), nbz = make_float2(-bz, -bz);
                float2 acco = make_float2(0.f, 0.f), accn = make_float2(0.f, 0.f);
                for (int c = gtid; c < nv; c += TPW) {
                    float4 X = reinterpret_cast<const float4 *>(sx)[c];
                    float4 Y = reinterpret_cast<const float4 *>(sy)[c];
                    float4 Z = reinterpret_cast<const float4 *>(sz)[c];
                    if (c == cs) {
                        const int e = ls - 4 * c;
                        Vec<float>::set(X, e, qnan<float>());
                        Vec<float>::set(Y, e, qnan<float>());
                        Vec<float>::set(Z, e, qnan<float>());
                    }
                    const float2 xa = make_float2(X.x, X.y), xb = make_float2(X.z, X.w);
                    const float2 ya = make_float2(Y.x, Y.y), yb = make_float2(Y.z, Y.w);
                    const float2 za = make_float2(Z.x, Z.y), zb = make_float2(Z.z, Z.w);
                    P.acc5(__fadd2_rn(xa, nax), __fadd2_rn(ya, nay), __fadd2_rn(za, naz), acco);
                    P.acc5(__fadd2_rn(xa, nbx), __fadd2_rn(ya, nby), __fadd2_rn(za, nbz), accn);
                    P.acc5(__fadd2_rn(xb, nax), __fadd2_rn(yb, nay), __fadd2_rn(zb, naz), acco);
                    P.acc5(__fadd2_rn(xb, nbx), __fadd2_rn(yb, nby), __fadd2_rn(zb, nbz), accn);
                }
                float delta = 0.f;
                if (!exchange(J.c * ((accn.x + accn.y) - (acco.x + acco.y)), delta)) {
                    ok = false;
                    break;
                }
                if (delta != delta) {
                    if (gtid == 0 && rank == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_RATIO);
                    ok = false;
                    break;
                }
                if (2.f * delta > lxi) {  // Eq. (Decision)
                    if (gtid == 0 && rank == 0) lp.add(delta);
                    ++nacc;
                    if (owner == (int)rank && gtid == (ls >> 2) % TPW) {
                        sx[ls] = bx;
                        sy[ls] = by;
                        sz[ls] = bz;
                    }
                    rs = s;
                    rx = bx;
                    ry = by;
                    rz = bz;
                } else {
                    rs = -1;
                }
            }
        }
    }
    __syncthreads();
    if (ok) {  // write back (every CTA its slice; rank 0 the walker's scalars)
        for (int i = gtid; i < ns; i += TPW) {
            gx[j0 + i] = sx[i];
            gx[d.pad + j0 + i] = sy[i];
            gx[2 * (size_t)d.pad + j0 + i] = sz[i];
        }
        if (gtid == 0 && rank == 0) {
            a.accum[8 * (size_t)d.slot + 7] += (double)nacc;
            a.logpsi[d.slot] = lp.value();
            a.sweep[d.slot] = k0 + (unsigned long long)a.nsweeps;
        }
    }
    cluster_sync_all();  // no CTA leaves while another may still address its shared memory
}

cudaError_t launch_sweep_cluster(int grid, size_t smem, cudaStream_t st, const ClusterArgs &a);
cudaError_t cluster_capacity(int C, size_t smem, int *clusters);

}  // namespace qmc
