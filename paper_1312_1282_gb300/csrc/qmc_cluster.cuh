// qmc_cluster.cuh -- one walker split over a thread-block cluster: few walkers of very large N.
//
// With fewer walkers than SMs, one CTA per walker leaves most of the GPU idle (the paper's own
// 40 960-atom run used 13 walkers).  Here each walker is served by a cluster of C CTAs (C = 2, 4
// or 8, one per SM): CTA r holds atoms [rS, rS + S) of the walker in its shared memory.  Moves
// go in batches of CLUSTER_KB.  Every CTA draws the same random numbers (the counters of
// Sec. 5.2, as in the one-CTA sweep), reads the moved atoms' positions from their owners' shared
// memory through distributed shared memory (DSMEM), evaluates the partner terms of
// Eq. (JastrowUpdate) over its slice, and the C partial sums of each move are exchanged: threads
// 0 .. CLUSTER_KB-1 of every CTA store their partial into each CTA's slot and arrive on each
// CTA's mbarrier (release at cluster scope); every thread waits on its own CTA's mbarrier
// (acquire, bounded) and adds the C partials in rank order, so all CTAs take the same decisions
// (Eq. Decision).  The owners of the moved atoms write their new positions; all threads keep a
// copy of the previous batch's accepted moves for the reads that may precede those writes'
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
    unsigned long long wait_ns;  // limit of every exchange wait (global-timer nanoseconds)
    int drop_rank;               // failure test only: this CTA rank of the first walker's cluster
                                 // never stores or arrives, so its peers' waits run out (-1 normally)
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

// bounded like every other wait: the call's limit of global time (10 s unless a failure test
// shortens it), then QMC_DEVERR_TIMEOUT; once that bit is set, later waits fail at once
__device__ __forceinline__ bool mb_wait_cluster(unsigned long long *mb, unsigned parity, unsigned long long limit_ns,
                                                unsigned *err)
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
            else if (now - t0 > limit_ns)
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

// Moves per exchange.  A batch of CLUSTER_KB consecutive moves of distinct atoms is evaluated
// against the configuration at the start of the batch, as in the one-CTA batched moves: every CTA
// sums the partner terms of all the batch's moves over its slice in one pass (the batch's atoms
// masked), one exchange carries the CLUSTER_KB partial sums, and the decisions are taken in order
// with the moved atoms' own terms and the cross terms D_ik, which every warp computes (one pair
// per lane).  One cluster round trip per batch instead of one per move.
// Measured with 13 walkers of N = 40 960 (alternating runs on one GB300), ms per macroupdate:
// each move's (old, new) position in one f32x2, 8 moves per exchange 84.4, 4 moves 87.4; two
// partners per f32x2 (eight registers more per move), 4 moves 87.7, 8 moves in two passes over
// the slice 88.4; one move per exchange 131.
#ifndef QMC_CLUSTER_KB
#define QMC_CLUSTER_KB 8
#endif
constexpr int CLUSTER_KB = QMC_CLUSTER_KB;
static_assert(CLUSTER_KB == 1 || CLUSTER_KB == 2 || CLUSTER_KB == 4 || CLUSTER_KB == 8,
              "moves per exchange: 1, 2, 4 or 8");

// shared memory of one CTA: x | y | z slices (slice floats each), CLUSTER_KB x 32 warp partials,
// 2 x CLUSTER_KB x 8 exchange slots, 2 mbarriers
__host__ __device__ constexpr size_t cluster_smem(int slice)
{
    return (size_t)3 * slice * 4 + (size_t)CLUSTER_KB * 32 * 4 + (size_t)2 * CLUSTER_KB * 8 * 4 + 16;
}

template <int TPW>
__global__ void __launch_bounds__(TPW, 1) sweep_cluster_kernel(ClusterArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NW = TPW / 32;
    constexpr int K = CLUSTER_KB;
    const int gtid = threadIdx.x, lane = gtid & 31, warp = gtid >> 5;
    const unsigned rank = cluster_rank();
    const int C = a.C;
    float *sx = reinterpret_cast<float *>(smem), *sy = sx + a.slice, *sz = sy + a.slice;
    float *red = sz + a.slice;  // [K][NW]
    float *part = red + K * 32;  // [2][K][8]
    unsigned long long *mb = reinterpret_cast<unsigned long long *>(part + 2 * K * 8);
    if (gtid == 0) {
        // every exchange: threads 0 .. K-1 of each of the C CTAs arrive once
        mb_init(mb, (unsigned)(C * K));
        mb_init(mb + 1, (unsigned)(C * K));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    cluster_sync_all();  // every CTA's mbarriers exist before the first remote arrive

    const DevWalker d = a.walkers[blockIdx.x / C];
    const bool mute = blockIdx.x / C == 0 && (int)rank == a.drop_rank;  // failure test only
    const int n = d.n;
    const int S = ((n + C - 1) / C + 3) & ~3;  // this walker's slice (multiple of 4, <= a.slice)
    const int j0 = (int)rank * S;
    const int ns = max(0, min(S, n - j0));
    const int nv = S / 4;
    float *gx = reinterpret_cast<float *>(a.pos) + d.off;
    const float L = (float)d.L, step = (float)d.step;
    Jas<float, 5, true> J;
    J.init(d);

    // A failure (a wait that ran out, a non-finite ratio) never changes the control flow: every
    // thread of every CTA goes through the same exchanges and barriers to the end, where a
    // barrier vote decides the write-back.  A thread whose wait ran out skips its later waits.
    bool tmo = false;
    unsigned jx = 0;  // exchanges so far: slot set jx & 1, phase parity (jx >> 1) & 1
    // the sums over the cluster of K values per thread, identical in every CTA (rank order):
    // warp sums, then threads 0 .. K-1 each add one value over the warps, store it into every
    // CTA's slot and arrive on every CTA's mbarrier (release at cluster scope)
    auto exchange = [&](float (&v)[K]) {
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] = warp_sum(v[i]);
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < K; ++i) red[i * NW + warp] = v[i];
        __syncthreads();
        const unsigned ph = jx & 1u, par = (jx >> 1) & 1u;
        ++jx;
        if (gtid < K && !mute) {
            float s = red[gtid * NW];
#pragma unroll
            for (int w = 1; w < NW; ++w) s += red[gtid * NW + w];
            float *slot = &part[(ph * K + gtid) * 8 + rank];
            // all stores first, then the arrives: each release arrive orders every earlier store
            // of this thread, so the C stores travel together instead of one round trip each
            for (int r = 0; r < C; ++r) st_cluster(map_rank(slot, (unsigned)r), s);
            for (int r = 0; r < C; ++r) mb_arrive_remote(map_rank(&mb[ph], (unsigned)r));
        }
        if (!tmo && !mb_wait_cluster(&mb[ph], par, a.wait_ns, a.err)) tmo = true;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const float *p = &part[(ph * K + i) * 8];
            float t = p[0];
            for (int r = 1; r < C; ++r) t += p[r];
            v[i] = t;
        }
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
    bool ok;
    {
        float v[K];
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] = i == 0 ? (float)bad : 0.f;
        exchange(v);
        if (!tmo && v[0] != 0.f && gtid == 0 && rank == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_POS);
        ok = __syncthreads_and(!tmo && v[0] == 0.f) != 0;  // the same in every thread of the CTA
    }
    const bool run = ok;

    LogPsiAcc<float> lp;
    lp.set(a.logpsi[d.slot]);
    const unsigned long long k0 = a.sweep[d.slot];
    int nacc = 0;
    // the accepted moves of the previous exchange (atom, or -1, and new position): their owners'
    // writes become visible to other threads only after the next exchange
    int ps[K];
    float pbx[K], pby[K], pbz[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        ps[q] = -1;
        pbx[q] = pby[q] = pbz[q] = 0.f;
    }
    Packed5 P;
    P.init(J);
    // the block's per-lane move parameters (atom, displacement, ln xi)
    int my_s = 0;
    float mdx = 0.f, mdy = 0.f, mdz = 0.f, mxi = 0.f;

    // moves tt .. tt+KK-1 of the current block (distinct atoms) with one exchange
    auto moves = [&](auto kk_tag, int tt) {
        constexpr int KK = decltype(kk_tag)::value;
        int s[KK], own[KK], ls[KK], cs[KK];
        float ax[KK], ay[KK], az[KK], bx[KK], by[KK], bz[KK], lxi[KK];
#pragma unroll
        for (int i = 0; i < KK; ++i) {
            s[i] = __shfl_sync(FULL, my_s, tt + i);
            own[i] = s[i] / S;
            ls[i] = s[i] - own[i] * S;
            lxi[i] = __shfl_sync(FULL, mxi, tt + i);
            if (own[i] == (int)rank) {
                ax[i] = sx[ls[i]];
                ay[i] = sy[ls[i]];
                az[i] = sz[ls[i]];
            } else {
                ax[i] = ld_cluster(map_rank(&sx[ls[i]], (unsigned)own[i]));
                ay[i] = ld_cluster(map_rank(&sy[ls[i]], (unsigned)own[i]));
                az[i] = ld_cluster(map_rank(&sz[ls[i]], (unsigned)own[i]));
            }
#pragma unroll
            for (int q = 0; q < K; ++q)
                if (ps[q] == s[i]) {
                    ax[i] = pbx[q];
                    ay[i] = pby[q];
                    az[i] = pbz[q];
                }
            bx[i] = wrap(ax[i] + __shfl_sync(FULL, mdx, tt + i), L);
            by[i] = wrap(ay[i] + __shfl_sync(FULL, mdy, tt + i), L);
            bz[i] = wrap(az[i] + __shfl_sync(FULL, mdz, tt + i), L);
            cs[i] = own[i] == (int)rank ? ls[i] >> 2 : -1;
        }
        // partner terms over this slice, the batch's atoms masked (they add zero): each move holds
        // its old and new position in one f32x2 and every partner is duplicated into both lanes
        float v[K];
        {
            float2 px[KK], py[KK], pz[KK], acc2[KK];
#pragma unroll
            for (int i = 0; i < KK; ++i) {
                px[i] = make_float2(ax[i], bx[i]);
                py[i] = make_float2(ay[i], by[i]);
                pz[i] = make_float2(az[i], bz[i]);
                acc2[i] = make_float2(0.f, 0.f);
            }
            for (int c = gtid; c < nv; c += TPW) {
                float4 X = reinterpret_cast<const float4 *>(sx)[c];
                float4 Y = reinterpret_cast<const float4 *>(sy)[c];
                float4 Z = reinterpret_cast<const float4 *>(sz)[c];
#pragma unroll
                for (int i = 0; i < KK; ++i)
                    if (c == cs[i]) {
                        const int e = ls[i] - 4 * c;
                        Vec<float>::set(X, e, qnan<float>());
                        Vec<float>::set(Y, e, qnan<float>());
                        Vec<float>::set(Z, e, qnan<float>());
                    }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float xe = Vec<float>::get(X, e), ye = Vec<float>::get(Y, e), ze = Vec<float>::get(Z, e);
                    const float2 xj = make_float2(xe, xe), yj = make_float2(ye, ye), zj = make_float2(ze, ze);
#pragma unroll
                    for (int i = 0; i < KK; ++i)
                        P.acc5(__ffma2_rn(px[i], P.m1, xj), __ffma2_rn(py[i], P.m1, yj), __ffma2_rn(pz[i], P.m1, zj),
                               acc2[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < K; ++i) v[i] = i < KK ? J.c * (acc2[i].y - acc2[i].x) : 0.f;
        }
        // The batch's atoms as partners of its other moves: pair p = lane + 32 r (round r) stands
        // for move i = p / KK and atom k = p % KK; for k != i it holds
        // t_ik = u(|b_i - a_k|) - u(|a_i - a_k|) and, for i > k, the cross term
        // D_ik = u(|b_i - b_k|) - u(|a_i - b_k|) - t_ik (atom s_k accepted before move i).
        // A round covers 32 / KK moves, so eight moves take two rounds.
        constexpr int PER = KK > 1 ? 32 / KK : 1;             // moves per round
        constexpr int ROUNDS = KK > 1 ? (KK + PER - 1) / PER : 1;
        float tl[ROUNDS], dl[ROUNDS];
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            tl[r] = 0.f;
            dl[r] = 0.f;
        }
        if constexpr (KK > 1) {
#pragma unroll
            for (int r = 0; r < ROUNDS; ++r) {
                const int pidx = lane + 32 * r, li = pidx / KK, lk = pidx % KK;
                float aix = 0.f, aiy = 0.f, aiz = 0.f, bix = 0.f, biy = 0.f, biz = 0.f;
                float akx = 0.f, aky = 0.f, akz = 0.f, bkx = 0.f, bky = 0.f, bkz = 0.f;
#pragma unroll
                for (int q = 0; q < KK; ++q) {
                    if (q == li) {
                        aix = ax[q];
                        aiy = ay[q];
                        aiz = az[q];
                        bix = bx[q];
                        biy = by[q];
                        biz = bz[q];
                    }
                    if (q == lk) {
                        akx = ax[q];
                        aky = ay[q];
                        akz = az[q];
                        bkx = bx[q];
                        bky = by[q];
                        bkz = bz[q];
                    }
                }
                if (pidx < KK * KK && li != lk) {
                    tl[r] = cross5(J, aix, aiy, aiz, bix, biy, biz, akx, aky, akz);
                    if (li > lk) dl[r] = cross5(J, aix, aiy, aiz, bix, biy, biz, bkx, bky, bkz) - tl[r];
                }
                // sum of t_ik over k within each group of KK lanes
#pragma unroll
                for (int o = KK / 2; o > 0; o >>= 1) tl[r] += __shfl_xor_sync(FULL, tl[r], o);
            }
        }
        exchange(v);
        bool acc[KK];
#pragma unroll
        for (int i = 0; i < KK; ++i) {
            float delta = v[i];
            if constexpr (KK > 1) {
                const int r = i / PER, base = (i % PER) * KK;  // move i's round and first lane
                delta += __shfl_sync(FULL, tl[r], base);
#pragma unroll
                for (int k = 0; k < i; ++k) {
                    const float dik = __shfl_sync(FULL, dl[r], base + k);
                    if (acc[k]) delta += dik;
                }
            }
            if (delta != delta) {  // flagged; the move is rejected and the sweep goes on
                if (gtid == 0 && rank == 0) atomicOr(a.err, QMC_DEVERR_NONFINITE_RATIO);
                ok = false;
            }
            acc[i] = 2.f * delta > lxi[i];  // Eq. (Decision)
            if (acc[i]) {
                if (gtid == 0 && rank == 0) lp.add(delta);
                ++nacc;
            }
        }
#pragma unroll
        for (int q = 0; q < KK; ++q) {
            if (acc[q] && own[q] == (int)rank && gtid == (ls[q] >> 2) % TPW) {
                sx[ls[q]] = bx[q];
                sy[ls[q]] = by[q];
                sz[ls[q]] = bz[q];
            }
            ps[q] = acc[q] ? s[q] : -1;
            pbx[q] = bx[q];
            pby[q] = by[q];
            pbz[q] = bz[q];
        }
#pragma unroll
        for (int q = KK; q < K; ++q) ps[q] = -1;
    };

    for (int it = 0; run && it < a.nsweeps; ++it) {
        const uint32_t k = (uint32_t)(k0 + (unsigned long long)it);
        for (int t0 = 0; t0 < n; t0 += 32) {
            // random numbers of moves t0 .. t0+31, one move per lane, as in the one-CTA sweep
            const uint32_t t = (uint32_t)(t0 + lane);
            const uint4 rw = philox(t, k, d.wid, ST_STEP, a.seed);
            if (a.sequential) {
                my_s = (int)t;
            } else {
                const uint4 ri = philox(((uint32_t)t0 >> 2) + (uint32_t)(lane >> 2), k, d.wid, ST_INDEX, a.seed);
                my_s = (int)index_of(word(ri, lane & 3), (uint32_t)n);
            }
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
            int tt = 0;
            if constexpr (K > 1) {
                for (; tt + K <= cnt; tt += K) {
                    // a batch that draws an atom twice is done one move at a time: every lane of the
                    // batch's window checks that no other lane of the window drew its atom
                    const unsigned win = ((1u << K) - 1u) << tt;
                    const unsigned same = __match_any_sync(FULL, my_s) & win;
                    const bool distinct = __all_sync(FULL, !((win >> lane) & 1u) || same == (1u << lane));
                    if (distinct) {
                        moves(std::integral_constant<int, K>(), tt);
                    } else {
                        for (int i = 0; i < K; ++i) moves(std::integral_constant<int, 1>(), tt + i);
                    }
                }
            }
            for (; tt < cnt; ++tt) moves(std::integral_constant<int, 1>(), tt);
        }
    }
    // write back (every CTA its slice; rank 0 the walker's scalars) unless a thread failed
    if (__syncthreads_and(ok && !tmo)) {
        for (int i = gtid; i < ns; i += TPW) {
            gx[j0 + i] = sx[i];
            gx[d.pad + j0 + i] = sy[i];
            gx[2 * (size_t)d.pad + j0 + i] = sz[i];
        }
        if (gtid == 0 && rank == 0) {
            a.accum[QMC_ACCUM_FIELDS * (size_t)d.slot + 7] += (double)nacc;
            a.logpsi[d.slot] = lp.value();
            a.sweep[d.slot] = k0 + (unsigned long long)a.nsweeps;
        }
    }
    cluster_sync_all();  // no CTA leaves while another may still address its shared memory
}

cudaError_t launch_sweep_cluster(int grid, size_t smem, cudaStream_t st, const ClusterArgs &a);
cudaError_t cluster_capacity(int C, size_t smem, int *clusters);

}  // namespace qmc
