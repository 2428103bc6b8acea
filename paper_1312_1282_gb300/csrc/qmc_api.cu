// qmc_api.cu -- host side of libqmc: the C ABI declared in include/qmc.h.
//
// Validates arguments, resolves walker descriptors into a device table (cached by content),
// picks the launch shape (threads per walker from the autotuner or a heuristic, walkers per
// CTA), and enqueues the kernels of qmc_kernels.cuh on the caller's stream.  Nothing here
// computes physics: every step of the method runs in the kernels.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qmc_cluster.cuh"
#include "qmc_launch.h"

using namespace qmc;

namespace {

constexpr size_t MAX_SMEM = 232448;  // opt-in dynamic shared memory per CTA (227 KB)
#ifndef QMC_CHUNK_DIV
#define QMC_CHUNK_DIV 8  // persistent sweep: chunks of 1/QMC_CHUNK_DIV sweep of the largest walker (>= 128 moves)
#endif
constexpr int MAX_DEVICES = 64;
constexpr size_t MAX_PLANS = 32;

thread_local std::string g_err;
std::atomic<unsigned long long> g_launches{0};

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(QMC_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

struct DeviceState {
    unsigned *err = nullptr;
    int nsm = 0;
};

std::mutex g_mu;
DeviceState g_dev[MAX_DEVICES];

// device address of the error word of qmc_sweep_static on device `dev` (nullptr until that entry
// point has run there); defined with the static scratch at the end of this file
unsigned *static_error_word(int dev);

struct Plan {
    int device = 0;
    uint64_t key = 0;
    std::vector<qmc_walker_desc> descs;
    int sym = 1;
    int W = 0;
    DevWalker *d_walkers = nullptr;
    int *d_order = nullptr;
    uint2 *q_slots = nullptr;  // walker FIFO of the persistent sweep
    int *q_prog = nullptr;
    unsigned *q_ctr = nullptr;  // head, tail, next dominant walker (mixed sweep)
    double *part_out = nullptr;  // shares of split passes: W x parts x 8 doubles (grown on demand)
    unsigned *part_ctr = nullptr;  // [W] finished parts per walker, zero between launches
    size_t part_cap = 0;
    float *fscr = nullptr;  // drift arrays of the tiled energy pass kept in global memory, per
    size_t fscr_bytes = 0;  // batch, so that sweeps of different batches may overlap
    int maxn = 0, maxpad = 0, maxsites = 0;
    bool m5 = true;
    bool gauss_ok = false;  // descriptors validated for the Gaussian proposal's longer reach
};

struct Tuned {
    int tpw, G;  // threads per walker, walkers per CTA
};
std::list<Plan *> g_plans;                    // most recently used first
std::unordered_map<uint64_t, Tuned> g_tuned;  // shape key -> autotuned launch shape

// Failure tests only (the library's own tests run them in child processes): QMC_WAIT_LIMIT_MS
// shortens the limit of every bounded device wait (default 10 s); QMC_TEST_DROP=queue makes the
// first persistent sweep of the process never push back the first walker of its order after its
// first chunk, and QMC_TEST_DROP=cluster makes CTA rank 1 of the first walker's cluster in the
// first cluster sweep of the process never take part in an exchange -- so that waits run out and
// QMC_DEVERR_TIMEOUT is raised without any fault, and later calls run normally.
struct TestKnobs {
    unsigned long long wait_ns = 10000000000ull;
    int drop_queue = 0, drop_cluster = 0;
};
const TestKnobs &knobs()
{
    static const TestKnobs k = [] {
        TestKnobs t;
        if (const char *e = std::getenv("QMC_WAIT_LIMIT_MS")) {
            const long long ms = std::atoll(e);
            if (ms > 0 && ms < 10000) t.wait_ns = (unsigned long long)ms * 1000000ull;
        }
        if (const char *e = std::getenv("QMC_TEST_DROP")) {
            t.drop_queue = std::strcmp(e, "queue") == 0;
            t.drop_cluster = std::strcmp(e, "cluster") == 0;
        }
        return t;
    }();
    return k;
}

// the one call of the process that withholds a push or an exchange (failure tests only)
bool take_drop(int wanted)
{
    static std::atomic<int> left{1};
    return wanted && left.exchange(0) == 1;
}

uint64_t fnv(const void *p, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

int current_device(int &dev)
{
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) return fail(QMC_ERR_CUDA, "device ordinal %d out of range", dev);
    return QMC_OK;
}

// Per-device error word and SM count, created on first use (not capturable: make the first
// call of a process outside stream capture).
int device_state(int dev, DeviceState *&ds)
{
    std::lock_guard<std::mutex> lk(g_mu);
    ds = &g_dev[dev];
    if (ds->err) return QMC_OK;
    cudaError_t e = cudaDeviceGetAttribute(&ds->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    unsigned *p = nullptr;
    e = cudaMalloc(&p, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(error word)");
    e = cudaMemset(p, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(error word)");
    ds->err = p;
    return QMC_OK;
}

bool is_fin(double x) { return std::isfinite(x); }

int check_options(const qmc_options *o)
{
    if (!o) return fail(QMC_ERR_ARG, "options pointer is NULL");
    if (o->precision != QMC_FP32 && o->precision != QMC_FP64)
        return fail(QMC_ERR_ARG, "precision must be QMC_FP32 or QMC_FP64");
    if (o->proposal != QMC_CUBE && o->proposal != QMC_GAUSS)
        return fail(QMC_ERR_ARG, "proposal must be QMC_CUBE or QMC_GAUSS");
    if (o->sym != 0 && o->sym != 1) return fail(QMC_ERR_ARG, "sym must be 0 or 1");
    if (o->sequential != 0 && o->sequential != 1) return fail(QMC_ERR_ARG, "sequential must be 0 or 1");
    if (!is_fin(o->hbar2_over_m) || o->hbar2_over_m <= 0) return fail(QMC_ERR_ARG, "hbar2_over_m must be > 0");
    if (o->recompute_every < 0) return fail(QMC_ERR_ARG, "recompute_every must be >= 0");
    const int t = o->threads_per_walker;
    if (t != 0 && t != 32 && t != 64 && t != 128 && t != 256 && t != 512 && t != 1024)
        return fail(QMC_ERR_ARG, "threads_per_walker must be 0 or a power of two in 32..1024");
    const int g = o->walkers_per_cta;
    if (g < 0 || g > 8) return fail(QMC_ERR_ARG, "walkers_per_cta must be in 0..8");
    if (g > 1 && t != 0 && g * t > 256) return fail(QMC_ERR_ARG, "walkers_per_cta x threads_per_walker exceeds 256");
    if (o->reserved != 0) return fail(QMC_ERR_ARG, "options.reserved must be 0");
    return QMC_OK;
}

size_t elem_size(int precision) { return precision == QMC_FP64 ? sizeof(double) : sizeof(float); }

// shared memory of one walker group: positions (the block stride is the largest pad rounded up
// to 32), reduction scratch, and with the tiled energy pass the drift arrays
size_t smem_group(int precision, int maxpad, int tpw, bool tile = false)
{
    const int stride = stride_of(maxpad);
    return precision == QMC_FP64 ? group_smem<double>(stride, tpw, false) : group_smem<float>(stride, tpw, tile);
}

// Walkers whose coordinates do not fit one CTA's shared memory are used in place in HBM.
// QMC_GLOBAL_WALKERS=1 in the environment forces that path for every batch (used by the tests).
bool use_gmem(int precision, int maxpad, int tpw)
{
    static const bool forced = [] {
        const char *e = std::getenv("QMC_GLOBAL_WALKERS");
        return e && e[0] == '1';
    }();
    return forced || smem_group(precision, maxpad, tpw, false) > MAX_SMEM;
}

// the tiled local-energy pass (FP32) is used whenever its drift arrays fit next to G walkers
bool use_tile(int precision, int maxpad, int tpw, int G)
{
    return precision == QMC_FP32 && (size_t)G * smem_group(precision, maxpad, tpw, true) <= MAX_SMEM;
}

// CTAs of G groups that fit one SM by shared memory (228 KB, 1 KB reserved per CTA) and by
// registers (the sweep kernels' launch bounds give at most 128 registers a thread for groups of
// up to 256 threads, 512 resident threads; larger groups run one CTA)
int ctas_per_sm(size_t smem_cta, int tpw, int G)
{
    const int by_regs = tpw <= 256 ? std::max(1, 512 / (G * tpw)) : 1;
    const int by_smem = (int)(233472 / (smem_cta + 1024));
    return std::min(by_regs, by_smem);
}

// Sweep energy pass: 1 = tiled with the drift arrays in shared memory, 2 = tiled with them in
// global scratch (when the arrays in shared memory would leave fewer walkers resident per SM,
// e.g. N > 2400 with 128 threads per walker), 0 = by rows.  QMC_TILE_GLOBAL=1 in the
// environment makes every tiled sweep use global scratch (used by the tests).
int sweep_tile_mode(int precision, int maxpad, int tpw, int G)
{
    static const bool forced = [] {
        const char *e = std::getenv("QMC_TILE_GLOBAL");
        return e && e[0] == '1';
    }();
    if (precision != QMC_FP32) return 0;
    const size_t plain = smem_group(precision, maxpad, tpw, false), tiled = smem_group(precision, maxpad, tpw, true);
    if (forced) return 2;
    if ((size_t)G * tiled <= MAX_SMEM && ctas_per_sm((size_t)G * tiled, tpw, G) >= ctas_per_sm((size_t)G * plain, tpw, G))
        return 1;
    return 2;
}

int sites_of(int n)
{
    int nc = 1;
    while (4LL * nc * nc * nc < n) ++nc;
    return 4 * nc * nc * nc;
}

// Validate one descriptor into a device-table entry.  Used by resolve() (qmc_sweep and the
// passes) and by qmc_sweep_static, which has no containers to fill.
int resolve_one(const qmc_walker_desc &x, int w, const qmc_options *o, DevWalker &v)
{
    if (x.n < 2) return fail(QMC_ERR_ARG, "walker %d: n = %d < 2", w, x.n);
    if (x.pad_n < x.n || x.pad_n % 4) return fail(QMC_ERR_ARG, "walker %d: pad_n must be >= n and a multiple of 4", w);
    if (x.offset < 0 || x.offset % 4) return fail(QMC_ERR_ARG, "walker %d: offset must be >= 0 and a multiple of 4", w);
    double L = x.L;
    if (!(L > 0)) {
        if (!is_fin(x.rho) || x.rho <= 0) return fail(QMC_ERR_ARG, "walker %d: need L > 0 or rho > 0", w);
        L = std::cbrt((double)x.n / x.rho);
    }
    if (!is_fin(L)) return fail(QMC_ERR_ARG, "walker %d: non-finite box side", w);
    if (!is_fin(x.b) || x.b < 0) return fail(QMC_ERR_ARG, "walker %d: b must be finite and >= 0", w);
    if (!is_fin(x.m_exp) || x.m_exp <= 0) return fail(QMC_ERR_ARG, "walker %d: m_exp must be finite and > 0", w);
    if (!is_fin(x.step) || x.step <= 0) return fail(QMC_ERR_ARG, "walker %d: step must be finite and > 0", w);
    // a displacement must stay below one box length so one fold puts it back into the box
    const double reach = o->proposal == QMC_CUBE ? x.step : 6.8 * x.step;
    if (reach >= L) return fail(QMC_ERR_ARG, "walker %d: step too large for box side %g", w, L);
    v.n = x.n;
    v.pad = x.pad_n;
    v.off = x.offset;
    v.wid = (uint32_t)x.id;
    v.slot = w;
    v.L = L;
    v.b = x.b;
    v.m = x.m_exp;
    v.step = x.step;
    v.c = -0.5 * std::pow(x.b, x.m_exp);
    v.K = o->sym ? 2.0 * v.c * std::pow(2.0 / L, x.m_exp) : 0.0;
    return QMC_OK;
}

// Validate and resolve descriptors (host copy of the device table).
int resolve(const qmc_walker_desc *d, int W, const qmc_options *o, Plan &P, std::vector<DevWalker> &out,
            std::vector<int> &order)
{
    out.resize(W);
    P.maxn = P.maxpad = P.maxsites = 0;
    P.m5 = true;
    for (int w = 0; w < W; ++w) {
        const qmc_walker_desc &x = d[w];
        const int rc = resolve_one(x, w, o, out[w]);
        if (rc) return rc;
        P.maxn = std::max(P.maxn, x.n);
        P.maxpad = std::max(P.maxpad, x.pad_n);
        P.maxsites = std::max(P.maxsites, sites_of(x.n));
        if (x.m_exp != 5.0) P.m5 = false;
    }
    order.resize(W);
    for (int w = 0; w < W; ++w) order[w] = w;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return d[a].n > d[b].n; });
    return QMC_OK;
}

void free_plan(Plan *p)
{
    if (p->d_walkers) cudaFree(p->d_walkers);
    if (p->d_order) cudaFree(p->d_order);
    if (p->q_slots) cudaFree(p->q_slots);
    if (p->q_prog) cudaFree(p->q_prog);
    if (p->q_ctr) cudaFree(p->q_ctr);
    if (p->part_out) cudaFree(p->part_out);
    if (p->part_ctr) cudaFree(p->part_ctr);
    if (p->fscr) cudaFree(p->fscr);
    delete p;
}

// Find or build the device table of a batch.
int get_plan(const qmc_walker_desc *d, int W, const qmc_options *o, cudaStream_t st, Plan *&out)
{
    if (!d) return fail(QMC_ERR_ARG, "descriptor pointer is NULL");
    if (W <= 0) return fail(QMC_ERR_ARG, "W must be > 0");
    int dev;
    int rc = current_device(dev);
    if (rc) return rc;
    const int sym = o->sym;
    uint64_t key = fnv(d, sizeof(qmc_walker_desc) * (size_t)W);
    key = fnv(&W, sizeof W, key);
    key = fnv(&dev, sizeof dev, key);
    key = fnv(&sym, sizeof sym, key);
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_plans.begin(); it != g_plans.end(); ++it) {
        Plan *p = *it;
        if (p->key == key && p->W == W && p->device == dev && p->sym == sym &&
            std::memcmp(p->descs.data(), d, sizeof(qmc_walker_desc) * (size_t)W) == 0) {
            // the step check depends on the proposal: a batch registered by a cube-proposal call
            // is checked again, once, for the Gaussian proposal's reach
            if (o->proposal == QMC_GAUSS && !p->gauss_ok) {
                DevWalker tmp;
                for (int w = 0; w < W; ++w)
                    if ((rc = resolve_one(d[w], w, o, tmp))) return rc;
                p->gauss_ok = true;
            }
            g_plans.splice(g_plans.begin(), g_plans, it);
            out = p;
            return QMC_OK;
        }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(QMC_ERR_ARG, "a new walker batch cannot be registered during stream capture; "
                                 "call once with this batch before capturing");
    Plan *p = new Plan;
    p->device = dev;
    p->key = key;
    p->W = W;
    p->sym = sym;
    p->gauss_ok = o->proposal == QMC_GAUSS;
    p->descs.assign(d, d + W);
    std::vector<DevWalker> host;
    std::vector<int> order;
    rc = resolve(d, W, o, *p, host, order);
    if (rc) {
        delete p;
        return rc;
    }
    cudaError_t e = cudaMalloc(&p->d_walkers, sizeof(DevWalker) * (size_t)W);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_order, sizeof(int) * (size_t)W);
    if (e == cudaSuccess) e = cudaMalloc(&p->q_slots, sizeof(uint2) * (size_t)W);
    if (e == cudaSuccess) e = cudaMalloc(&p->q_prog, sizeof(int) * (size_t)W);
    if (e == cudaSuccess) e = cudaMalloc(&p->q_ctr, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_walkers, host.data(), sizeof(DevWalker) * (size_t)W, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_order, order.data(), sizeof(int) * (size_t)W, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "walker table upload");
    }
    g_plans.push_front(p);
    while (g_plans.size() > MAX_PLANS) {
        free_plan(g_plans.back());
        g_plans.pop_back();
    }
    out = p;
    return QMC_OK;
}

Variant variant_of(const Plan &P, const qmc_options *o) { return o->sym ? (P.m5 ? V5S : VGS) : VGN; }

uint64_t shape_key(int dev, const Plan &P, const qmc_options *o)
{
    int v[6] = {dev, o->precision, (int)variant_of(P, o), P.maxn, P.W, o->proposal};
    return fnv(v, sizeof v);
}

int pow2_at_least(int x)
{
    int p = 32;
    while (p < x && p < 1024) p <<= 1;
    return p;
}

// the autotuned launch shape of this batch shape, if any
bool tuned_shape(const Plan &P, const qmc_options *o, int dev, Tuned &t)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_tuned.find(shape_key(dev, P, o));
    if (it == g_tuned.end()) return false;
    t = it->second;
    return true;
}

// Threads per walker: explicit option, then the autotuned choice, then a heuristic aiming at
// ~16 resident warps per SM while every thread keeps at least one 4-atom partner chunk.
int choose_tpw(const Plan &P, const qmc_options *o, int dev, int nsm)
{
    if (o->threads_per_walker) return o->threads_per_walker;
    Tuned tu;
    if (tuned_shape(P, o, dev, tu)) return tu.tpw;
    const int chunks = (P.maxn + 3) / 4;
    int t = pow2_at_least((int)std::ceil(512.0 * nsm / P.W));
    t = std::min(t, pow2_at_least(chunks));
    return std::max(32, std::min(t, 1024));
}

// the batch's drift scratch of the tiled energy pass, at least `need` bytes (not under capture)
int drift_scratch(Plan &P, size_t need, float **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (P.fscr_bytes < need) {
        if (P.fscr) cudaFree(P.fscr);
        P.fscr = nullptr;
        P.fscr_bytes = 0;
        cudaError_t e = cudaMalloc(&P.fscr, need);
        if (e != cudaSuccess) return cuda_fail(e, "drift scratch");
        P.fscr_bytes = need;
    }
    *out = P.fscr;
    return QMC_OK;
}

// Walkers per CTA: 1 for walkers in HBM or groups of more than 256 threads; else the explicit
// option (refused if G groups do not fit one CTA), then the autotuned choice for this threads
// per walker, then a heuristic: one, unless the batch has so many small walkers that the
// 32-CTA-per-SM limit would cap residency.  G x tpw <= 256 and G groups fit one CTA's shared
// memory (with the drift arrays when a tiled energy pass would keep them there).
int choose_groups(const Plan &P, const qmc_options *o, int tpw, int dev, int nsm, int &G)
{
    const int precision = o->precision;
    G = 1;
    if (use_gmem(precision, P.maxpad, tpw) || tpw > 256) return QMC_OK;
    const size_t per = smem_group(precision, P.maxpad, tpw, use_tile(precision, P.maxpad, tpw, 1));
    const size_t plain = smem_group(precision, P.maxpad, tpw, false);
    if (o->walkers_per_cta) {
        G = o->walkers_per_cta;
        if (G > 1 && ((size_t)G * plain > MAX_SMEM || G * tpw > 256))
            return fail(QMC_ERR_ARG, "walkers_per_cta = %d groups of %d threads do not fit one CTA", G, tpw);
        return QMC_OK;
    }
    Tuned t;
    if (tuned_shape(P, o, dev, t) && t.tpw == tpw) {
        G = t.G;
    } else if (tpw <= 128 && P.W > 24 * nsm) {
        G = std::min(256 / tpw, (P.W + 24 * nsm - 1) / (24 * nsm));
    }
    while (G > 1 && ((size_t)G * per > MAX_SMEM || G * tpw > 256)) --G;
    G = std::max(1, std::min(G, 8));
    return QMC_OK;
}

// shared memory a launch needs per group and the layout flags that go with it
struct Shape {
    int stride, tile, gmem;
    size_t smem;  // per group
};
Shape shape_of(const Plan &P, int precision, int tpw, int G, bool energy_pass, bool sweep = false)
{
    Shape sh;
    sh.gmem = use_gmem(precision, P.maxpad, tpw) ? 1 : 0;
    sh.stride = sh.gmem ? 0 : stride_of(P.maxpad);
    if (sh.gmem || !energy_pass)
        sh.tile = 0;
    else if (sweep)
        sh.tile = sweep_tile_mode(precision, P.maxpad, tpw, G);
    else
        sh.tile = use_tile(precision, P.maxpad, tpw, G) ? 1 : 0;
    sh.smem = sh.gmem ? smem_group(precision, 0, tpw, false) : smem_group(precision, P.maxpad, tpw, sh.tile == 1);
    return sh;
}

int check_ptr(const void *p, const char *name, size_t align)
{
    if (!p) return fail(QMC_ERR_ARG, "%s is NULL", name);
    if ((uintptr_t)p % align) return fail(QMC_ERR_ARG, "%s must be %zu-byte aligned", name, align);
    return QMC_OK;
}

cudaError_t sweep_occupancy(int precision, int tpw, Variant v, int block, size_t smem, int *ctas)
{
    if (precision == QMC_FP64)
        return tpw <= 128 ? occupancy_sweep_f64_small(tpw, v, block, smem, ctas)
                          : occupancy_sweep_f64_big(tpw, v, block, smem, ctas);
    return tpw <= 128 ? occupancy_sweep_f32_small(tpw, v, block, smem, ctas)
                      : occupancy_sweep_f32_big(tpw, v, block, smem, ctas);
}

cudaError_t launch_sweep(int precision, int tpw, Variant v, int grid, int block, size_t smem, cudaStream_t st,
                         const SweepArgs &a)
{
    if (precision == QMC_FP64)
        return tpw <= 128 ? launch_sweep_f64_small(tpw, v, grid, block, smem, st, a)
                          : launch_sweep_f64_big(tpw, v, grid, block, smem, st, a);
    return tpw <= 128 ? launch_sweep_f32_small(tpw, v, grid, block, smem, st, a)
                      : launch_sweep_f32_big(tpw, v, grid, block, smem, st, a);
}

struct Prep {
    Plan *plan = nullptr;
    DeviceState *ds = nullptr;
    int dev = 0;
};

// Host-only checks come first, so argument errors are reported without touching the device.
int prepare(const qmc_walker_desc *d, int W, const qmc_options *o, cudaStream_t st, Prep &p)
{
    int rc = check_options(o);
    if (rc) return rc;
    if (!d) return fail(QMC_ERR_ARG, "descriptor pointer is NULL");
    if (W <= 0) return fail(QMC_ERR_ARG, "W must be > 0");
    if ((rc = current_device(p.dev))) return rc;
    if ((rc = device_state(p.dev, p.ds))) return rc;
    return get_plan(d, W, o, st, p.plan);
}

// Uneven batch with dominant walkers (n >= whole_n): the mixed kernel runs those on whole CTAs of
// MIXED_TPWB threads, one whole call each, and the other walkers on groups of tpw threads from
// the queue.  Returns -1 (nothing launched) when the batch does not suit it: FP32 exponent-5
// symmetrised walkers in shared memory, tpw 64 or 128, both phases within one CTA's shared memory.
// QMC_MIXED=0 in the environment turns it off.
int mixed_sweep(const qmc_walker_desc *d, int W, const qmc_options *o, const Plan &P, Prep &p, int tpw, Variant v,
                int whole_n, int nsweeps, const SweepArgs &a, cudaStream_t st)
{
    static const bool off = [] {
        const char *e = std::getenv("QMC_MIXED");
        return e && e[0] == '0';
    }();
    if (off || o->precision != QMC_FP32 || v != V5S || (tpw != 64 && tpw != 128)) return -1;
    int n_big = 0, maxpad_b = 0, maxpad_s = 0, maxn_s = 0;
    for (int w = 0; w < W; ++w) {
        if (d[w].n >= whole_n) {
            ++n_big;
            maxpad_b = std::max(maxpad_b, (int)d[w].pad_n);
        } else {
            maxpad_s = std::max(maxpad_s, (int)d[w].pad_n);
            maxn_s = std::max(maxn_s, (int)d[w].n);
        }
    }
    if (n_big == 0 || n_big == W) return -1;
    if (use_gmem(QMC_FP32, maxpad_b, MIXED_TPWB) || use_gmem(QMC_FP32, maxpad_s, tpw)) return -1;
    const int Gs = MIXED_TPWB / tpw;
    const int tile_b = sweep_tile_mode(QMC_FP32, maxpad_b, MIXED_TPWB, 1);
    const int tile_s = sweep_tile_mode(QMC_FP32, maxpad_s, tpw, Gs);
    const size_t smem_b = smem_group(QMC_FP32, maxpad_b, MIXED_TPWB, tile_b == 1);
    const size_t smem_s = (size_t)Gs * smem_group(QMC_FP32, maxpad_s, tpw, tile_s == 1);
    const size_t smem = std::max(smem_b, smem_s);
    if (smem > MAX_SMEM) return -1;
    static std::mutex mu;
    static std::unordered_map<uint64_t, int> cache;
    int key_v[3] = {p.dev, tpw, (int)smem};
    const uint64_t key = fnv(key_v, sizeof key_v);
    int ctas = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) ctas = it->second;
    }
    cudaError_t e;
    if (ctas == 0) {
        e = occupancy_sweep_mixed(tpw, smem, &ctas);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = ctas;
    }
    if (ctas < 1) return -1;
    const int grid = ctas * p.ds->nsm;
    const long long chunk = std::max(128, ((maxn_s + QMC_CHUNK_DIV - 1) / QMC_CHUNK_DIV + 31) / 32 * 32);
    long long total = 0;
    for (int w = 0; w < W; ++w)
        if (d[w].n < whole_n) total += ((long long)nsweeps * d[w].n + chunk - 1) / chunk;
    if (total >= (1ll << 31)) return -1;

    SweepArgs big = a, small = a;
    big.order = P.d_order;  // longest first: the dominant walkers lead the order
    big.W = n_big;
    big.G = 1;
    big.stride = stride_of(maxpad_b);
    big.tile = tile_b;
    big.gmem = 0;
    big.dynamic = 0;
    small.order = P.d_order + n_big;
    small.W = W - n_big;
    small.G = Gs;
    small.stride = stride_of(maxpad_s);
    small.tile = tile_s;
    small.gmem = 0;
    small.dynamic = 1;
    small.chunk_moves = (int)chunk;
    small.q_total = (unsigned)total;
    small.q_head = P.q_ctr;
    small.q_tail = P.q_ctr + 1;
    small.q_slots = P.q_slots;
    small.q_prog = P.q_prog;
    small.drop_push = take_drop(knobs().drop_queue) ? 1 : 0;
    big.fscr = small.fscr = nullptr;
    const size_t fb = tile_b == 2 ? (size_t)grid * 3 * big.stride : 0;
    const size_t fs = tile_s == 2 ? (size_t)grid * Gs * 3 * small.stride : 0;
    if (fb + fs > 0) {
        float *f = nullptr;
        int rc = drift_scratch(*p.plan, (fb + fs) * sizeof(float), &f);
        if (rc) return rc;
        if (fb) big.fscr = f;
        if (fs) small.fscr = f + fb;
    }
    e = launch_queue_init(small.order, small.W, P.q_slots, P.q_prog, P.q_ctr, P.q_ctr + 1, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.q_ctr + 2, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e, "walker queue init");
    g_launches.fetch_add(1);
    e = launch_sweep_mixed(tpw, grid, smem, st, small, big, P.q_ctr + 2);
    if (e != cudaSuccess) return cuda_fail(e, "mixed sweep launch");
    g_launches.fetch_add(1);
    return QMC_OK;
}

// Few walkers of very large N (at most one per two SMs, N >= 4096): each walker runs on a
// thread-block cluster of C CTAs, one per SM (qmc_cluster.cuh).  FP32 exponent-5 symmetrised
// walkers, calls without energy samples or ln psi recomputes.  Returns -1 (nothing launched) when
// the batch does not suit it.  QMC_CLUSTER=0 turns it off; QMC_CLUSTER=1 uses it for every
// batch that suits it apart from the size rule (used by the tests).
int cluster_sweep(const qmc_walker_desc *d, int W, const qmc_options *o, const Plan &P, Prep &p, void *pos,
                  double *logpsi, uint64_t *sweep, uint64_t seed, int nsweeps, int energy_every, double *accum,
                  cudaStream_t st)
{
    static const int mode = [] {
        const char *e = std::getenv("QMC_CLUSTER");
        return e ? (e[0] == '0' ? 0 : (e[0] == '1' ? 2 : 1)) : 1;
    }();
    if (mode == 0 || o->precision != QMC_FP32 || variant_of(P, o) != V5S || energy_every != 0 ||
        o->recompute_every != 0)
        return -1;
    const int nsm = p.ds->nsm;
    if (mode == 1 && (2 * W > nsm || P.maxn < 4096)) return -1;
    int C = CLUSTER_MAX;
    while (C > 2 && W * C > nsm) C /= 2;
    int slice = ((P.maxn + C - 1) / C + 3) & ~3;
    while (cluster_smem(slice) > MAX_SMEM && C < CLUSTER_MAX) {
        C *= 2;
        slice = ((P.maxn + C - 1) / C + 3) & ~3;
    }
    const size_t smem = cluster_smem(slice);
    if (smem > MAX_SMEM) return -1;
    int clusters = 0;
    cudaError_t e = cluster_capacity(C, smem, &clusters);
    if (e != cudaSuccess) return cuda_fail(e, "cluster occupancy query");
    if (clusters < 1) return -1;
    ClusterArgs a;
    a.walkers = P.d_walkers;
    a.W = W;
    a.C = C;
    a.slice = slice;
    a.pos = pos;
    a.logpsi = logpsi;
    a.sweep = reinterpret_cast<unsigned long long *>(sweep);
    a.accum = accum;
    a.seed = seed;
    a.nsweeps = nsweeps;
    a.proposal = o->proposal;
    a.sequential = o->sequential;
    a.err = p.ds->err;
    a.wait_ns = knobs().wait_ns;
    a.drop_rank = take_drop(knobs().drop_cluster) ? 1 : -1;
    e = launch_sweep_cluster(W * C, smem, st, a);
    if (e != cudaSuccess) return cuda_fail(e, "cluster sweep launch");
    g_launches.fetch_add(1);
    return QMC_OK;
}

int sweep_impl(const qmc_walker_desc *d, int W, const qmc_options *o, void *pos, double *logpsi, uint64_t *sweep,
               uint64_t seed, int nsweeps, int energy_every, double *accum, cudaStream_t st, int tpw_force,
               int g_force = 0)
{
    int rc;
    if ((rc = check_ptr(pos, "pos", 16)) || (rc = check_ptr(logpsi, "logpsi", 8)) ||
        (rc = check_ptr(sweep, "sweep", 8)) || (rc = check_ptr(accum, "accum", 8)))
        return rc;
    if (nsweeps < 0) return fail(QMC_ERR_ARG, "nsweeps must be >= 0");
    if (energy_every < 0) return fail(QMC_ERR_ARG, "energy_every must be >= 0");
    Prep p;
    if ((rc = prepare(d, W, o, st, p))) return rc;
    const Plan &P = *p.plan;
    const int tpw = tpw_force ? tpw_force : choose_tpw(P, o, p.dev, p.ds->nsm);
    if (nsweeps == 0) return QMC_OK;
    if (!tpw_force) {
        const int crc = cluster_sweep(d, W, o, P, p, pos, logpsi, sweep, seed, nsweeps, energy_every, accum, st);
        if (crc != -1) return crc;
    }
    int G = 1;
    if (g_force) {
        G = g_force;
    } else if ((rc = choose_groups(P, o, tpw, p.dev, p.ds->nsm, G))) {
        return rc;
    }
    const Shape sh = shape_of(P, o->precision, tpw, G, true, true);
    SweepArgs a;
    a.walkers = P.d_walkers;
    a.order = P.d_order;
    a.W = W;
    a.G = G;
    a.stride = sh.stride;
    a.tile = sh.tile;
    a.gmem = sh.gmem;
    a.pos = pos;
    a.logpsi = logpsi;
    a.sweep = reinterpret_cast<unsigned long long *>(sweep);
    a.accum = accum;
    a.seed = seed;
    a.nsweeps = nsweeps;
    a.energy_every = energy_every;
    a.recompute_every = o->recompute_every;
    a.proposal = o->proposal;
    a.sequential = o->sequential;
    a.h2m = o->hbar2_over_m;
    a.err = p.ds->err;
    a.dynamic = 0;
    a.chunk_moves = 0;
    a.q_total = 0;
    a.q_head = a.q_tail = nullptr;
    a.q_slots = nullptr;
    a.q_prog = nullptr;
    a.wait_ns = knobs().wait_ns;
    a.drop_push = 0;
    int grid = (W + G - 1) / G;
    const size_t smem = (size_t)G * sh.smem;
    const Variant v = variant_of(P, o);
    cudaError_t e;
    if (W > p.ds->nsm) {
        // persistent mode: every resident CTA slot takes ready walkers in chunks of about an eighth
        // of a sweep of the largest walker, so that SMs stay evenly loaded when W is not a multiple
        // of the SM count
        // resident CTAs per SM, cached so that calls under stream capture make no query
        static std::mutex occ_mu;
        static std::unordered_map<uint64_t, int> occ_cache;
        int key_v[6] = {p.dev, o->precision, tpw, (int)v, G * tpw, (int)smem};
        const uint64_t okey = fnv(key_v, sizeof key_v);
        int ctas = 0;
        {
            std::lock_guard<std::mutex> lk(occ_mu);
            auto it = occ_cache.find(okey);
            if (it != occ_cache.end()) ctas = it->second;
        }
        if (ctas == 0) {
            e = sweep_occupancy(o->precision, tpw, v, G * tpw, smem, &ctas);
            if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
            std::lock_guard<std::mutex> lk(occ_mu);
            occ_cache[okey] = ctas;
        }
        const long long chunk = std::max(128, ((P.maxn + QMC_CHUNK_DIV - 1) / QMC_CHUNK_DIV + 31) / 32 * 32);
        // Dominant walkers: pair work alone at least the mean load of a resident group and four
        // times the batch mean.  Their sequential moves bound the call, so waiting in the queue
        // between chunks would lengthen that bound: the mixed kernel runs each for the whole call
        // (in a batch of equal walkers nobody qualifies)
        const long long slots = (long long)std::max(ctas, 1) * p.ds->nsm * G;
        double work_sum = 0;
        for (int w = 0; w < W; ++w) work_sum += (double)d[w].n * d[w].n;
        int whole_n = INT_MAX;
        for (int w = 0; w < W; ++w) {
            const double wk = (double)d[w].n * d[w].n;
            if (wk >= work_sum / (double)slots && wk >= 4.0 * work_sum / W) whole_n = std::min(whole_n, d[w].n);
        }
        long long total = 0;
        for (int w = 0; w < W; ++w) total += ((long long)nsweeps * d[w].n + chunk - 1) / chunk;
        if (whole_n < INT_MAX && ctas > 0) {
            const int mrc = mixed_sweep(d, W, o, P, p, tpw, v, whole_n, nsweeps, a, st);
            if (mrc != -1) return mrc;  // launched (or failed); -1: the batch does not suit it
        }
        // a batch that fills every SM with the same number of resident groups gains nothing from
        // the queue: each group keeps its walker for the whole call
        const bool even = W % p.ds->nsm == 0 && (long long)W <= (long long)ctas * p.ds->nsm * G;
        if (ctas > 0 && !even && total < (1ll << 31)) {
            a.dynamic = 1;
            a.chunk_moves = (int)chunk;
            a.q_total = (unsigned)total;
            a.q_head = P.q_ctr;
            a.q_tail = P.q_ctr + 1;
            a.q_slots = P.q_slots;
            a.q_prog = P.q_prog;
            a.drop_push = take_drop(knobs().drop_queue) ? 1 : 0;
            grid = ctas * p.ds->nsm;
            e = launch_queue_init(P.d_order, W, P.q_slots, P.q_prog, P.q_ctr, P.q_ctr + 1, st);
            if (e != cudaSuccess) return cuda_fail(e, "walker queue init");
            g_launches.fetch_add(1);
        }
    }
    a.fscr = nullptr;
    if (a.tile == 2) {  // drift scratch of every resident group, grown on demand (not under capture)
        if ((rc = drift_scratch(*p.plan, (size_t)grid * G * 3 * sh.stride * sizeof(float), &a.fscr))) return rc;
    }
    e = launch_sweep(o->precision, tpw, v, grid, G * tpw, smem, st, a);
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    g_launches.fetch_add(1);
    return QMC_OK;
}

// CTAs per walker of a row-wise pass: with fewer walkers than SMs, a walker's rows are split over
// about SMs / W CTAs (at least one block of tpw rows each), so that few large walkers use the GPU.
int choose_parts(const Plan &P, int W, int nsm, int tpw)
{
    if (W >= nsm) return 1;
    const int by_rows = (P.maxn + tpw - 1) / tpw;
    return std::max(1, std::min({nsm / W, by_rows, 64}));
}

// the plan's scratch of split passes, at least W x parts x 8 doubles, and its zeroed counters
// (allocated on first use: not under stream capture)
int pass_scratch(Plan &P, int parts, cudaStream_t st, double **out, unsigned **ctr)
{
    std::lock_guard<std::mutex> lk(g_mu);
    const size_t need = (size_t)P.W * parts * 8;
    if (P.part_cap < need) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            return fail(QMC_ERR_ARG, "a split pass of this batch needs its scratch allocated before stream capture; "
                                     "call it once outside capture");
        if (P.part_out) cudaFree(P.part_out);
        P.part_out = nullptr;
        P.part_cap = 0;
        cudaError_t e = cudaMalloc(&P.part_out, need * sizeof(double));
        if (e == cudaSuccess && !P.part_ctr) {
            e = cudaMalloc(&P.part_ctr, sizeof(unsigned) * (size_t)P.W);
            if (e == cudaSuccess) e = cudaMemsetAsync(P.part_ctr, 0, sizeof(unsigned) * (size_t)P.W, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "split-pass scratch");
        P.part_cap = need;
    }
    *out = P.part_out;
    *ctr = P.part_ctr;
    return QMC_OK;
}

int pass_impl(const qmc_walker_desc *d, int W, const qmc_options *o, const void *pos, double *out, int kind,
              const int32_t *s, const double *delta, int M, cudaStream_t st)
{
    int rc;
    if ((rc = check_ptr(pos, "pos", 16)) || (rc = check_ptr(out, "out", 8))) return rc;
    Prep p;
    if ((rc = prepare(d, W, o, st, p))) return rc;
    const Plan &P = *p.plan;
    const int tpw = kind == 2 ? TRIAL_TPW : PASS_TPW;
    const Shape sh = shape_of(P, o->precision, tpw, 1, kind == 0);
    PassArgs a;
    a.walkers = P.d_walkers;
    a.W = W;
    a.stride = sh.stride;
    a.tile = sh.tile;
    a.gmem = sh.gmem;
    a.pos = pos;
    a.out = out;
    a.h2m = o->hbar2_over_m;
    a.s = s;
    a.delta = delta;
    a.M = M;
    a.err = p.ds->err;
    // row-wise passes of few walkers are split over several CTAs per walker (the tiled energy
    // pass and the trial ratios are not)
    a.parts = (kind == 2 || (kind == 0 && sh.tile)) ? 1 : choose_parts(P, W, p.ds->nsm, tpw);
    a.part_out = nullptr;
    a.part_ctr = nullptr;
    if (a.parts > 1 && (rc = pass_scratch(*p.plan, a.parts, st, &a.part_out, &a.part_ctr))) return rc;
    const size_t smem = sh.smem;
    cudaError_t e = launch_pass(o->precision, variant_of(P, o), kind, W * a.parts, smem, st, a);
    if (e != cudaSuccess) return cuda_fail(e, "pass launch");
    g_launches.fetch_add(1);
    return QMC_OK;
}

}  // namespace

extern "C" {

int qmc_init_walkers(const qmc_walker_desc *d, int W, uint64_t seed, double jitter_sigma, const qmc_options *opt,
                     void *pos, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if ((rc = check_ptr(pos, "pos", 16))) return rc;
    if (!is_fin(jitter_sigma) || jitter_sigma < 0) return fail(QMC_ERR_ARG, "jitter_sigma must be finite and >= 0");
    Prep p;
    if ((rc = prepare(d, W, opt, st, p))) return rc;
    const size_t smem = sizeof(int) * (size_t)p.plan->maxsites;
    if (smem > MAX_SMEM) return fail(QMC_ERR_CAPACITY, "too many lattice sites for the start configuration");
    cudaError_t e = launch_init(opt->precision, W, smem, st, p.plan->d_walkers, seed, jitter_sigma, pos);
    if (e != cudaSuccess) return cuda_fail(e, "init launch");
    g_launches.fetch_add(1);
    return QMC_OK;
}

int qmc_sweep(const qmc_walker_desc *d, int W, const qmc_options *opt, void *pos, double *logpsi, uint64_t *sweep,
              uint64_t seed, int nsweeps, int energy_every, double *accum, void *stream)
{
    return sweep_impl(d, W, opt, pos, logpsi, sweep, seed, nsweeps, energy_every, accum, (cudaStream_t)stream, 0);
}

int qmc_local_energy(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos, double *out,
                     void *stream)
{
    return pass_impl(d, W, opt, pos, out, 0, nullptr, nullptr, 0, (cudaStream_t)stream);
}

int qmc_log_psi(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos, double *out, void *stream)
{
    return pass_impl(d, W, opt, pos, out, 1, nullptr, nullptr, 0, (cudaStream_t)stream);
}

int qmc_trial_delta(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos, const int32_t *s,
                    const double *delta, int M, double *out, void *stream)
{
    if (M <= 0) return fail(QMC_ERR_ARG, "M must be > 0");
    if (!s || !delta) return fail(QMC_ERR_ARG, "s and delta must not be NULL");
    return pass_impl(d, W, opt, pos, out, 2, s, delta, M, (cudaStream_t)stream);
}

int qmc_energy_grad(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos, double *out,
                    void *stream)
{
    return pass_impl(d, W, opt, pos, out, 3, nullptr, nullptr, 0, (cudaStream_t)stream);
}

int qmc_pair_hist(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos, int nbins, double rmax,
                  uint64_t *hist, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if ((rc = check_ptr(pos, "pos", 16)) || (rc = check_ptr(hist, "hist", 8))) return rc;
    if (nbins < 1 || nbins > 16384) return fail(QMC_ERR_ARG, "nbins must be in 1..16384");
    if (!is_fin(rmax) || rmax <= 0) return fail(QMC_ERR_ARG, "rmax must be finite and > 0");
    Prep p;
    if ((rc = prepare(d, W, opt, st, p))) return rc;
    const Plan &P = *p.plan;
    const Shape sh = shape_of(P, opt->precision, PASS_TPW, 1, false);
    PassArgs a;
    a.walkers = P.d_walkers;
    a.W = W;
    a.stride = sh.stride;
    a.tile = 0;
    a.gmem = sh.gmem;
    a.pos = pos;
    a.out = nullptr;
    a.h2m = opt->hbar2_over_m;
    a.s = nullptr;
    a.delta = nullptr;
    a.M = 0;
    a.err = p.ds->err;
    a.parts = choose_parts(P, W, p.ds->nsm, PASS_TPW);  // counts of the parts add with atomics
    a.part_out = nullptr;
    a.part_ctr = nullptr;
    const size_t smem = sh.smem + sizeof(unsigned) * (size_t)nbins;
    if (smem > MAX_SMEM) return fail(QMC_ERR_CAPACITY, "histogram does not fit shared memory next to the walker");
    cudaError_t e = launch_hist(opt->precision, W * a.parts, smem, st, a, nbins, rmax,
                                reinterpret_cast<unsigned long long *>(hist));
    if (e != cudaSuccess) return cuda_fail(e, "histogram launch");
    g_launches.fetch_add(1);
    return QMC_OK;
}

int qmc_autotune(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos, void *stream,
                 int *tpw_out, int *groups_out)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if ((rc = check_ptr(pos, "pos", 16))) return rc;
    Prep p;
    if ((rc = prepare(d, W, opt, st, p))) return rc;
    const Plan &P = *p.plan;
    size_t elems = 0;
    for (int w = 0; w < W; ++w) elems = std::max(elems, (size_t)(d[w].offset + 3 * (int64_t)d[w].pad_n));
    const size_t bytes = elems * elem_size(opt->precision);
    void *scratch = nullptr;
    double *lp = nullptr, *acc = nullptr;
    uint64_t *sw = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Tuned best{0, 0};
    float best_ms = 0;
    const size_t acc_bytes = sizeof(double) * QMC_ACCUM_FIELDS * (size_t)W;
    cudaError_t e = cudaMalloc(&scratch, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&lp, sizeof(double) * W);
    if (e == cudaSuccess) e = cudaMalloc(&acc, acc_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sw, sizeof(uint64_t) * W);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(lp, 0, sizeof(double) * W, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, acc_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sw, 0, sizeof(uint64_t) * W, st);
    // the search space: threads per walker up to one thread per 4-atom partner chunk, walkers per
    // CTA with at most 256 threads and G groups within one CTA's shared memory (explicit options
    // narrow it)
    const int chunk_cap = pow2_at_least((P.maxn + 3) / 4);
    const size_t plain_cap = MAX_SMEM;
    for (int tpw = 32; e == cudaSuccess && rc == QMC_OK && tpw <= 1024; tpw <<= 1) {
        if (tpw > chunk_cap) break;
        if (opt->threads_per_walker && tpw != opt->threads_per_walker) continue;
        const bool gm = use_gmem(opt->precision, P.maxpad, tpw);
        for (int G = 1; G <= 8; G <<= 1) {
            if (opt->walkers_per_cta && G != opt->walkers_per_cta) continue;
            if (G > 1 && (gm || G * tpw > 256 || (size_t)G * smem_group(opt->precision, P.maxpad, tpw, false) > plain_cap))
                break;
            if (G > 1 && (W + G - 1) / G < p.ds->nsm / 2) break;  // too few CTAs to fill the GPU
            e = cudaMemcpyAsync(scratch, pos, bytes, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) break;
            rc = sweep_impl(d, W, opt, scratch, lp, sw, 0x7E57ull, 1, 0, acc, st, tpw, G);  // warm-up
            if (rc) break;
            e = cudaEventRecord(e0, st);
            if (e != cudaSuccess) break;
            rc = sweep_impl(d, W, opt, scratch, lp, sw, 0x7E57ull, 2, 0, acc, st, tpw, G);
            if (rc) break;
            e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (best.tpw == 0 || ms < best_ms)) {
                best = Tuned{tpw, G};
                best_ms = ms;
            }
            if (e != cudaSuccess) break;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(scratch);
    cudaFree(lp);
    cudaFree(acc);
    cudaFree(sw);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    if (best.tpw == 0) return fail(QMC_ERR_CAPACITY, "no admissible launch shape");
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_tuned[shape_key(p.dev, P, opt)] = best;
    }
    if (tpw_out) *tpw_out = best.tpw;
    if (groups_out) *groups_out = best.G;
    return QMC_OK;
}

int qmc_capacity(int precision)
{
    if (precision != QMC_FP32 && precision != QMC_FP64) return fail(QMC_ERR_ARG, "bad precision");
    const size_t es = elem_size(precision);
    const size_t red = smem_group(precision, 0, 1024);
    return (int)(((MAX_SMEM - red) / (3 * es)) / 32 * 32);
}

int qmc_status(void *stream, int timeout_ms, uint32_t *bits)
{
    cudaStream_t st = (cudaStream_t)stream;
    int dev;
    int rc = current_device(dev);
    if (rc) return rc;
    DeviceState *ds;
    if ((rc = device_state(dev, ds))) return rc;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaStreamQuery(st);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_fail(q, "cudaStreamQuery");
        if (timeout_ms > 0 && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
            return fail(QMC_ERR_TIMEOUT, "stream not finished after %d ms", timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    unsigned h = 0, hs = 0;
    unsigned *sw = static_error_word(dev);
    cudaError_t e = cudaMemcpyAsync(&h, ds->err, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ds->err, 0, sizeof(unsigned), st);
    if (e == cudaSuccess && sw) e = cudaMemcpyAsync(&hs, sw, sizeof hs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && sw) e = cudaMemsetAsync(sw, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    h |= hs;
    if (bits) *bits = h;
    if (h)
        return fail(QMC_ERR_DEVICE, "kernel flagged %s%s%s%s", (h & QMC_DEVERR_NONFINITE_POS) ? "[bad coordinate]" : "",
                    (h & QMC_DEVERR_NONFINITE_RATIO) ? "[non-finite ratio]" : "",
                    (h & QMC_DEVERR_BAD_INDEX) ? "[atom index out of range]" : "",
                    (h & QMC_DEVERR_TIMEOUT) ? "[a bounded device wait timed out]" : "");
    return QMC_OK;
}

int qmc_probe_rates(int blocks_per_sm, int threads, int iters, double *out, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (!out) return fail(QMC_ERR_ARG, "out is NULL");
    if (blocks_per_sm < 1 || blocks_per_sm > 32) return fail(QMC_ERR_ARG, "blocks_per_sm must be in 1..32");
    if (threads < 32 || threads > 1024 || threads % 32) return fail(QMC_ERR_ARG, "threads must be a multiple of 32 in 32..1024");
    if (iters < 1 || iters > 1000000) return fail(QMC_ERR_ARG, "iters must be in 1..1000000");
    int dev, rc;
    if ((rc = current_device(dev))) return rc;
    DeviceState *ds;
    if ((rc = device_state(dev, ds))) return rc;
    const int nsm = ds->nsm;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(float) * (size_t)blocks_per_sm * nsm * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double res[QMC_PROBE_COUNT] = {};
    for (int kind = 0; e == cudaSuccess && kind < QMC_PROBE_COUNT; ++kind) {
        // the pair probe keeps the sweep's register budget: at most 512 threads per CTA
        const int thr = kind == QMC_PROBE_PAIR ? std::min(threads, 512) : threads;
        int resident = 0;
        e = probe_occupancy(kind, thr, &resident);
        if (e != cudaSuccess) break;
        resident = std::min(resident, blocks_per_sm);
        if (resident < 1) {
            e = cudaErrorInvalidConfiguration;
            break;
        }
        const int grid = resident * nsm;  // every CTA resident at once, the same number on every SM
        e = launch_probe(kind, grid, thr, std::max(1, iters / 16), sink, st);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = launch_probe(kind, grid, thr, iters, sink, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        g_launches.fetch_add(2);
        res[kind] = (double)grid * thr * iters * probe_ops_per_thread_iter(kind) / (ms * 1e-3) / nsm;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "probe");
    for (int k = 0; k < QMC_PROBE_COUNT; ++k) out[k] = res[k];
    return QMC_OK;
}

uint64_t qmc_launch_count(void) { return g_launches.load(); }

const char *qmc_last_error(void) { return g_err.c_str(); }

int qmc_version(void) { return QMC_VERSION; }

void qmc_shutdown(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (Plan *p : g_plans) free_plan(p);
    g_plans.clear();
    g_tuned.clear();
    for (auto &ds : g_dev) {
        if (ds.err) cudaFree(ds.err);
        ds.err = nullptr;
        ds.nsm = 0;
    }
}

}  // extern "C"

// ----------------------------------------------------------------------------------------------
// qmc_sweep_static: the same sweep with every piece of device scratch in one fixed array of
// the library image, for callers that cannot allocate device memory (see include/qmc.h).
// Layout of the array: DevWalker table [QMC_STATIC_MAX_WALKERS] | order [QMC_STATIC_MAX_WALKERS]
// | error word.  Host code must not use the array's name as an address: on the host it is a
// stand-in symbol.  Its device address is looked up once per device with cudaGetSymbolAddress.
// ----------------------------------------------------------------------------------------------
static_assert(sizeof(DevWalker) == 72, "DevWalker layout");
static_assert(QMC_STATIC_SCRATCH_BYTES >= QMC_STATIC_MAX_WALKERS * (sizeof(DevWalker) + sizeof(int)) + 256,
              "static scratch size");
static __device__ __align__(256) unsigned char g_static_scratch[QMC_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_static_mu;                                   // guards the staging area below
unsigned char *g_static_dev[MAX_DEVICES];                 // device address of g_static_scratch
DevWalker g_static_walkers[QMC_STATIC_MAX_WALKERS];       // host staging of the table
int g_static_order[QMC_STATIC_MAX_WALKERS];               // host staging of the order

unsigned *static_error_word(int dev)
{
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_dev[dev]) return nullptr;
    return reinterpret_cast<unsigned *>(g_static_dev[dev] +
                                        QMC_STATIC_MAX_WALKERS * (sizeof(DevWalker) + sizeof(int)));
}

int static_setup(int dev, unsigned char *&base)
{
    // caller holds g_static_mu; `dev` is the current device
    if (!g_static_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_static_dev[dev] = static_cast<unsigned char *>(p);
    }
    base = g_static_dev[dev];
    return QMC_OK;
}

}  // namespace

extern "C" int qmc_sweep_static(const qmc_walker_desc *d, int W, const qmc_options *opt, void *pos, double *logpsi,
                                uint64_t *sweep, uint64_t seed, int nsweeps, int energy_every, double *accum,
                                uint32_t *err, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = check_options(opt);
    if (rc) return rc;
    if (!d) return fail(QMC_ERR_ARG, "descriptor pointer is NULL");
    if (W <= 0) return fail(QMC_ERR_ARG, "W must be > 0");
    // the host staging area below is reused by the next call, so a copy recorded into a graph
    // would read whatever the latest call staged: refuse before anything is enqueued
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(QMC_ERR_ARG, "qmc_sweep_static stages its walker table from host memory reused by the next "
                                 "call and cannot be recorded during stream capture; call it outside capture");
    if (W > QMC_STATIC_MAX_WALKERS)
        return fail(QMC_ERR_ARG, "qmc_sweep_static takes at most %d walkers (got %d); use qmc_sweep",
                    QMC_STATIC_MAX_WALKERS, W);
    if ((rc = check_ptr(pos, "pos", 16)) || (rc = check_ptr(logpsi, "logpsi", 8)) ||
        (rc = check_ptr(sweep, "sweep", 8)) || (rc = check_ptr(accum, "accum", 8)))
        return rc;
    if (err && (uintptr_t)err % 4) return fail(QMC_ERR_ARG, "err must be 4-byte aligned");
    if (nsweeps < 0) return fail(QMC_ERR_ARG, "nsweeps must be >= 0");
    if (energy_every < 0) return fail(QMC_ERR_ARG, "energy_every must be >= 0");
    int dev;
    if ((rc = current_device(dev))) return rc;
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");

    std::lock_guard<std::mutex> lk(g_static_mu);
    unsigned char *base = nullptr;
    if ((rc = static_setup(dev, base))) return rc;
    Plan P;  // shape summary only: no device table, no containers filled
    P.device = dev;
    P.W = W;
    P.sym = opt->sym;
    P.maxn = P.maxpad = 0;
    P.m5 = true;
    for (int w = 0; w < W; ++w) {
        if ((rc = resolve_one(d[w], w, opt, g_static_walkers[w]))) return rc;
        P.maxn = std::max(P.maxn, d[w].n);
        P.maxpad = std::max(P.maxpad, d[w].pad_n);
        if (d[w].m_exp != 5.0) P.m5 = false;
        g_static_order[w] = w;
    }
    // longest walkers first; ties by index (std::sort works in place)
    std::sort(g_static_order, g_static_order + W, [&](int a, int b) {
        return d[a].n != d[b].n ? d[a].n > d[b].n : a < b;
    });
    const int tpw = choose_tpw(P, opt, dev, nsm);
    if (nsweeps == 0) return QMC_OK;

    DevWalker *d_walkers = reinterpret_cast<DevWalker *>(base);
    int *d_order = reinterpret_cast<int *>(base + QMC_STATIC_MAX_WALKERS * sizeof(DevWalker));
    unsigned *d_err = reinterpret_cast<unsigned *>(base + QMC_STATIC_MAX_WALKERS * (sizeof(DevWalker) + sizeof(int)));
    // pageable host -> device: the staging area may be reused once these calls return
    e = cudaMemcpyAsync(d_walkers, g_static_walkers, sizeof(DevWalker) * (size_t)W, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, g_static_order, sizeof(int) * (size_t)W, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !err) e = cudaMemsetAsync(d_err, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e, "static walker table upload");

    int G = 1;
    if ((rc = choose_groups(P, opt, tpw, dev, nsm, G))) return rc;
    const Shape sh = shape_of(P, opt->precision, tpw, G, true);
    SweepArgs a;
    a.walkers = d_walkers;
    a.order = d_order;
    a.W = W;
    a.G = G;
    a.stride = sh.stride;
    a.tile = sh.tile;  // 0 or 1: no drift scratch to allocate
    a.fscr = nullptr;
    a.gmem = sh.gmem;
    a.pos = pos;
    a.logpsi = logpsi;
    a.sweep = reinterpret_cast<unsigned long long *>(sweep);
    a.accum = accum;
    a.seed = seed;
    a.nsweeps = nsweeps;
    a.energy_every = energy_every;
    a.recompute_every = opt->recompute_every;
    a.proposal = opt->proposal;
    a.sequential = opt->sequential;
    a.h2m = opt->hbar2_over_m;
    a.err = err ? reinterpret_cast<unsigned *>(err) : d_err;
    a.dynamic = 0;  // one walker per group: no queue memory needed
    a.chunk_moves = 0;
    a.q_total = 0;
    a.q_head = a.q_tail = nullptr;
    a.q_slots = nullptr;
    a.q_prog = nullptr;
    a.wait_ns = knobs().wait_ns;
    a.drop_push = 0;
    const int grid = (W + G - 1) / G;
    const size_t smem = (size_t)G * sh.smem;
    e = launch_sweep(opt->precision, tpw, variant_of(P, opt), grid, G * tpw, smem, st, a);
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    g_launches.fetch_add(1);
    return QMC_OK;
}
