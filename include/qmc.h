/*
 * qmc.h -- C ABI of libqmc: variational Monte Carlo of liquid 4He on one GB300 GPU
 * (the single-particle Metropolis sweep, its local-energy estimator and the Jastrow-parameter
 * adjoint of Y. Lutsyshyn, "Fast quantum Monte Carlo on a GPU").
 *
 * Conventions shared by every call
 * --------------------------------
 *  Units:       lengths in Angstrom, energies in Kelvin (totals per walker, not per atom).
 *  Walkers:     `d` is a HOST array of W walker descriptors.  It is read during the call and
 *               copied to a library-owned device table, cached by content, so repeated calls
 *               with the same batch upload nothing.
 *  Positions:   `pos` is a DEVICE buffer owned by the caller, float (QMC_FP32) or double
 *               (QMC_FP64).  Walker w occupies pos[d[w].offset ...] as three blocks of d[w].pad_n
 *               elements: x[pad_n] | y[pad_n] | z[pad_n] (structure of arrays).  Entries
 *               n .. pad_n-1 of each block are ignored on input and left unchanged.  Coordinates
 *               lie in [0, L]; the sweep keeps them there.  A walker stays in one CTA's shared
 *               memory for a whole call when it fits (qmc_capacity); larger walkers are used in
 *               place in HBM (their coordinates change during the call; slower, any size).
 *  Outputs:     DEVICE buffers owned by the caller, double precision, W-major.
 *  Streams:     `stream` is a cudaStream_t (NULL = legacy default stream).  Every compute call
 *               only enqueues work on it and returns; results are ready when the stream is.
 *  Errors:      return 0 or a negative QMC_ERR_* code; qmc_last_error() gives a message
 *               (per host thread).  Argument and capacity errors are detected before anything
 *               is enqueued, so no output or position is touched.  Faults found by a kernel
 *               (a non-finite coordinate or ratio) set a device error word that qmc_status()
 *               reads; a walker that trips it stops and writes back neither its positions nor
 *               its ln psi and sweep counter (energy samples it took before stay in accum).
 *  Threads:     calls may come from several host threads; the descriptor cache is locked.
 *  Overlap:     calls with the same walker descriptors share the library's device table of that
 *               batch, and qmc_sweep calls of a batch with more walkers than SMs also share its
 *               walker queue: two such qmc_sweep calls must not run at the same time on the GPU
 *               (issue them on one stream, or order their streams).  Batches with different
 *               descriptors (for instance other walker ids) are independent.
 *
 * Citations are to sections and equations of the paper.
 */
#ifndef QMC_H
#define QMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QMC_VERSION 110 /* 1.1.0 */

#define QMC_OK 0
#define QMC_ERR_ARG (-1)      /* null pointer, W <= 0, n < 2, bad padding/alignment, non-finite or
                                 out-of-range parameter */
#define QMC_ERR_CAPACITY (-2) /* qmc_init_walkers: the start lattice of a walker is too large */
#define QMC_ERR_CUDA (-3)     /* a CUDA runtime call failed (message has the CUDA error string) */
#define QMC_ERR_DEVICE (-4)   /* a kernel flagged a non-finite coordinate or ratio (qmc_status) */
#define QMC_ERR_TIMEOUT (-5)  /* qmc_status: the stream did not finish within the time limit */

#define QMC_FP32 0 /* pair arithmetic in float, per-walker sums and ln psi in double */
#define QMC_FP64 1 /* everything in double */

#define QMC_CUBE 0  /* trial displacement uniform in the cube [-step, step]^3 */
#define QMC_GAUSS 1 /* trial displacement Gaussian, standard deviation `step` per component */

/* Device error word bits (qmc_status) */
#define QMC_DEVERR_NONFINITE_POS 1u   /* a loaded coordinate was NaN/Inf or outside [0, L] */
#define QMC_DEVERR_NONFINITE_RATIO 2u /* a trial log-ratio was NaN */
#define QMC_DEVERR_BAD_INDEX 4u       /* qmc_trial_delta: an atom index outside [0, n) (move skipped) */
#define QMC_DEVERR_TIMEOUT 8u         /* qmc_sweep: a wait on the walker queue or on a cluster
                                         exchange exceeded its limit (10 s) */

/* Per-walker accumulator record of qmc_sweep: QMC_ACCUM_FIELDS doubles per walker, W-major.
 *   0 sum E_L   1 sum E_L^2   2 sum V   3 sum T_L   4 sum T_PB   5 sum T_F   (energy samples)
 *   6 number of energy samples            7 number of accepted moves
 *   8 sum over ln psi recomputes of |ln psi carried - ln psi recomputed|   (the drift of the
 *     incrementally updated ln psi of Eq. (JastrowUpdate) against Eq. (Jastrow))
 *   9 largest such |drift| (a maximum, not a sum; starts from the value passed in) */
#define QMC_ACCUM_FIELDS 10

/* One walker (one Markov chain).  64 bytes. */
typedef struct qmc_walker_desc {
    int32_t n;      /* number of atoms N, >= 2 */
    int32_t pad_n;  /* block stride of pos in elements: >= n and a multiple of 4 */
    int64_t offset; /* element offset of this walker's x block in pos: multiple of 4, >= 0 */
    int64_t id;     /* walker id in the random-number counter (low 32 bits are used) */
    double L;       /* cubic box side (Angstrom); <= 0 means (n / rho)^(1/3) */
    double rho;     /* number density (Angstrom^-3), used only when L <= 0 */
    double b;       /* Jastrow length b of Eq. (fifthPower), Angstrom, >= 0 */
    double m_exp;   /* Jastrow exponent (5 in Eq. (fifthPower)), > 0 */
    double step;    /* trial step: cube half-width (QMC_CUBE) or sigma (QMC_GAUSS), Angstrom */
} qmc_walker_desc;

/* Options shared by a call.  40 bytes. */
typedef struct qmc_options {
    int32_t precision;          /* QMC_FP32 or QMC_FP64 */
    int32_t proposal;           /* QMC_CUBE or QMC_GAUSS */
    int32_t sym;                /* 1: symmetrised u(r) = f(r) + f(L-r) - 2 f(L/2) (Eq. uFunction);
                                   0: u(r) = f(r); both vanish for r >= L/2 */
    int32_t sequential;         /* 1: move t displaces atom t; 0: atom drawn at random (Sec. 2) */
    double hbar2_over_m;        /* hbar^2 / m_He in K Angstrom^2 (12.1194) */
    int32_t recompute_every;    /* qmc_sweep: recompute ln psi from scratch after sweeps k with
                                   (k+1) % recompute_every == 0; 0 = never */
    int32_t threads_per_walker; /* 0 = autotuned choice (or built-in heuristic); else one of
                                   32, 64, 128, 256, 512, 1024 */
    int32_t walkers_per_cta;    /* 0 = autotuned choice (or built-in heuristic); else 1..8 walkers
                                   share one CTA (walkers_per_cta * threads_per_walker <= 256, or
                                   1); ignored where a walker is served by a whole CTA or more */
    int32_t reserved;           /* must be 0 */
} qmc_options;

/*
 * qmc_init_walkers -- start configurations (the paper reads them from a file, Sec. 5.1).
 * For each walker: an fcc lattice of nc^3 cubic cells with nc the smallest integer such that
 * 4 nc^3 >= n; n of its sites picked by a Fisher-Yates shuffle driven by Philox4x32-10 stream 2;
 * each site displaced by Gaussian noise of standard deviation jitter_sigma (Box-Muller on
 * Philox stream 3) and wrapped into [0, L).  Key = seed; counters carry the walker id.
 * Writes pos (entries n..pad_n-1 are set to 0).  jitter_sigma >= 0.
 */
int qmc_init_walkers(const qmc_walker_desc *d, int W, uint64_t seed, double jitter_sigma,
                     const qmc_options *opt, void *pos, void *stream);

/*
 * qmc_sweep -- nsweeps Metropolis sweeps of every walker (Sec. 2, Sec. 5.1).
 * A sweep (the paper's macroupdate, Sec. 4.1) is n single-atom moves t = 0..n-1.  Move t of sweep
 * k draws Philox4x32-10 words with key = seed and counter (t, k, id, 0) for the displacement and
 * dice xi, and (t/4, k, id, 1) for the atom index s (word t mod 4; s = floor(word n / 2^32)).
 * The ratio |psi(X')|^2/|psi(X)|^2 = exp(2 Delta) with Delta of Eq. (JastrowUpdate) is compared
 * with xi (Eq. Decision); on acceptance r_s <- wrap(r_s + delta) and logpsi += Delta.
 * After sweep k: if recompute_every > 0 and (k+1) % recompute_every == 0, ln psi is recomputed
 * (Eq. Jastrow); if energy_every > 0 and (k+1) % energy_every == 0, the local energy is sampled
 * and added to accum.
 *   pos      in/out device positions
 *   logpsi   in/out [W] device, running ln psi (only carried, never used for decisions)
 *   sweep    in/out [W] device, uint64 absolute sweep index k of each walker's next sweep
 *   accum    in/out [W*QMC_ACCUM_FIELDS] device, added to: the energy sums, sample and
 *            acceptance counts and the ln psi drift of each recompute (see QMC_ACCUM_FIELDS)
 * The same (seed, id, k) always reproduces the same chain: a run split over several calls is
 * bit-identical to one call.
 * Device memory: the first call of a batch allocates its walker table (and, for batches of
 * more walkers than SMs, the walker queue); an FP32 call with an energy sample whose drift
 * arrays would crowd shared memory (about N > 2400 at 128 threads per walker) also grows a
 * library-owned drift scratch.  Under CUDA stream capture no allocation is possible, so a
 * captured call must follow an uncaptured call of the same batch shape.
 */
int qmc_sweep(const qmc_walker_desc *d, int W, const qmc_options *opt, void *pos, double *logpsi,
              uint64_t *sweep, uint64_t seed, int nsweeps, int energy_every, double *accum,
              void *stream);

/*
 * qmc_local_energy -- local energy of each configuration (Sec. 2 Hamiltonian, Jastrow of
 * Eqs. (Jastrow), (uFunction), (fifthPower); Aziz II potential; cutoff L/2 for V and u, Sec. 7).
 *   out [W*5] device: {V, T_L, T_PB, T_F, E_L} with
 *   V    = sum_{i<j, r<L/2} V(r_ij)
 *   T_L  = -(hbar^2/2m) sum_i [nabla_i^2 ln psi + |nabla_i ln psi|^2],  E_L = V + T_L
 *   T_PB = -(hbar^2/4m) sum_i nabla_i^2 ln psi,   T_F = (hbar^2/2m) sum_i |nabla_i ln psi|^2
 */
int qmc_local_energy(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos,
                     double *out, void *stream);

/*
 * qmc_energy_grad -- ln psi, E_L and their derivatives in the Jastrow parameters (b, m) of
 * Eq. (fifthPower), for VMC parameter optimisation (the paper has no counterpart; these are the
 * exact derivatives of the quantities above).
 *   out [W*6] device: {ln psi, E_L, d ln psi/db, d ln psi/dm, dE_L/db, dE_L/dm}
 */
int qmc_energy_grad(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos,
                    double *out, void *stream);

/*
 * qmc_log_psi -- ln psi = sum_{i<j} u(r_ij) of each configuration (Eq. Jastrow).
 *   out [W] device.
 */
int qmc_log_psi(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos,
                double *out, void *stream);

/*
 * qmc_trial_delta -- the log-ratio Delta of Eq. (JastrowUpdate) for M trial moves per walker,
 * each from the unchanged configuration, with the same device code as the sweep.
 *   s     [W*M] device int32, atom index of each trial move (0 <= s < n)
 *   delta [W*M*3] device double, displacement (dx, dy, dz) of each trial move
 *   out   [W*M] device double, Delta of each move
 */
int qmc_trial_delta(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos,
                    const int32_t *s, const double *delta, int M, double *out, void *stream);

/*
 * qmc_pair_hist -- pair-distance histogram of each configuration, the data of the pair
 * distribution function g(r) (the paper's analysis, Sec. 5.4 and Sec. 7.1).
 *   hist  [W*nbins] device uint64, added to: the number of pairs i < j whose minimum-image
 *         distance r satisfies r < rmax, in bin floor(r * nbins / rmax).
 *   nbins 1..16384; rmax > 0 (normally <= L/2).  Counts are exact integers; in FP64 the distance
 *         is computed as sqrt((dx*dx + dy*dy) + dz*dz) without fused operations.
 * g(r) of bin k is its count divided by samples * n(n-1)/2 * (4 pi / 3)(r_{k+1}^3 - r_k^3) / L^3.
 */
int qmc_pair_hist(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos, int nbins,
                  double rmax, uint64_t *hist, void *stream);

/*
 * qmc_autotune -- the launch shape of qmc_sweep chosen by measurement (the paper's heuristics of
 * Sec. 4.4 -- as many resident blocks as fit, fewer threads than atoms, multiples of 32 -- are
 * the search space): qmc_sweep is timed on a scratch copy of `pos` for every admissible pair
 * (threads per walker, walkers per CTA) -- threads 32 .. 1024 in powers of two, at most one
 * thread per 4-atom partner chunk; walkers per CTA 1, 2, 4, 8 with at most 256 threads and the
 * shared memory of one CTA -- and the fastest pair is remembered for batches of this shape
 * (largest n, W, precision, exponent, proposal).  Later calls whose options leave
 * threads_per_walker or walkers_per_cta at 0 use it.  Synchronises the stream.
 *   tpw_out, groups_out   (may be NULL) receive the chosen threads per walker and walkers per CTA.
 */
int qmc_autotune(const qmc_walker_desc *d, int W, const qmc_options *opt, const void *pos,
                 void *stream, int *tpw_out, int *groups_out);

/*
 * qmc_sweep_static -- qmc_sweep for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a service of the library.  Some callers cannot call
 * cudaMalloc at all: code running while its device memory is fully reserved by another
 * allocator, code that must not trigger the implicit synchronisation of an allocation, or
 * hosts that forbid runtime allocation.  qmc_sweep itself allocates a walker table and an
 * error word on first use of a batch; this entry point instead keeps its walker table, its
 * processing order and its error word in one fixed array in device memory that is part of
 * the library image (QMC_STATIC_SCRATCH_BYTES, about 304 KiB, held by every GPU that loads
 * the library until the process exits).  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   Arguments and results are those of qmc_sweep, plus
 *   err      optional device uint32 that receives QMC_DEVERR_* bits of this call (OR-ed into
 *            it); if NULL the bits go to a word in the fixed array, which is cleared at the
 *            start of every call and which qmc_status() reads and clears with its own word.
 *   W        at most QMC_STATIC_MAX_WALKERS; larger batches are rejected with QMC_ERR_ARG.
 * The first call on a device looks up the fixed array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  Every call overwrites the whole array:
 * calls whose work overlaps on the GPU (on different streams without ordering) race on it and
 * must not be issued.  Calls on one stream are ordered and safe.  The descriptors are copied
 * from host memory with cudaMemcpyAsync from a staging area inside the library, so two host
 * threads calling at once are serialised while they enqueue.  Because that staging area is
 * reused by the next call, a call made while `stream` is being captured is refused with
 * QMC_ERR_ARG before anything is enqueued (a recorded copy would read whatever the latest
 * call staged when the graph is replayed).
 */
#define QMC_STATIC_MAX_WALKERS 4096
#define QMC_STATIC_SCRATCH_BYTES (QMC_STATIC_MAX_WALKERS * 76 + 256)
int qmc_sweep_static(const qmc_walker_desc *d, int W, const qmc_options *opt, void *pos, double *logpsi,
                     uint64_t *sweep, uint64_t seed, int nsweeps, int energy_every, double *accum,
                     uint32_t *err, void *stream);

/* Largest n kept in one CTA's shared memory at this precision; larger walkers run from HBM. */
int qmc_capacity(int precision);

/*
 * qmc_status -- wait for `stream` (at most timeout_ms, <= 0 means no limit), then read and clear
 * the device error word of the current device (and the word that qmc_sweep_static uses when it
 * is given no `err`).  Returns QMC_OK, QMC_ERR_DEVICE (bits in *bits if non-NULL),
 * QMC_ERR_TIMEOUT or QMC_ERR_CUDA.
 */
int qmc_status(void *stream, int timeout_ms, uint32_t *bits);

/* Number of kernels this library has launched since load (process-wide counter). */
uint64_t qmc_launch_count(void);

/* Message of the last error on this host thread ("" if none). */
const char *qmc_last_error(void);

/* QMC_VERSION of the loaded library. */
int qmc_version(void);

/* Free the library's device tables, autotune cache and error words. */
void qmc_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* QMC_H */
