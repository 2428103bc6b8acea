/*
 * qmc_probe.h -- calibration entry point of libqmc: the measured arithmetic rates that bound the
 * sweep of include/qmc.h on the current GPU.  The paper has no counterpart; the rates are the
 * denominators of the sweep's roofline (the sweep is bound by plain FP32 arithmetic with the SFU
 * as co-limit, not by memory or tensor cores).
 */
#ifndef QMC_PROBE_H
#define QMC_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Indices of qmc_probe_rates' results: lane operations per second per SM, except the last,
 * which is pair evaluations per second per SM.  Divided by the SM clock of the run they give the
 * rates per clock. */
#define QMC_PROBE_FFMA 0      /* FP32 fused multiply-add, scalar (fma.rn.f32) */
#define QMC_PROBE_FFMA2 1     /* FP32 fused multiply-add, packed pairs (fma.rn.f32x2), 2 per instruction */
#define QMC_PROBE_FMNMX 2     /* FP32 minimum (min.f32) */
#define QMC_PROBE_RSQRT 3     /* SFU reciprocal square root (rsqrt.approx.ftz.f32) */
#define QMC_PROBE_DFMA 4      /* FP64 fused multiply-add (fma.rn.f64) */
#define QMC_PROBE_PAIR 5      /* the sweep's FP32 partner arithmetic alone (Eqs. JastrowUpdate,
                                 uFunction, fifthPower with exponent 5): two moves, each with its
                                 old and new position in one f32x2, four partners per
                                 shared-memory chunk, no reduction */
#define QMC_PROBE_COUNT 6

/*
 * qmc_probe_rates -- run each probe kernel on blocks_per_sm x (SM count) CTAs of `threads`
 * threads (a multiple of 32, 32..1024; the pair probe at most 512) for `iters` loop iterations
 * (1..1e6) on `stream`, after a short warm-up launch, and time it with CUDA events; the rate is
 * the operations of all CTAs over the elapsed time and the SM count (the CTAs are spread evenly,
 * all resident at once; fewer per SM if the kernel's occupancy is lower).  Eight independent
 * dependency chains per thread (pair probe: one accumulator per move, eight independent pair
 * evaluations per chunk); the operations are inline PTX (pair probe: packed f32x2 intrinsics) on
 * values that change every iteration, so none is folded away or hoisted out of the loop.
 *   out    host array of QMC_PROBE_COUNT doubles, written on success.
 * Allocates and frees a small device buffer, synchronises the stream.  Returns QMC_OK, QMC_ERR_ARG
 * for out-of-range arguments or QMC_ERR_CUDA.  Not for use during stream capture.
 */
int qmc_probe_rates(int blocks_per_sm, int threads, int iters, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QMC_PROBE_H */
