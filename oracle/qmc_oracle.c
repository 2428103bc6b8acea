/*
 * qmc_oracle.c -- plain FP64 CPU oracle for variational Monte Carlo of liquid 4He
 * (Y. Lutsyshyn, "Fast quantum Monte Carlo on a GPU").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA library is compared against.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load it; the library
 * never calls it and shares no code with it.  Every routine is the plain definition written
 * out in double precision, in the order and notation of the paper, with no blocking, fusion
 * or reordering.  OpenMP is used only to run independent walkers side by side.
 *
 * Readings of the paper taken here (where it is silent or garbled):
 *  - Eq. (uFunction) prints a ratio that is the pair factor exp(u); the Jastrow exponent is
 *    read as u(r) = f(r) + f(L-r) - 2 f(L/2) for r < L/2 and 0 beyond, with f of
 *    Eq. (fifthPower) and its exponent 5 generalised to a parameter m.  sym = 0 gives the
 *    plain truncated u(r) = f(r) for r < L/2.
 *  - The Aziz II (HFD-B(HE)) constants are not printed in the paper; the published 1987
 *    values are used (eps = 10.948 K, r_m = 2.963 A, ...), pinned by the minimum of V.
 *  - The paper draws its random numbers with KISS on the host (Sec. 5.2).  Here both sides use
 *    the counter-based Philox4x32-10 generator (Salmon, Moraes, Dror, Shaw, SC'11), with the
 *    counter = (move t, sweep k, walker id w, stream) and key = the 64-bit seed.
 *  - Trial displacement: uniform cube of half-width `step` (default) or Gaussian with
 *    per-component sigma `step` (the paper's choice, Sec. 2 and Sec. 7).
 *  - Start configuration (the paper reads it from a file, Sec. 5.1): fcc sites chosen by a
 *    Philox Fisher-Yates shuffle, plus Gaussian jitter, wrapped into the box.
 *  - Kinetic energy: three estimators (local T_L, Pandharipande-Bethe T_PB, Fisher-like T_F);
 *    the paper (Sec. 5.4) says two of them are written and agree statistically.
 *  - The (b, m) derivatives are not in the paper; they are the exact derivatives of the
 *    expressions above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of a multiply/xor Feistel-like bijection
 * on a 128-bit counter, with a 64-bit key bumped by the Weyl constants between rounds.      */
/* ------------------------------------------------------------------------------------------ */
ORC_API void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t out[4])
{
    uint32_t ctr[4] = {a, b, c, d};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Stream numbers in the fourth counter word. */
enum { STREAM_STEP = 0, STREAM_INDEX = 1, STREAM_SHUFFLE = 2, STREAM_JITTER = 3, STREAM_DICE = 4 };

/* uniform on (0,1): (x + 1/2) 2^-32, exact in double */
static double unif(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }
/* 2u - 1 in (-1,1), exact in double */
static double sym_unif(uint32_t x) { return ((double)(2 * (int64_t)x + 1 - 4294967296LL)) * 0x1p-32; }
/* integer in [0, n) from a 32-bit word: floor(x n / 2^32) */
static uint32_t index_of(uint32_t x, uint32_t n) { return (uint32_t)(((uint64_t)x * (uint64_t)n) >> 32); }

/* ------------------------------------------------------------------------------------------ */
/* Pair functions                                                                             */
/* ------------------------------------------------------------------------------------------ */

/* Eq. (fifthPower), exponent m: f(r) = -(1/2) (b/r)^m, and its r-derivatives. */
static double f_sv(double r, double b, double m) { return -0.5 * pow(b / r, m); }
static double f_sv_1(double r, double b, double m) { return 0.5 * m * pow(b, m) * pow(r, -m - 1.0); }
static double f_sv_2(double r, double b, double m) { return -0.5 * m * (m + 1.0) * pow(b, m) * pow(r, -m - 2.0); }
/* m-derivatives of f, f', f'' (exact derivatives of the three expressions above) */
static double f_sv_m(double r, double b, double m) { return -0.5 * pow(b / r, m) * log(b / r); }
static double f_sv_1m(double r, double b, double m)
{
    return 0.5 * pow(b, m) * pow(r, -m - 1.0) * (1.0 + m * log(b / r));
}
static double f_sv_2m(double r, double b, double m)
{
    return -0.5 * pow(b, m) * pow(r, -m - 2.0) * ((2.0 * m + 1.0) + m * (m + 1.0) * log(b / r));
}
/* b-derivatives of f, f', f'' */
static double f_sv_b(double r, double b, double m) { return -0.5 * m * pow(b, m - 1.0) * pow(r, -m); }
static double f_sv_1b(double r, double b, double m) { return 0.5 * m * m * pow(b, m - 1.0) * pow(r, -m - 1.0); }
static double f_sv_2b(double r, double b, double m)
{
    return -0.5 * m * m * (m + 1.0) * pow(b, m - 1.0) * pow(r, -m - 2.0);
}

typedef struct {
    double L, b, m;
    int sym;
} jastrow_t;

/* Eq. (uFunction), as read above: u at distance r (zero for r >= L/2, the cutoff of Sec. 7),
 * and in pair_t also u', u'' and the b and m derivatives of all three.                      */
typedef struct {
    double u, u1, u2;       /* u, du/dr, d2u/dr2 */
    double ub, u1b, u2b;    /* d/db of the three */
    double um, u1m, u2m;    /* d/dm of the three */
} pair_t;

static double u_of(double r, const jastrow_t *J)
{
    const double h = 0.5 * J->L;
    if (!(r < h)) return 0.0;
    double u = f_sv(r, J->b, J->m);
    if (J->sym) u += f_sv(J->L - r, J->b, J->m) - 2.0 * f_sv(h, J->b, J->m);
    return u;
}

static pair_t pair_terms(double r, const jastrow_t *J, int with_params)
{
    pair_t p;
    memset(&p, 0, sizeof p);
    const double L = J->L, b = J->b, m = J->m, h = 0.5 * J->L;
    if (!(r < h)) return p;
    p.u = f_sv(r, b, m);
    p.u1 = f_sv_1(r, b, m);
    p.u2 = f_sv_2(r, b, m);
    if (J->sym) {
        const double s = L - r;
        /* f(L - r): its r-derivative is -f'(L - r), its second derivative +f''(L - r) */
        p.u += f_sv(s, b, m) - 2.0 * f_sv(h, b, m);
        p.u1 -= f_sv_1(s, b, m);
        p.u2 += f_sv_2(s, b, m);
    }
    if (with_params) {
        p.ub = f_sv_b(r, b, m);
        p.u1b = f_sv_1b(r, b, m);
        p.u2b = f_sv_2b(r, b, m);
        p.um = f_sv_m(r, b, m);
        p.u1m = f_sv_1m(r, b, m);
        p.u2m = f_sv_2m(r, b, m);
        if (J->sym) {
            const double s = L - r;
            p.ub += f_sv_b(s, b, m) - 2.0 * f_sv_b(h, b, m);
            p.u1b -= f_sv_1b(s, b, m);
            p.u2b += f_sv_2b(s, b, m);
            p.um += f_sv_m(s, b, m) - 2.0 * f_sv_m(h, b, m);
            p.u1m -= f_sv_1m(s, b, m);
            p.u2m += f_sv_2m(s, b, m);
        }
    }
    return p;
}

ORC_API void orc_pair_u(double r, double L, double b, double m, int sym, double out[9])
{
    jastrow_t J = {L, b, m, sym};
    pair_t p = pair_terms(r, &J, 1);
    out[0] = p.u; out[1] = p.u1; out[2] = p.u2;
    out[3] = p.ub; out[4] = p.u1b; out[5] = p.u2b;
    out[6] = p.um; out[7] = p.u1m; out[8] = p.u2m;
}

/* orc_pair_u at each of cnt distances r[k]: out[9 k .. 9 k + 8] (test scales need many pairs). */
ORC_API void orc_pair_u_many(int cnt, const double *r, double L, double b, double m, int sym, double *out)
{
    for (int k = 0; k < cnt; ++k) orc_pair_u(r[k], L, b, m, sym, out + 9 * (size_t)k);
}

/* HFD-B(HE) ("Aziz II") pair potential in K, r in A, without cutoff. */
ORC_API double orc_aziz(double r)
{
    const double eps = 10.948, rm = 2.963;
    const double A = 1.8443101e5, alpha = 10.43329537, beta = -2.27965105;
    const double C6 = 1.36745214, C8 = 0.42123807, C10 = 0.17473318, D = 1.4826;
    const double x = r / rm;
    const double F = (x < D) ? exp(-pow(D / x - 1.0, 2.0)) : 1.0;
    return eps * (A * exp(-alpha * x + beta * x * x) - F * (C6 / pow(x, 6.0) + C8 / pow(x, 8.0) + C10 / pow(x, 10.0)));
}

/* ------------------------------------------------------------------------------------------ */
/* Periodic cubic box                                                                         */
/* ------------------------------------------------------------------------------------------ */

/* nearest periodic image of a coordinate difference */
static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

/* put a coordinate displaced by less than one box length back into [0, L] */
static double wrap(double x, double L)
{
    if (x < 0.0) return x + L;
    if (x >= L) return x - L;
    return x;
}

static double pair_dist(const double *x, const double *y, const double *z, int i, int j, double L,
                        double d[3])
{
    d[0] = min_image(x[i] - x[j], L);
    d[1] = min_image(y[i] - y[j], L);
    d[2] = min_image(z[i] - z[j], L);
    return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

/* ------------------------------------------------------------------------------------------ */
/* Wavefunction and local energy                                                              */
/* ------------------------------------------------------------------------------------------ */

/* Eq. (Jastrow): ln psi = sum_{i<j} u(r_ij) */
ORC_API double orc_log_psi(int n, const double *x, const double *y, const double *z, double L, double b,
                           double m, int sym)
{
    jastrow_t J = {L, b, m, sym};
    double s = 0.0, d[3];
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) s += u_of(pair_dist(x, y, z, i, j, L, d), &J);
    return s;
}

/* Per-particle pieces of the local kinetic energy:
 *   lap[i] = nabla_i^2 ln psi = sum_{j != i} (u'' + 2 u'/r),
 *   F[i]   = nabla_i ln psi   = sum_{j != i} u'(r_ij) (r_i - r_j)/r_ij.                        */
ORC_API void orc_local_terms(int n, const double *x, const double *y, const double *z, double L, double b,
                             double m, int sym, double *lap, double *Fx, double *Fy, double *Fz)
{
    jastrow_t J = {L, b, m, sym};
    double d[3];
    for (int i = 0; i < n; ++i) {
        double l = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double r = pair_dist(x, y, z, i, j, L, d);
            pair_t p = pair_terms(r, &J, 0);
            l += p.u2 + 2.0 * p.u1 / r;
            fx += p.u1 * d[0] / r;
            fy += p.u1 * d[1] / r;
            fz += p.u1 * d[2] / r;
        }
        lap[i] = l; Fx[i] = fx; Fy[i] = fy; Fz[i] = fz;
    }
}

/* Local energy E_L = H psi / psi for the Hamiltonian of Sec. 2 (totals in K):
 *   out = {V, T_L, T_PB, T_F, E_L}
 *   V    = sum_{i<j, r < L/2} V_Aziz(r_ij)
 *   T_L  = -(hbar^2/2m) sum_i [ lap_i + |F_i|^2 ]         (local kinetic energy)
 *   T_PB = -(hbar^2/4m) sum_i lap_i                        (Pandharipande-Bethe form)
 *   T_F  = +(hbar^2/2m) sum_i |F_i|^2                      (drift-squared form)
 * The three kinetic estimators have the same expectation (integration by parts).           */
ORC_API void orc_local_energy(int n, const double *x, const double *y, const double *z, double L, double b,
                              double m, int sym, double hbar2_over_m, double out[5])
{
    double *lap = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    double *Fx = lap + n, *Fy = lap + 2 * n, *Fz = lap + 3 * n;
    orc_local_terms(n, x, y, z, L, b, m, sym, lap, Fx, Fy, Fz);
    double V = 0.0, d[3];
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double r = pair_dist(x, y, z, i, j, L, d);
            if (r < 0.5 * L) V += orc_aziz(r);
        }
    double sl = 0.0, sf = 0.0;
    for (int i = 0; i < n; ++i) {
        sl += lap[i];
        sf += Fx[i] * Fx[i] + Fy[i] * Fy[i] + Fz[i] * Fz[i];
    }
    free(lap);
    const double k = 0.5 * hbar2_over_m; /* hbar^2 / 2m */
    out[0] = V;
    out[1] = -k * (sl + sf);
    out[2] = -0.5 * k * sl;
    out[3] = k * sf;
    out[4] = V + out[1];
}

/* ln psi, E_L and their derivatives in the Jastrow parameters b and m:
 *   out = {ln psi, E_L, d ln psi/db, d ln psi/dm, dE_L/db, dE_L/dm}
 * dE_L/da = -(hbar^2/2m) sum_i [ d lap_i/da + 2 F_i . dF_i/da ]   (V does not depend on a). */
ORC_API void orc_energy_grad(int n, const double *x, const double *y, const double *z, double L, double b,
                             double m, int sym, double hbar2_over_m, double out[6])
{
    jastrow_t J = {L, b, m, sym};
    double e[5], d[3];
    orc_local_energy(n, x, y, z, L, b, m, sym, hbar2_over_m, e);
    double lp = 0.0, lpb = 0.0, lpm = 0.0, gb = 0.0, gm = 0.0;
    for (int i = 0; i < n; ++i) {
        double F[3] = {0, 0, 0}, Fb[3] = {0, 0, 0}, Fm[3] = {0, 0, 0};
        double lapb = 0.0, lapm = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double r = pair_dist(x, y, z, i, j, L, d);
            pair_t p = pair_terms(r, &J, 1);
            if (j > i) {
                lp += p.u;
                lpb += p.ub;
                lpm += p.um;
            }
            lapb += p.u2b + 2.0 * p.u1b / r;
            lapm += p.u2m + 2.0 * p.u1m / r;
            for (int c = 0; c < 3; ++c) {
                F[c] += p.u1 * d[c] / r;
                Fb[c] += p.u1b * d[c] / r;
                Fm[c] += p.u1m * d[c] / r;
            }
        }
        gb += lapb + 2.0 * (F[0] * Fb[0] + F[1] * Fb[1] + F[2] * Fb[2]);
        gm += lapm + 2.0 * (F[0] * Fm[0] + F[1] * Fm[1] + F[2] * Fm[2]);
    }
    const double k = 0.5 * hbar2_over_m;
    out[0] = lp;
    out[1] = e[4];
    out[2] = lpb;
    out[3] = lpm;
    out[4] = -k * gb;
    out[5] = -k * gm;
}

/* Eq. (JastrowUpdate): ln psi(X') - ln psi(X) for particle s moved to wrap(r_s + delta):
 * sum_{i != s} [u(|r_s + delta - r_i|) - u(|r_s - r_i|)].  The new position is returned.    */
ORC_API double orc_trial_delta(int n, const double *x, const double *y, const double *z, double L, double b,
                               double m, int sym, int s, double dx, double dy, double dz, double newpos[3])
{
    jastrow_t J = {L, b, m, sym};
    const double xn = wrap(x[s] + dx, L), yn = wrap(y[s] + dy, L), zn = wrap(z[s] + dz, L);
    double sum = 0.0;
    for (int i = 0; i < n; ++i) {
        if (i == s) continue;
        double a0 = min_image(xn - x[i], L), a1 = min_image(yn - y[i], L), a2 = min_image(zn - z[i], L);
        double b0 = min_image(x[s] - x[i], L), b1 = min_image(y[s] - y[i], L), b2 = min_image(z[s] - z[i], L);
        double rn = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
        double ro = sqrt(b0 * b0 + b1 * b1 + b2 * b2);
        sum += u_of(rn, &J) - u_of(ro, &J);
    }
    if (newpos) {
        newpos[0] = xn; newpos[1] = yn; newpos[2] = zn;
    }
    return sum;
}

/* Pair-distance histogram (the paper's g(r) analysis, Sec. 5.4): pairs i < j with r < rmax,
 * bin floor(r nbins / rmax); counts added to out[nbins].                                      */
ORC_API void orc_pair_hist(int n, const double *x, const double *y, const double *z, double L, int nbins,
                           double rmax, uint64_t *out)
{
    double d[3];
    const double scale = (double)nbins / rmax;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double r = pair_dist(x, y, z, i, j, L, d);
            if (r < rmax) {
                int b = (int)(r * scale);
                if (b > nbins - 1) b = nbins - 1;
                out[b] += 1;
            }
        }
}

/* ------------------------------------------------------------------------------------------ */
/* Random numbers of one move: particle s, displacement delta, dice xi                         */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    uint64_t seed;
    uint32_t wid;
    int proposal;   /* 0: uniform cube of half-width step, 1: Gaussian of sigma step */
    int sequential; /* 1: s = t */
} rng_t;

static void move_randoms(const rng_t *R, int n, uint32_t t, uint32_t k, double step, int *s, double delta[3],
                         double *xi)
{
    uint32_t w[4], iw[4];
    philox(R->seed, t, k, R->wid, STREAM_STEP, w);
    if (R->sequential) {
        *s = (int)t;
    } else {
        philox(R->seed, t >> 2, k, R->wid, STREAM_INDEX, iw);
        *s = (int)index_of(iw[t & 3u], (uint32_t)n);
    }
    if (R->proposal == 0) {
        delta[0] = step * sym_unif(w[0]);
        delta[1] = step * sym_unif(w[1]);
        delta[2] = step * sym_unif(w[2]);
        *xi = unif(w[3]);
    } else {
        /* Box-Muller on (u0, u1) and (u2, u3); three of the four normals are used */
        const double two_pi = 6.283185307179586;
        double r0 = sqrt(-2.0 * log(unif(w[0]))), r1 = sqrt(-2.0 * log(unif(w[2])));
        delta[0] = step * (r0 * cos(two_pi * unif(w[1])));
        delta[1] = step * (r0 * sin(two_pi * unif(w[1])));
        delta[2] = step * (r1 * cos(two_pi * unif(w[3])));
        uint32_t dw[4];
        philox(R->seed, t >> 2, k, R->wid, STREAM_DICE, dw);
        *xi = unif(dw[t & 3u]);
    }
}

ORC_API void orc_move_randoms(uint64_t seed, uint32_t wid, int proposal, int sequential, int n, uint32_t t,
                              uint32_t k, double step, int *s, double delta[3], double *xi)
{
    rng_t R = {seed, wid, proposal, sequential};
    move_randoms(&R, n, t, k, step, s, delta, xi);
}

/* ------------------------------------------------------------------------------------------ */
/* Start configuration                                                                        */
/* ------------------------------------------------------------------------------------------ */

/* fcc lattice with nc^3 cubic cells (4 sites each, enumerated (ix, iy, iz, basis)); a shuffle
 * driven by Philox stream 2 picks n sites; Box-Muller jitter of width sigma from stream 3.    */
ORC_API void orc_init_walker(int n, double L, uint64_t seed, uint32_t wid, double sigma, double *x, double *y,
                             double *z)
{
    int nc = 1;
    while (4LL * nc * nc * nc < n) ++nc;
    const int M = 4 * nc * nc * nc;
    const double a = L / nc;
    const double bx[4] = {0.0, 0.5, 0.5, 0.0}, by[4] = {0.0, 0.5, 0.0, 0.5}, bz[4] = {0.0, 0.0, 0.5, 0.5};
    int *perm = (int *)malloc(sizeof(int) * (size_t)M);
    for (int q = 0; q < M; ++q) perm[q] = q;
    for (int i = 0; i < n; ++i) {
        uint32_t w[4];
        philox(seed, (uint32_t)i >> 2, 0u, wid, STREAM_SHUFFLE, w);
        int j = i + (int)index_of(w[i & 3], (uint32_t)(M - i));
        int tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
    }
    const double two_pi = 6.283185307179586;
    for (int i = 0; i < n; ++i) {
        int q = perm[i];
        int basis = q % 4, cell = q / 4;
        int iz = cell % nc, iy = (cell / nc) % nc, ix = cell / (nc * nc);
        uint32_t w[4];
        philox(seed, (uint32_t)i, 0u, wid, STREAM_JITTER, w);
        double r0 = sqrt(-2.0 * log(unif(w[0]))), r1 = sqrt(-2.0 * log(unif(w[2])));
        double gx = r0 * cos(two_pi * unif(w[1]));
        double gy = r0 * sin(two_pi * unif(w[1]));
        double gz = r1 * cos(two_pi * unif(w[3]));
        x[i] = wrap((ix + bx[basis]) * a + sigma * gx, L);
        y[i] = wrap((iy + by[basis]) * a + sigma * gy, L);
        z[i] = wrap((iz + bz[basis]) * a + sigma * gz, L);
    }
    free(perm);
}

/* ------------------------------------------------------------------------------------------ */
/* Metropolis sweeps                                                                          */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int n;
    double L, b, m, step;
    int sym, proposal, sequential;
    double hbar2_over_m;
    int recompute_every;
    uint64_t seed;
    uint32_t wid;
} orc_walker_t;

/* One walker, sweeps k = *sweep .. *sweep + nsweeps - 1.  A sweep (the paper's macroupdate,
 * Sec. 4.1) is n single-particle moves.  Each move: draw (s, delta, xi), evaluate
 * Eq. (JastrowUpdate), accept iff exp(2 Delta) > xi (Eq. Decision), and on acceptance move the
 * particle and add Delta to ln psi.  After sweep k: ln psi is recomputed from scratch when
 * (k+1) is a multiple of recompute_every, and the local energy is sampled when (k+1) is a
 * multiple of energy_every.
 * accum (added to): {sum E_L, sum E_L^2, sum V, sum T_L, sum T_PB, sum T_F, samples, accepted}.
 * margins (optional, n*nsweeps entries): 2 Delta - ln xi of every move, in order.            */
ORC_API void orc_run_walker(const orc_walker_t *P, double *x, double *y, double *z, double *logpsi,
                            uint64_t *sweep, int nsweeps, int energy_every, double accum[8], double *margins)
{
    rng_t R = {P->seed, P->wid, P->proposal, P->sequential};
    const int n = P->n;
    uint64_t k = *sweep;
    for (int it = 0; it < nsweeps; ++it, ++k) {
        for (int t = 0; t < n; ++t) {
            int s;
            double delta[3], xi, np[3];
            move_randoms(&R, n, (uint32_t)t, (uint32_t)k, P->step, &s, delta, &xi);
            double D = orc_trial_delta(n, x, y, z, P->L, P->b, P->m, P->sym, s, delta[0], delta[1], delta[2], np);
            if (margins) margins[(size_t)it * n + t] = 2.0 * D - log(xi);
            if (exp(2.0 * D) > xi) {
                x[s] = np[0];
                y[s] = np[1];
                z[s] = np[2];
                *logpsi += D;
                accum[7] += 1.0;
            }
        }
        if (P->recompute_every > 0 && (k + 1) % (uint64_t)P->recompute_every == 0)
            *logpsi = orc_log_psi(n, x, y, z, P->L, P->b, P->m, P->sym);
        if (energy_every > 0 && (k + 1) % (uint64_t)energy_every == 0) {
            double e[5];
            orc_local_energy(n, x, y, z, P->L, P->b, P->m, P->sym, P->hbar2_over_m, e);
            accum[0] += e[4];
            accum[1] += e[4] * e[4];
            accum[2] += e[0];
            accum[3] += e[1];
            accum[4] += e[2];
            accum[5] += e[3];
            accum[6] += 1.0;
        }
    }
    *sweep = k;
}

/* W independent walkers side by side (OpenMP over walkers when built with it).
 * Walker w's coordinates are x/y/z[off[w] .. off[w] + n_w); logpsi[W], sweep[W], accum[8 W].
 * Returns the number of threads used.                                                       */
ORC_API int orc_run_batch(int W, const orc_walker_t *P, const int64_t *off, double *x, double *y, double *z,
                          double *logpsi, uint64_t *sweep, int nsweeps, int energy_every, double *accum,
                          int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    used = nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (int w = 0; w < W; ++w) {
        const int64_t o = off[w];
        orc_run_walker(&P[w], x + o, y + o, z + o, &logpsi[w], &sweep[w], nsweeps, energy_every, &accum[8 * w],
                       NULL);
    }
    return used;
}

ORC_API int orc_sizeof_walker(void) { return (int)sizeof(orc_walker_t); }
