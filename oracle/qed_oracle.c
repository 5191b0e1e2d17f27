/*
 * FP64 CPU oracle for the QED Monte Carlo event generator of
 * "Optimized routines for event generators in QED-PIC codes" (arXiv:2008.10468).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * (the CUDA library) never calls it, includes it, or shares code with it.
 *
 * Everything is plain, slow and written to be checked against the paper by
 * eye:
 *   - synchrotron functions F(x) = x * int_x^inf K_{5/3}(t) dt and
 *     G(x) = x K_{2/3}(x) (Sec. 3.2.1) by trapezoidal quadrature of the
 *     integral representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt;
 *   - the quantum parameter chi (Sec. 2.2, after Eq. 1 and Eq. 2);
 *   - the emission density P(delta) (Eq. 1) in the form 3x^2 P(x^3) used by
 *     Algorithm 1, and the pair density P_p(delta_e) (Eq. 2, sign of the
 *     bracket corrected, see below);
 *   - the sub-step planner from the rate bounds f(b) of Sec. 3.1.1;
 *   - Algorithms 1 and 2 with local sub-stepping, recoil and children;
 *   - Philox4x32-10 (Salmon et al., SC'11) for the per-sub-step draws;
 *   - optionally, the Boris push of Algorithm 1 (inside its loop): every
 *     sub-step of an electron or positron first moves its momentum by the
 *     Lorentz force, then chi is recomputed for the draw.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   * Eq. 2 as printed, F(z) - (3/2) chi z G(z), is negative for every
 *     delta_e; the Baier-Katkov pair spectrum gives the opposite sign.  We use
 *     P_p = (c b / 3) [G(z) - delta(1-delta) F(z)].
 *   * The sub-step count is N = ceil(f / P_max) with f evaluated for the
 *     remaining time of the step; after every event the particle is
 *     re-planned from its post-event state over the time that remains.
 *   * Events are sampled at the end of a sub-step; children inherit the
 *     remaining time and are processed in the same global step.
 *   * Momentum bookkeeping conserves momentum: p <- (1-delta) p, k = delta p;
 *     p_e- = delta_e k, p_e+ = (1 - delta_e) k.
 *   * The f(b) pieces are [0,0.1) [0.1,0.5) [0.5,10) [10,inf).
 *   * A validity guard keeps the largest per-sub-step probability (the x->0
 *     limit of 3x^2 P(x^3)) at or below one.
 *
 * Compile with -ffp-contract=off, so that every product and sum is rounded
 * as written.  The remaining time is binary64 here; the CUDA path carries it
 * as a float-float pair, which agrees with it to about 1e-14 of the step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_PI 3.14159265358979323846
#define ORC_SQRT3 1.73205080756887729353

/* ------------------------------------------------------------------------ */
/* Units.  Code units: momentum in m c, fields in m c omega / e, time in     */
/* laser periods T = lambda / c.  CODATA 2022.                               */
/* ------------------------------------------------------------------------ */
static const double ORC_ALPHA = 7.2973525643e-3;       /* fine-structure     */
static const double ORC_TAU_C = 1.2880886664441626e-21;/* hbar/(m c^2), s    */
static const double ORC_C_LIGHT = 299792458.0;         /* m/s                */

/* R = alpha m c^2 / hbar in 1/period: the bracket [dt e^2 m c / hbar^2] of
 * Eq. 1 equals R * dt. */
double orc_rate_unit(double lambda_m) {
    double period = lambda_m / ORC_C_LIGHT;
    return ORC_ALPHA / ORC_TAU_C * period;
}

/* Schwinger field m^2 c^3 / (e hbar) in units of m c omega / e. */
double orc_schwinger_field(double lambda_m) {
    double omega = 2.0 * ORC_PI * ORC_C_LIGHT / lambda_m;
    return 1.0 / (omega * ORC_TAU_C);
}

/* ------------------------------------------------------------------------ */
/* Synchrotron functions, Sec. 3.2.1.                                        */
/* K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt, so                      */
/*   G(x) = x K_{2/3}(x)                                                     */
/*        = x int_0^inf exp(-x cosh t) cosh(2t/3) dt,                        */
/*   F(x) = x int_x^inf K_{5/3}(s) ds                                        */
/*        = x int_0^inf exp(-x cosh t) cosh(5t/3) / cosh t dt                */
/* (swap the order of integration).  The integrands are even and entire in  */
/* t, so the trapezoidal rule converges geometrically; the step shrinks like */
/* 1/sqrt(x) for large x, where the peak at t = 0 narrows.                   */
/* ------------------------------------------------------------------------ */
static double sync_trapezoid(double x, double nu, int divide_by_cosh) {
    if (!(x > 0.0)) return 0.0;
    if (x > 740.0) return 0.0;
    double tau = 1.0 / 16.0;
    double lim = 0.4 / sqrt(x);
    if (lim < tau) tau = lim;
    double sum = 0.0;
    for (long k = 0; k < 4000000; ++k) {
        double t = (double)k * tau;
        double ch = cosh(t);
        double g = 0.5 * (exp(-x * ch + nu * t) + exp(-x * ch - nu * t));
        if (divide_by_cosh) g /= ch;
        double wgt = (k == 0) ? 0.5 : 1.0;
        sum += wgt * g;
        /* stop once past the peak and the terms are negligible */
        if (k > 4 && t > 1.0 && g < 1e-19 * sum) break;
        if (k > 4 && g == 0.0) break;
    }
    return x * tau * sum;
}

/* Memoised form (for the timed CPU baseline only): ln F and ln G from a table
 * of the quadrature at nodes uniform in t = ln x over [ORC_TAB_LO,
 * ORC_TAB_HI], interpolated by the Lagrange polynomial through the 8 nearest
 * nodes (ln F is smooth in t: about t/3 at small x, -e^t at large x); the
 * quadrature itself outside that range.  Built by orc_table_build; off until
 * then and after orc_table_off. */
#define ORC_TAB_N 8192
#define ORC_TAB_LO 1e-8
#define ORC_TAB_HI 700.0
static double orc_tab_f[2][ORC_TAB_N];
static double orc_tab_t0, orc_tab_h;
static int orc_tab_on = 0;

static double tab_eval(int which, double x) {
    const double u = (log(x) - orc_tab_t0) / orc_tab_h;
    long k = (long)floor(u) - 3;
    if (k < 0) k = 0;
    if (k > ORC_TAB_N - 8) k = ORC_TAB_N - 8;
    double sum = 0.0;
    for (int a = 0; a < 8; ++a) {
        double w = 1.0;
        for (int b = 0; b < 8; ++b)
            if (b != a) w *= (u - (double)(k + b)) / (double)(a - b);
        sum += w * orc_tab_f[which][k + a];
    }
    return exp(sum);
}

/* F(x): first synchrotron function (F1). */
double orc_F1(double x) {
    if (orc_tab_on && x >= ORC_TAB_LO && x <= ORC_TAB_HI) return tab_eval(0, x);
    return sync_trapezoid(x, 5.0 / 3.0, 1);
}
/* G(x): second synchrotron function (F2). */
double orc_F2(double x) {
    if (orc_tab_on && x >= ORC_TAB_LO && x <= ORC_TAB_HI) return tab_eval(1, x);
    return sync_trapezoid(x, 2.0 / 3.0, 0);
}

typedef struct {
    const double* x; double* f1; double* f2; int64_t begin, end;
} sync_job;

static void* sync_worker(void* arg) {
    sync_job* j = (sync_job*)arg;
    for (int64_t i = j->begin; i < j->end; ++i) {
        if (j->f1) j->f1[i] = orc_F1(j->x[i]);
        if (j->f2) j->f2[i] = orc_F2(j->x[i]);
    }
    return NULL;
}

/* F1 and F2 over an array, on `threads` host threads. */
void orc_F1F2(int64_t n, const double* x, double* f1, double* f2, int threads);

/* Build the memoised table from the quadrature (on `threads` threads) and
 * switch it on. */
void orc_table_build(int threads) {
    static double xs[ORC_TAB_N];
    orc_tab_on = 0;
    orc_tab_t0 = log(ORC_TAB_LO);
    orc_tab_h = (log(ORC_TAB_HI) - orc_tab_t0) / (double)(ORC_TAB_N - 1);
    for (int k = 0; k < ORC_TAB_N; ++k) xs[k] = exp(orc_tab_t0 + orc_tab_h * (double)k);
    orc_F1F2(ORC_TAB_N, xs, orc_tab_f[0], orc_tab_f[1], threads);
    for (int k = 0; k < ORC_TAB_N; ++k) {
        orc_tab_f[0][k] = log(orc_tab_f[0][k]);
        orc_tab_f[1][k] = log(orc_tab_f[1][k]);
    }
    orc_tab_on = 1;
}
void orc_table_off(void) { orc_tab_on = 0; }

void orc_F1F2(int64_t n, const double* x, double* f1, double* f2, int threads) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t th[256];
    sync_job jobs[256];
    for (int t = 0; t < threads; ++t) {
        jobs[t].x = x; jobs[t].f1 = f1; jobs[t].f2 = f2;
        jobs[t].begin = n * t / threads; jobs[t].end = n * (t + 1) / threads;
        pthread_create(&th[t], NULL, sync_worker, &jobs[t]);
    }
    for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).                        */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Open-interval uniform from one 32-bit word: ((r >> 9) + 1/2) * 2^-23.
 * The value has 24 significant bits, so it is exact in binary32 too. */
double orc_uniform(uint32_t r) { return ((double)(r >> 9) + 0.5) * 0x1p-23; }

/* Draw (x, y) of sub-step s of a particle: counter (id_lo, id_hi, step,
 * s/2), key = seed; even s takes words 0,1 and odd s takes words 2,3. */
void orc_draw(uint64_t seed, uint64_t id, uint32_t step, uint32_t s, double* x, double* y) {
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, s >> 1};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    if ((s & 1u) == 0) { *x = orc_uniform(r[0]); *y = orc_uniform(r[1]); }
    else { *x = orc_uniform(r[2]); *y = orc_uniform(r[3]); }
}

/* Identifiers of the children of the event at sub-step s: counter
 * (id_lo, id_hi, step, s) under the key seed ^ (domain constant); the top
 * bit is set so that children never collide with caller-chosen ids below
 * 2^63. */
void orc_child_ids(uint64_t seed, uint64_t id, uint32_t step, uint32_t s, uint64_t out[2]) {
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, s};
    uint32_t key[2] = {(uint32_t)seed ^ 0xA511E9B3u, (uint32_t)(seed >> 32) ^ 0x63C1D2F5u};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    out[0] = ((uint64_t)r[0] | ((uint64_t)r[1] << 32)) | (1ull << 63);
    out[1] = ((uint64_t)r[2] | ((uint64_t)r[3] << 32)) | (1ull << 63);
}

/* ------------------------------------------------------------------------ */
/* Quantum parameter (Sec. 2.2):                                             */
/*   chi = sqrt((eps E / c + p x H)^2 - (p . E)^2) / E_s  (code units)       */
/* with eps = gamma for e+- (gamma = sqrt(1 + p^2)) and eps = |k| for a      */
/* photon.  Evaluated in long double from the binary32 inputs, because the   */
/* difference of squares cancels for particles co-moving with a crossed      */
/* field.                                                                    */
/* ------------------------------------------------------------------------ */
double orc_chi(int is_photon, double px, double py, double pz,
               double Ex, double Ey, double Ez, double Bx, double By, double Bz,
               double E_s, double* gamma_out) {
    long double X = px, Y = py, Z = pz;
    long double p2 = X * X + Y * Y + Z * Z;
    long double eps = is_photon ? sqrtl(p2) : sqrtl(1.0L + p2);
    long double ax = eps * Ex + (Y * Bz - Z * By);
    long double ay = eps * Ey + (Z * Bx - X * Bz);
    long double az = eps * Ez + (X * By - Y * Bx);
    long double pe = X * Ex + Y * Ey + Z * Ez;
    long double q = ax * ax + ay * ay + az * az - pe * pe;
    if (q < 0.0L) q = 0.0L;
    if (gamma_out) *gamma_out = (double)eps;
    return (double)(sqrtl(q) / (long double)E_s);
}

/* ------------------------------------------------------------------------ */
/* Boris push (Algorithm 1, the momentum update of every sub-step).          */
/* In code units (p in m c, E and B in m c omega / e, t in laser periods)    */
/* the Lorentz force reads dp/dt = 2 pi q (E + p x B / gamma), q = -1 for    */
/* an electron and +1 for a positron.  One step of length h with a = pi q h: */
/*   p- = p + a E;   gamma- = sqrt(1 + |p-|^2);   t = (a / gamma-) B;         */
/*   s = 2 t / (1 + |t|^2);   p' = p- + p- x t;   p+ = p- + p' x s;           */
/*   p(h) = p+ + a E                                                          */
/* (half an electric kick, a rotation about B by 2 atan|t|, half a kick).    */
/* ------------------------------------------------------------------------ */
void orc_boris64(int charge, double h, double p[3], const double E[3], const double B[3]) {
    const double a = ORC_PI * (double)charge * h;
    double m[3], t[3], s[3], q[3], r[3];
    for (int k = 0; k < 3; ++k) m[k] = p[k] + a * E[k];
    const double g = sqrt(1.0 + m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    for (int k = 0; k < 3; ++k) t[k] = a / g * B[k];
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int k = 0; k < 3; ++k) s[k] = 2.0 * t[k] / (1.0 + t2);
    q[0] = m[0] + (m[1] * t[2] - m[2] * t[1]);
    q[1] = m[1] + (m[2] * t[0] - m[0] * t[2]);
    q[2] = m[2] + (m[0] * t[1] - m[1] * t[0]);
    r[0] = m[0] + (q[1] * s[2] - q[2] * s[1]);
    r[1] = m[1] + (q[2] * s[0] - q[0] * s[2]);
    r[2] = m[2] + (q[0] * s[1] - q[1] * s[0]);
    for (int k = 0; k < 3; ++k) p[k] = r[k] + a * E[k];
}

/* The same step on the binary32 particle state, with t and s written over
 * one common denominator so that one division serves both:
 *   u = a B,  g^2 = 1 + |p-|^2,  w = g^2 + |u|^2,  D = g w,
 *   t = u (w / D) = u / g,        s = u (2 g^2 / D) = 2 t / (1 + |t|^2).
 * Every operation is IEEE binary32 with round-to-nearest, in this order
 * (the store holds the momentum in binary32, and the state after each
 * sub-step is a binary32 value); built with -ffp-contract=off, so no two
 * operations fuse.  Pinned to the binary64 form above. */
void orc_boris32(int charge, float h, float p[3], const float E[3], const float B[3]) {
    const float pi = (float)ORC_PI;
    const float ah = pi * h;
    const float a = charge < 0 ? -ah : ah;
    float m[3], u[3], t[3], s[3], q[3], r[3];
    for (int k = 0; k < 3; ++k) {
        const float kick = a * E[k];
        m[k] = p[k] + kick;
        u[k] = a * B[k];
    }
    const float m2 = (m[0] * m[0] + m[1] * m[1]) + m[2] * m[2];
    const float u2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    const float g2 = 1.0f + m2;
    const float g = sqrtf(g2);
    const float w = g2 + u2;
    const float R = 1.0f / (g * w);
    const float ct = w * R;
    const float cs = (2.0f * g2) * R;
    for (int k = 0; k < 3; ++k) {
        t[k] = ct * u[k];
        s[k] = cs * u[k];
    }
    q[0] = m[0] + (m[1] * t[2] - m[2] * t[1]);
    q[1] = m[1] + (m[2] * t[0] - m[0] * t[2]);
    q[2] = m[2] + (m[0] * t[1] - m[1] * t[0]);
    r[0] = m[0] + (q[1] * s[2] - q[2] * s[1]);
    r[1] = m[1] + (q[2] * s[0] - q[0] * s[2]);
    r[2] = m[2] + (q[0] * s[1] - q[1] * s[0]);
    for (int k = 0; k < 3; ++k) {
        const float kick = a * E[k];
        p[k] = r[k] + kick;
    }
}

/* ------------------------------------------------------------------------ */
/* Rate bounds, Sec. 3.1.1.  c = sqrt(3) R t / (pi gamma), b = 3 chi / 2.    */
/* ------------------------------------------------------------------------ */
/* The four pieces as printed: coefficient A_k of pi c b^{e_k} and exponent
 * e_k, plus 0.1 c b on every piece.  The tests may replace them through
 * orc_set_emission_bound (to check that their pins catch a mistyped value);
 * nothing else does. */
static const double ORC_BOUND_A[4] = {0.56, 0.45, 0.42, 0.55};
static const double ORC_BOUND_E[4] = {1.0, 11.0 / 12.0, 19.0 / 24.0, 2.0 / 3.0};
static double orc_bound_A[4] = {0.56, 0.45, 0.42, 0.55};
static double orc_bound_e[4] = {1.0, 11.0 / 12.0, 19.0 / 24.0, 2.0 / 3.0};
static double orc_bound_lin = 0.1;

/* Test hook: A, e (4 values each) and the linear coefficient; NULL A
 * restores the printed values. */
void orc_set_emission_bound(const double* A, const double* e, double lin) {
    for (int k = 0; k < 4; ++k) {
        orc_bound_A[k] = A ? A[k] : ORC_BOUND_A[k];
        orc_bound_e[k] = A ? e[k] : ORC_BOUND_E[k];
    }
    orc_bound_lin = A ? lin : 0.1;
}

double orc_bound_emission(double b, double c) {
    /* pieces [0, 0.1) [0.1, 0.5) [0.5, 10) [10, inf) */
    int k = b < 0.1 ? 0 : (b < 0.5 ? 1 : (b < 10.0 ? 2 : 3));
    double lead = orc_bound_A[k] * ORC_PI * c * pow(b, orc_bound_e[k]);   /* pow(b, 1) == b */
    return lead + orc_bound_lin * c * b;
}

double orc_bound_pair(double b, double c, double coeff) { return coeff * c * b; }

/* x -> 0 limit of 3 x^2 P(x^3) divided by c b^{2/3}: F(z) ~ C z^{1/3} with
 * C = 4 pi / (sqrt 3 Gamma(1/3) 2^{1/3}). */
static double orc_small_F1_coeff(void) {
    return 4.0 * ORC_PI / (ORC_SQRT3 * tgamma(1.0 / 3.0) * cbrt(2.0));
}

/* Emission acceptance function of Algorithm 1 (Eq. 1 with delta = x^3):
 *   3 x^2 P(x^3) = (c b / x) [ (1 - delta) F(z) + delta^2 G(z) ],
 *   z = delta / (b (1 - delta)),  c = sqrt(3) R h / (pi gamma). */
double orc_Pm(double b, double c, double x) {
    double delta = x * x * x;
    double omd = 1.0 - delta;
    double z = delta / (b * omd);
    double F = orc_F1(z), G = orc_F2(z);
    return (c * b / x) * (omd * F + delta * delta * G);
}

/* Pair acceptance function of Algorithm 2 (Eq. 2, bracket sign corrected):
 *   P_p(delta) = (c b / 3) [ G(z) - delta (1 - delta) F(z) ],
 *   z = 1 / (b delta (1 - delta)),  c = sqrt(3) R h / (pi gamma_photon). */
double orc_Pp(double b, double c, double delta) {
    double dd = delta * (1.0 - delta);
    double z = 1.0 / (b * dd);
    return (c * b / 3.0) * (orc_F2(z) - dd * orc_F1(z));
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [0,1] (Newton iteration on P_n).                  */
/* ------------------------------------------------------------------------ */
static void gauss_legendre01(int n, double* nodes, double* weights) {
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        nodes[i] = 0.5 * (1.0 - z);
        weights[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Composite Gauss-Legendre integral of the acceptance function over (0,1):
 * kind 0 -> int_0^1 3x^2 P(x^3) dx (emission), kind 1 -> int_0^1 P_p d delta
 * (pair).  Returned per unit c, i.e. the per-sub-step event probability is
 * c times this. */
double orc_total_per_c(int kind, double b, int panels, int order) {
    double nodes[64], weights[64];
    if (order > 64) order = 64;
    gauss_legendre01(order, nodes, weights);
    double sum = 0.0;
    for (int p = 0; p < panels; ++p) {
        double a = (double)p / panels, w = 1.0 / panels;
        for (int i = 0; i < order; ++i) {
            double x = a + w * nodes[i];
            double v = kind == 0 ? orc_Pm(b, 1.0, x) : orc_Pp(b, 1.0, x);
            sum += w * weights[i] * v;
        }
    }
    return sum;
}

/* ------------------------------------------------------------------------ */
/* Sub-step planner.                                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t seed;
    double dt;            /* global step, laser periods                  */
    double R;             /* alpha m c^2 / hbar, 1/period                */
    double E_s;           /* Schwinger field, code units                 */
    double p_max;         /* maximum per-sub-step event probability      */
    double pair_coeff;    /* coefficient of c b in the photon bound      */
    double tie_draw;      /* |y - P| <= tie_draw * P marks a draw as a tie */
    double tie_plan;      /* relative band on f/P_max that marks a tie   */
    uint32_t process_mask;/* 1 emission, 2 pair                          */
    int32_t cascade;      /* process children within the step            */
    int32_t recoil;       /* 0: events leave the parent unchanged (test) */
    int32_t threads;
    int32_t push;         /* 1: Boris push of e+- before every sub-step's draw */
    const uint32_t* first_N;  /* optional: at least this count for the first plan */
    int64_t first_N_rows;     /* ... of rows [0, first_N_rows) (one sub-step per cell) */
} orc_config;

typedef struct {
    uint64_t parent_id;
    uint64_t child_id[2];
    uint32_t s;           /* sub-step index of the event in this step    */
    uint32_t kind;        /* 1 emission, 2 pair                          */
    double delta;
    double chi;           /* parent chi at the event                     */
} orc_event;

typedef struct {
    uint64_t id;
    uint32_t s;           /* first sub-step whose outcome is uncertain   */
    uint32_t kind;        /* 1 draw near-tie, 2 plan near-tie            */
} orc_tie;

typedef struct {
    uint64_t substeps, emissions, pairs, children, guard_hits, plans;
    uint32_t max_N;
    int32_t status;
    int64_t required_capacity;
} orc_stats;

static uint32_t plan_count(const orc_config* cf, int is_photon, double b, double c,
                           double scale_b, double scale_q, int* guard) {
    double bb = b * scale_b;
    double f = is_photon ? orc_bound_pair(bb, c, cf->pair_coeff) : orc_bound_emission(bb, c);
    double q = f / cf->p_max * scale_q;
    double N = ceil(q);
    if (N < 1.0) N = 1.0;
    if (!is_photon) {
        double g = ceil(orc_small_F1_coeff() * c * pow(bb, 2.0 / 3.0) * scale_q);
        if (g > N) { N = g; if (guard) *guard = 1; }
    }
    if (N > 1073741824.0) N = 1073741824.0;   /* 2^30 */
    return (uint32_t)N;
}

/* ------------------------------------------------------------------------ */
/* Particle store (SoA, binary32 momenta and fields as in the workload).     */
/* ------------------------------------------------------------------------ */
typedef struct {
    float *px, *py, *pz, *Ex, *Ey, *Ez, *Bx, *By, *Bz, *w;
    uint64_t* id;
    uint8_t* type;        /* 0 e-, 1 e+, 2 photon, 3 removed             */
    int64_t count, capacity;
} orc_particles;

/* A pending unit of work: particle index, its remaining time and the
 * sub-step counter it starts from. */
typedef struct { int64_t idx; double t_rem; } orc_work;

typedef struct {
    orc_event* ev; int64_t n_ev, cap_ev;
    orc_tie* tie; int64_t n_tie, cap_tie;
} orc_log;

static void log_event(orc_log* L, const orc_event* e) {
    if (!L) return;
    if (L->n_ev == L->cap_ev) {
        L->cap_ev = L->cap_ev ? 2 * L->cap_ev : 1024;
        L->ev = (orc_event*)realloc(L->ev, (size_t)L->cap_ev * sizeof(orc_event));
    }
    L->ev[L->n_ev++] = *e;
}

static void log_tie(orc_log* L, uint64_t id, uint32_t s, uint32_t kind) {
    if (!L) return;
    if (L->n_tie == L->cap_tie) {
        L->cap_tie = L->cap_tie ? 2 * L->cap_tie : 256;
        L->tie = (orc_tie*)realloc(L->tie, (size_t)L->cap_tie * sizeof(orc_tie));
    }
    L->tie[L->n_tie].id = id; L->tie[L->n_tie].s = s; L->tie[L->n_tie].kind = kind;
    L->n_tie++;
}

/* Child rows produced while processing one particle. */
typedef struct {
    float px, py, pz; uint64_t id; uint8_t type; double t_rem;
    int64_t parent;   /* row of the parent (fields and weight are copied)  */
} orc_child;

typedef struct { orc_child* c; int64_t n, cap; } orc_childbuf;

static void push_child(orc_childbuf* B, const orc_child* c) {
    if (B->n == B->cap) {
        B->cap = B->cap ? 2 * B->cap : 64;
        B->c = (orc_child*)realloc(B->c, (size_t)B->cap * sizeof(orc_child));
    }
    B->c[B->n++] = *c;
}

/* Algorithms 1 and 2 for one particle over its remaining time t_rem.
 * Children go to `kids`; the particle's own row is updated in place. */
static void process_particle(const orc_config* cf, orc_particles* P, int64_t i, double t_rem,
                             uint32_t step, orc_stats* st, orc_log* L, orc_childbuf* kids) {
    uint8_t type = P->type[i];
    if (type > 2) return;
    int is_photon = (type == 2);
    if (is_photon && !(cf->process_mask & 2u)) return;
    if (!is_photon && !(cf->process_mask & 1u)) return;
    uint64_t id = P->id[i];
    int tied = 0;
    uint32_t s = 0;
    double px = P->px[i], py = P->py[i], pz = P->pz[i];
    const double Ex = P->Ex[i], Ey = P->Ey[i], Ez = P->Ez[i];
    const double Bx = P->Bx[i], By = P->By[i], Bz = P->Bz[i];
    const double k_sqrt3_pi = ORC_SQRT3 / ORC_PI;
    /* Algorithm 1 with the push: an electron (charge -1) or positron (+1) is
     * pushed before every draw.  A photon flies straight (Algorithm 2): its
     * momentum, and so chi, stays as it is. */
    const int push = cf->push && !is_photon;
    const int charge = type == 0 ? -1 : 1;
    const float fE[3] = {P->Ex[i], P->Ey[i], P->Ez[i]};
    const float fB[3] = {P->Bx[i], P->By[i], P->Bz[i]};

    while (t_rem > 0.0) {
        /* Algorithms 1/2, planning: sub-step for the remaining time. */
        double gamma;
        double chi = orc_chi(is_photon, px, py, pz, Ex, Ey, Ez, Bx, By, Bz, cf->E_s, &gamma);
        if (!(gamma > 0.0)) break;   /* a photon without momentum does nothing */
        double b = 1.5 * chi;
        double c_rem = k_sqrt3_pi * cf->R * t_rem / gamma;
        int guard = 0;
        uint32_t N = plan_count(cf, is_photon, b, c_rem, 1.0, 1.0, &guard);
        if (!tied) {
            /* a near-tie of the particle's own count */
            double eps = cf->tie_plan;
            uint32_t lo = plan_count(cf, is_photon, b, c_rem, 1.0 - eps, 1.0 - eps, NULL);
            uint32_t hi = plan_count(cf, is_photon, b, c_rem, 1.0 + eps, 1.0 + eps, NULL);
            uint32_t lo2 = plan_count(cf, is_photon, b, c_rem, 1.0 + eps, 1.0 - eps, NULL);
            uint32_t hi2 = plan_count(cf, is_photon, b, c_rem, 1.0 - eps, 1.0 + eps, NULL);
            if (lo != N || hi != N || lo2 != N || hi2 != N) { tied = 1; log_tie(L, id, s, 2); }
        }
        /* one sub-step per cell (as Algorithms 1/2 start): an initial
         * row's first plan takes its cell's count when that is larger (a
         * near-tie of the cell's count is the caller's to flag) */
        if (cf->first_N && s == 0 && i < cf->first_N_rows && cf->first_N[i] > N)
            N = cf->first_N[i];
        st->plans++;
        if (guard) st->guard_hits++;
        if (N > st->max_N) st->max_N = N;
        double h = t_rem / (double)N;
        double c_h = k_sqrt3_pi * cf->R * h / gamma;
        int event = 0;
        for (uint32_t k = 0; k < N; ++k) {
            /* with the push: move the momentum over this sub-step, then chi */
            double chi_k = chi, b_k = b, c_k = c_h;
            if (push) {
                float pf[3] = {(float)px, (float)py, (float)pz};
                orc_boris32(charge, (float)h, pf, fE, fB);
                px = pf[0]; py = pf[1]; pz = pf[2];
                double g;
                chi_k = orc_chi(0, px, py, pz, Ex, Ey, Ez, Bx, By, Bz, cf->E_s, &g);
                b_k = 1.5 * chi_k;
                c_k = k_sqrt3_pi * cf->R * h / g;
            }
            /* draw x, y for this sub-step */
            double x, y;
            orc_draw(cf->seed, id, step, s, &x, &y);
            st->substeps++;
            /* acceptance test */
            double P_acc = is_photon ? orc_Pp(b_k, c_k, x) : orc_Pm(b_k, c_k, x);
            if (!tied && fabs(y - P_acc) <= cf->tie_draw * P_acc) { tied = 1; log_tie(L, id, s, 1); }
            if (y < P_acc) {
                /* the event closes sub-step k */
                double t_after = (k + 1 == N) ? 0.0 : t_rem - (double)(k + 1) * h;
                orc_event e;
                memset(&e, 0, sizeof e);
                e.parent_id = id; e.s = s; e.chi = chi_k;
                orc_child_ids(cf->seed, id, step, s, e.child_id);
                if (!is_photon) {
                    double delta = x * x * x;
                    e.kind = 1; e.delta = delta;
                    orc_child ph;
                    ph.px = (float)(delta * px); ph.py = (float)(delta * py); ph.pz = (float)(delta * pz);
                    ph.id = e.child_id[0]; ph.type = 2; ph.t_rem = t_after; ph.parent = i;
                    push_child(kids, &ph);
                    if (cf->recoil) {
                        px = (double)(float)((1.0 - delta) * px);
                        py = (double)(float)((1.0 - delta) * py);
                        pz = (double)(float)((1.0 - delta) * pz);
                    }
                    st->emissions++;
                    st->children++;
                    e.child_id[1] = 0;
                    log_event(L, &e);
                } else {
                    double delta = x;
                    e.kind = 2; e.delta = delta;
                    orc_child el, po;
                    el.px = (float)(delta * px); el.py = (float)(delta * py); el.pz = (float)(delta * pz);
                    el.id = e.child_id[0]; el.type = 0; el.t_rem = t_after; el.parent = i;
                    po.px = (float)((1.0 - delta) * px); po.py = (float)((1.0 - delta) * py);
                    po.pz = (float)((1.0 - delta) * pz);
                    po.id = e.child_id[1]; po.type = 1; po.t_rem = t_after; po.parent = i;
                    push_child(kids, &el);
                    push_child(kids, &po);
                    st->pairs++;
                    st->children += 2;
                    log_event(L, &e);
                    if (cf->recoil) {
                        /* Algorithm 2: the decayed photon is deleted and stops */
                        P->type[i] = 3;
                        P->px[i] = (float)px; P->py[i] = (float)py; P->pz[i] = (float)pz;
                        return;
                    }
                }
                ++s;
                t_rem = t_after;
                event = 1;
                break;
            }
            ++s;
        }
        if (!event) t_rem = 0.0;
    }
    P->px[i] = (float)px; P->py[i] = (float)py; P->pz[i] = (float)pz;
}

/* Append the children of one particle to the store and, if they are to be
 * processed in this step, to the work list. */
static int append_children(const orc_config* cf, orc_particles* P, orc_childbuf* kids,
                           orc_work** work, int64_t* n_work, int64_t* cap_work, orc_stats* st) {
    for (int64_t k = 0; k < kids->n; ++k) {
        const orc_child* c = &kids->c[k];
        if (P->count >= P->capacity) {
            st->status = 3;
            st->required_capacity = P->count + (kids->n - k);
            return -1;
        }
        int64_t j = P->count++;
        P->px[j] = c->px; P->py[j] = c->py; P->pz[j] = c->pz;
        P->Ex[j] = P->Ex[c->parent]; P->Ey[j] = P->Ey[c->parent]; P->Ez[j] = P->Ez[c->parent];
        P->Bx[j] = P->Bx[c->parent]; P->By[j] = P->By[c->parent]; P->Bz[j] = P->Bz[c->parent];
        P->w[j] = P->w[c->parent];
        P->id[j] = c->id;
        P->type[j] = c->type;
        if (cf->cascade && c->t_rem > 0.0) {
            if (*n_work == *cap_work) {
                *cap_work = *cap_work ? 2 * *cap_work : 1024;
                *work = (orc_work*)realloc(*work, (size_t)*cap_work * sizeof(orc_work));
            }
            (*work)[*n_work].idx = j; (*work)[*n_work].t_rem = c->t_rem; (*n_work)++;
        }
    }
    kids->n = 0;
    return 0;
}

/* One global step for the whole store, single-threaded, particles in index
 * order and children in creation order (first in, first out).  Returns the
 * status (0 ok, 3 capacity exceeded). */
int orc_event_step(const orc_config* cf, orc_particles* P, uint32_t step, orc_stats* st,
                   orc_log* L) {
    memset(st, 0, sizeof *st);
    orc_childbuf kids = {0};
    orc_work* work = NULL;
    int64_t n_work = 0, cap_work = 0;
    int64_t n0 = P->count;
    for (int64_t i = 0; i < n0 && st->status == 0; ++i) {
        process_particle(cf, P, i, cf->dt, step, st, L, &kids);
        append_children(cf, P, &kids, &work, &n_work, &cap_work, st);
    }
    for (int64_t q = 0; q < n_work && st->status == 0; ++q) {
        process_particle(cf, P, work[q].idx, work[q].t_rem, step, st, L, &kids);
        append_children(cf, P, &kids, &work, &n_work, &cap_work, st);
    }
    free(kids.c);
    free(work);
    return st->status;
}

/* Multi-threaded variant used only to time the oracle on the host cores: the
 * particles are taken in chunks of ORC_CHUNK rows from a shared counter (so
 * that a clump of long plans does not fall on one thread), each chunk's
 * children are processed locally from a FIFO, and the chunks' children are
 * appended afterwards in chunk order.  No event log.  Emission and pairs as
 * configured. */
#define ORC_CHUNK 32
typedef struct {
    const orc_config* cf; orc_particles* P; int64_t n0; uint32_t step;
    int64_t* next; orc_childbuf* outs; orc_stats st;
} mt_job;

static void mt_chunk(mt_job* j, int64_t c, orc_childbuf* kids, orc_childbuf* fifo) {
    const int64_t begin = c * ORC_CHUNK;
    const int64_t end = begin + ORC_CHUNK < j->n0 ? begin + ORC_CHUNK : j->n0;
    fifo->n = 0;
    for (int64_t i = begin; i < end; ++i) {
        process_particle(j->cf, j->P, i, j->cf->dt, j->step, &j->st, NULL, kids);
        for (int64_t k = 0; k < kids->n; ++k) push_child(fifo, &kids->c[k]);
        kids->n = 0;
    }
    /* children are not written into the shared store by workers; a child
     * with remaining time is processed on a private one-row store */
    orc_childbuf* out = &j->outs[c];
    for (int64_t q = 0; q < fifo->n; ++q) {
        orc_child ch = fifo->c[q];
        if (j->cf->cascade && ch.t_rem > 0.0) {
            float px = ch.px, py = ch.py, pz = ch.pz, w = j->P->w[ch.parent];
            float Ex = j->P->Ex[ch.parent], Ey = j->P->Ey[ch.parent], Ez = j->P->Ez[ch.parent];
            float Bx = j->P->Bx[ch.parent], By = j->P->By[ch.parent], Bz = j->P->Bz[ch.parent];
            uint64_t id = ch.id; uint8_t type = ch.type;
            orc_particles one = {&px, &py, &pz, &Ex, &Ey, &Ez, &Bx, &By, &Bz, &w, &id, &type, 1, 1};
            process_particle(j->cf, &one, 0, ch.t_rem, j->step, &j->st, NULL, kids);
            for (int64_t k = 0; k < kids->n; ++k) {
                kids->c[k].parent = ch.parent;   /* same fields and weight */
                push_child(fifo, &kids->c[k]);
            }
            kids->n = 0;
            ch.px = px; ch.py = py; ch.pz = pz; ch.type = type;
        }
        push_child(out, &ch);
    }
}

static void* mt_worker(void* arg) {
    mt_job* j = (mt_job*)arg;
    memset(&j->st, 0, sizeof j->st);
    orc_childbuf kids = {0}, fifo = {0};
    const int64_t nchunks = (j->n0 + ORC_CHUNK - 1) / ORC_CHUNK;
    for (;;) {
        const int64_t c = __atomic_fetch_add(j->next, 1, __ATOMIC_RELAXED);
        if (c >= nchunks) break;
        mt_chunk(j, c, &kids, &fifo);
    }
    free(kids.c);
    free(fifo.c);
    return NULL;
}

int orc_event_step_mt(const orc_config* cf, orc_particles* P, uint32_t step, orc_stats* st) {
    int T = cf->threads < 1 ? 1 : (cf->threads > 256 ? 256 : cf->threads);
    pthread_t th[256];
    mt_job* jobs = (mt_job*)calloc((size_t)T, sizeof(mt_job));
    const int64_t n0 = P->count;
    const int64_t nchunks = (n0 + ORC_CHUNK - 1) / ORC_CHUNK;
    orc_childbuf* outs = (orc_childbuf*)calloc((size_t)(nchunks > 0 ? nchunks : 1), sizeof(orc_childbuf));
    int64_t next = 0;
    for (int t = 0; t < T; ++t) {
        jobs[t].cf = cf; jobs[t].P = P; jobs[t].step = step; jobs[t].n0 = n0;
        jobs[t].next = &next; jobs[t].outs = outs;
        pthread_create(&th[t], NULL, mt_worker, &jobs[t]);
    }
    memset(st, 0, sizeof *st);
    for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < T; ++t) {
        orc_stats* s = &jobs[t].st;
        st->substeps += s->substeps; st->emissions += s->emissions; st->pairs += s->pairs;
        st->children += s->children; st->guard_hits += s->guard_hits; st->plans += s->plans;
        if (s->max_N > st->max_N) st->max_N = s->max_N;
    }
    for (int64_t c = 0; c < nchunks; ++c) {
        for (int64_t k = 0; k < outs[c].n && st->status == 0; ++k) {
            orc_child* ch = &outs[c].c[k];
            if (P->count >= P->capacity) { st->status = 3; st->required_capacity = P->count + 1; break; }
            int64_t j = P->count++;
            P->px[j] = ch->px; P->py[j] = ch->py; P->pz[j] = ch->pz;
            P->Ex[j] = P->Ex[ch->parent]; P->Ey[j] = P->Ey[ch->parent]; P->Ez[j] = P->Ez[ch->parent];
            P->Bx[j] = P->Bx[ch->parent]; P->By[j] = P->By[ch->parent]; P->Bz[j] = P->Bz[ch->parent];
            P->w[j] = P->w[ch->parent]; P->id[j] = ch->id; P->type[j] = ch->type;
        }
        free(outs[c].c);
    }
    free(outs);
    free(jobs);
    return st->status;
}

void orc_log_free(orc_log* L) {
    free(L->ev); free(L->tie);
    L->ev = NULL; L->tie = NULL; L->n_ev = L->cap_ev = L->n_tie = L->cap_tie = 0;
}

/* Plan query for tests: N, the bound f, chi and gamma of one particle. */
uint32_t orc_plan(const orc_config* cf, int is_photon, double px, double py, double pz,
                  double Ex, double Ey, double Ez, double Bx, double By, double Bz,
                  double t_rem, double* chi_out, double* gamma_out, double* f_out) {
    double gamma;
    double chi = orc_chi(is_photon, px, py, pz, Ex, Ey, Ez, Bx, By, Bz, cf->E_s, &gamma);
    double b = 1.5 * chi;
    double c = ORC_SQRT3 / ORC_PI * cf->R * t_rem / gamma;
    if (chi_out) *chi_out = chi;
    if (gamma_out) *gamma_out = gamma;
    if (f_out) *f_out = is_photon ? orc_bound_pair(b, c, cf->pair_coeff) : orc_bound_emission(b, c);
    return plan_count(cf, is_photon, b, c, 1.0, 1.0, NULL);
}
