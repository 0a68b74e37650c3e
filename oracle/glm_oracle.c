/*
 * Plain FP64 CPU oracle for the Bayesian logistic-regression log-posterior
 * and its gradient (Mahani & Sharabiani, "SIMD Parallel MCMC Sampling with
 * Applications for Big-Data Bayesian Analytics").
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code. It shares no code, header,
 * table or helper with the CUDA library; it is a slow, obviously-correct
 * restatement of the paper's definitions in single-threaded loops:
 *
 *   log-likelihood  (§3.1.1, eq-loglike-binlogit)
 *       L(b) = - sum_n { (1 - y_n) x_n.b + log(1 + exp(-x_n.b)) }
 *   gradient        (§4.2, eq-grad-expanded / eq-grad-compact)
 *       g_L(b) = sum_n f_n'(x_n.b) x_n = X^t g_f,   g_f,n = y_n - 1/(1 + exp(-x_n.b))
 *   prior           (§3.1.1: "multivariate Gaussian"; read as N(0, s^2 I),
 *                    normalising constant included)
 *   HB group term   (§4.1, the per-group L_m(b_m)) with prior N(mu, tau^2 I)
 *   random-walk Metropolis consumer (§2.2/§3.4.4: the sampler calls the
 *       log-posterior once per step)
 *
 * Numerical readings: log(1 + exp(-e)) is evaluated without overflow
 * (for e < 0 it is -e + log1p(exp(e))), and 1/(1 + exp(-e)) is evaluated as
 * exp(e)/(1 + exp(e)) for e < 0. Both are the same real numbers as the
 * paper's expressions. Sums run in row order, j ascending, in FP64.
 *
 * Parity is pinned by the oracle tests (closed forms at b = 0, an
 * intercept-only closed form, extended-precision brute force of the Bernoulli
 * likelihood, central finite differences, symmetries, the Gaussian log-density
 * from scipy, quadrature of a 1-D posterior for the Metropolis chain, and
 * library/format-definition cases for the quantisers).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

#define ORACLE_LN_2PI 1.8378770664093454835606594728112

/* log(1 + exp(-e)), written so that it never overflows. */
static double log1p_exp_neg(double e)
{
    if (e >= 0.0)
        return log1p(exp(-e));
    return -e + log1p(exp(e));
}

/* 1 / (1 + exp(-e)) without overflow. */
static double logistic(double e)
{
    if (e >= 0.0)
        return 1.0 / (1.0 + exp(-e));
    double t = exp(e);
    return t / (1.0 + t);
}

/*
 * Likelihood part of one group of rows [r0, r1) at coefficient vector b.
 * Adds sum_n ell_n to *f and sum_n g_f,n x_n to g[0..P-1].
 */
static void loglik_rows(const double *X, int64_t ld, int32_t P,
                        const uint8_t *y, int64_t r0, int64_t r1,
                        const double *b, double *f, double *g)
{
    for (int64_t n = r0; n < r1; ++n) {
        const double *x = X + n * ld;
        double eta = 0.0;                       /* LA map: x_n^t b */
        for (int32_t j = 0; j < P; ++j)
            eta += x[j] * b[j];
        double yn = (double)y[n];
        /* TR map: the paper's per-row term and its derivative f_n' */
        double ell = -((1.0 - yn) * eta + log1p_exp_neg(eta));
        double gf = yn - logistic(eta);
        *f += ell;
        for (int32_t j = 0; j < P; ++j)         /* second LA map: g += g_f,n x_n */
            g[j] += gf * x[j];
    }
}

/*
 * f_k = L(b_k) + log N(b_k | 0, s^2 I),  g_k = g_L(b_k) - b_k / s^2
 * for k = 0..K-1. X is N x ld row-major (first P columns used), beta is K x P.
 * Returns 0, or -1 on a bad argument.
 */
int oracle_logpost_grad(const double *X, int64_t N, int32_t P, int64_t ld,
                        const uint8_t *y, const double *beta, int32_t K,
                        double prior_sigma, double *f_out, double *g_out)
{
    if (N < 0 || P < 1 || ld < P || K < 1 || !(prior_sigma > 0.0))
        return -1;
    double s2 = prior_sigma * prior_sigma;
    for (int32_t k = 0; k < K; ++k) {
        const double *b = beta + (int64_t)k * P;
        double *g = g_out + (int64_t)k * P;
        double f = 0.0;
        for (int32_t j = 0; j < P; ++j)
            g[j] = 0.0;
        loglik_rows(X, ld, P, y, 0, N, b, &f, g);
        double bb = 0.0;
        for (int32_t j = 0; j < P; ++j)
            bb += b[j] * b[j];
        f += -bb / (2.0 * s2) - 0.5 * (double)P * (ORACLE_LN_2PI + log(s2));
        for (int32_t j = 0; j < P; ++j)
            g[j] -= b[j] / s2;
        f_out[k] = f;
    }
    return 0;
}

/*
 * Likelihood-only partial sums over rows [r0, r1) (no prior): the quantity a
 * row shard contributes before the cross-shard sum.
 */
int oracle_loglik_partial(const double *X, int64_t r0, int64_t r1, int32_t P,
                          int64_t ld, const uint8_t *y, const double *beta,
                          int32_t K, double *f_out, double *g_out)
{
    if (r0 < 0 || r1 < r0 || P < 1 || ld < P || K < 1)
        return -1;
    for (int32_t k = 0; k < K; ++k) {
        double f = 0.0;
        double *g = g_out + (int64_t)k * P;
        for (int32_t j = 0; j < P; ++j)
            g[j] = 0.0;
        loglik_rows(X, ld, P, y, r0, r1, beta + (int64_t)k * P, &f, g);
        f_out[k] = f;
    }
    return 0;
}

/*
 * Hierarchical-Bayes batch (§4.1): group m owns rows [off[m], off[m+1]) and
 * coefficient vector b_m; its conditional log-posterior is
 *   L_m(b_m) + log N(b_m | mu, tau^2 I)
 * with gradient g_L,m(b_m) - (b_m - mu) / tau^2.
 */
int oracle_logpost_grad_grouped(const double *X, int32_t P, int64_t ld,
                                const uint8_t *y, const int64_t *off, int32_t G,
                                const double *beta, const double *mu, double tau,
                                double *f_out, double *g_out)
{
    if (P < 1 || ld < P || G < 1 || !(tau > 0.0))
        return -1;
    double t2 = tau * tau;
    for (int32_t m = 0; m < G; ++m) {
        if (off[m + 1] < off[m])
            return -1;
        const double *b = beta + (int64_t)m * P;
        double *g = g_out + (int64_t)m * P;
        double f = 0.0;
        for (int32_t j = 0; j < P; ++j)
            g[j] = 0.0;
        loglik_rows(X, ld, P, y, off[m], off[m + 1], b, &f, g);
        double dd = 0.0;
        for (int32_t j = 0; j < P; ++j) {
            double d = b[j] - mu[j];
            dd += d * d;
            g[j] -= d / t2;
        }
        f += -dd / (2.0 * t2) - 0.5 * (double)P * (ORACLE_LN_2PI + log(t2));
        f_out[m] = f;
    }
    return 0;
}

/*
 * K independent random-walk Metropolis chains, n_steps each.
 * Chain state b is FP32 (as stored on the device). Step t proposes
 *   b'_j = fmaf(step, z[t][k][j], b_j)          (single rounding, FP32)
 * evaluates f(b') in FP64 on the FP32 values, and accepts iff
 *   log_u[t][k] < f(b') - f(b)                   (FP64 comparison).
 * Outputs (each may be NULL): samples[t][k][:] = state after step t,
 * accept[t][k], logpost[t][k] = f(state after step t),
 * log_alpha[t][k] = f(b') - f(b). beta_state (K x P) and f_state (K) are
 * updated in place; f_state is computed first when init_f != 0.
 */
int oracle_rwm(const double *X, int64_t N, int32_t P, int64_t ld,
               const uint8_t *y, double prior_sigma, int32_t K, int32_t n_steps,
               float step, const float *z, const double *log_u,
               float *beta_state, double *f_state, int32_t init_f,
               float *samples, uint8_t *accept, double *logpost,
               double *log_alpha)
{
    if (N < 0 || P < 1 || ld < P || K < 1 || n_steps < 0)
        return -1;
    double *b = (double *)malloc(sizeof(double) * (size_t)P);
    double *g = (double *)malloc(sizeof(double) * (size_t)P);
    float *prop = (float *)malloc(sizeof(float) * (size_t)P);
    if (!b || !g || !prop) {
        free(b); free(g); free(prop);
        return -1;
    }
    for (int32_t k = 0; k < K; ++k) {
        float *state = beta_state + (int64_t)k * P;
        if (init_f) {
            for (int32_t j = 0; j < P; ++j)
                b[j] = (double)state[j];
            oracle_logpost_grad(X, N, P, ld, y, b, 1, prior_sigma, &f_state[k], g);
        }
    }
    for (int32_t t = 0; t < n_steps; ++t) {
        for (int32_t k = 0; k < K; ++k) {
            float *state = beta_state + (int64_t)k * P;
            const float *zz = z + ((int64_t)t * K + k) * P;
            for (int32_t j = 0; j < P; ++j) {
                prop[j] = fmaf(step, zz[j], state[j]);
                b[j] = (double)prop[j];
            }
            double fp;
            oracle_logpost_grad(X, N, P, ld, y, b, 1, prior_sigma, &fp, g);
            double la = fp - f_state[k];
            int acc = log_u[(int64_t)t * K + k] < la;
            if (acc) {
                memcpy(state, prop, sizeof(float) * (size_t)P);
                f_state[k] = fp;
            }
            int64_t o = (int64_t)t * K + k;
            if (samples)
                memcpy(samples + o * P, state, sizeof(float) * (size_t)P);
            if (accept)
                accept[o] = (uint8_t)acc;
            if (logpost)
                logpost[o] = f_state[k];
            if (log_alpha)
                log_alpha[o] = la;
        }
    }
    free(b); free(g); free(prop);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Reduced-precision storage of X (the storage formats, not the paper's):
 *   BF16: the nearest bfloat16 to each FP32 value, ties to even.
 *   FP8 E4M3 (OCP 8-bit floating point, "E4M3FN": bias 7, 3 mantissa bits,
 *   no infinities, max finite 448, NaN = S.1111.111) with one power-of-two
 *   scale per column: s_j = smallest 2^e with 448 * 2^e >= max_n |x_nj|
 *   (s_j = 1 for an all-zero column), q_nj = nearest E4M3 to x_nj / s_j,
 *   ties to even, saturating to +-448.
 * ------------------------------------------------------------------------- */

static uint32_t f32_bits(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    return u;
}

void oracle_bf16_from_f32(const float *in, int64_t n, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u = f32_bits(in[i]);
        if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) {
            out[i] = (uint16_t)((u >> 16) | 0x0040u);      /* quiet NaN */
            continue;
        }
        uint32_t lsb = (u >> 16) & 1u;
        u += 0x7FFFu + lsb;                                  /* ties to even */
        out[i] = (uint16_t)(u >> 16);
    }
}

void oracle_bf16_to_f64(const uint16_t *in, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u = (uint32_t)in[i] << 16;
        float f;
        memcpy(&f, &u, 4);
        out[i] = (double)f;
    }
}

/* Round-half-even of a non-negative double that is an exact multiple of 1/2. */
static double round_half_even(double a)
{
    double fl = floor(a);
    double d = a - fl;
    if (d > 0.5)
        return fl + 1.0;
    if (d < 0.5)
        return fl;
    return (fmod(fl, 2.0) == 0.0) ? fl : fl + 1.0;
}

/* Encode a finite double v (already divided by the column scale) as E4M3. */
static uint8_t e4m3_encode(double v)
{
    uint8_t sign = signbit(v) ? 0x80u : 0x00u;
    double a = fabs(v);
    if (a == 0.0)
        return sign;
    int ex;
    frexp(a, &ex);                 /* a = m * 2^ex, m in [0.5, 1) */
    int e = ex - 1;                /* a in [2^e, 2^(e+1)) */
    if (e < -6)
        e = -6;                    /* subnormals share the quantum of binade -6 */
    double quantum = ldexp(1.0, e - 3);          /* 3 mantissa bits */
    double nr = round_half_even(a / quantum);    /* exact: power-of-two division */
    if (nr * quantum > 448.0)
        return (uint8_t)(sign | 0x7Eu);          /* saturate to the max finite, 448 */
    if (nr < 8.0)                                /* subnormal: 0.mmm * 2^-6 */
        return (uint8_t)(sign | (uint8_t)nr);
    if (nr == 16.0) {                            /* rounded up into the next binade */
        nr = 8.0;
        e += 1;
    }
    uint8_t field = (uint8_t)(e + 7);            /* exponent bias 7 */
    uint8_t mant = (uint8_t)(nr - 8.0);
    return (uint8_t)(sign | (uint8_t)(field << 3) | mant);
}

double oracle_e4m3_value(uint8_t q)
{
    int s = (q >> 7) & 1;
    int E = (q >> 3) & 0xF;
    int M = q & 7;
    double v;
    if (E == 15 && M == 7)
        return NAN;
    if (E == 0)
        v = ldexp((double)M, -9);
    else
        v = ldexp((double)(8 + M), E - 10);
    return s ? -v : v;
}

uint8_t oracle_e4m3_from_f64(double v)
{
    return e4m3_encode(v);
}

/* Smallest power of two s with 448 * s >= amax (s = 1 when amax == 0), but
 * not below 2^-126 so that s is a normal FP32 number. Every comparison is
 * exact: 448 * 2^e is representable. */
double oracle_e4m3_column_scale(double amax)
{
    if (!(amax > 0.0))
        return 1.0;
    int ex;
    frexp(amax, &ex);              /* amax in [2^(ex-1), 2^ex) */
    int e = ex - 10;               /* 448 * 2^(ex-10) < 2^(ex-1) <= amax */
    while (448.0 * ldexp(1.0, e) < amax)
        ++e;
    if (e < -126)                  /* keep the scale a normal FP32 number */
        e = -126;
    return ldexp(1.0, e);
}

/*
 * X (N x ld_in, FP32, first P columns) -> Q (N x ld_q, E4M3 bytes, padding
 * columns zero) and scale[0..P-1] (FP32 powers of two).
 */
int oracle_quantize_e4m3(const float *X, int64_t N, int32_t P, int64_t ld_in,
                         uint8_t *Q, int64_t ld_q, float *scale)
{
    if (N < 0 || P < 1 || ld_in < P || ld_q < P)
        return -1;
    for (int32_t j = 0; j < P; ++j) {
        double amax = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            double a = fabs((double)X[n * ld_in + j]);
            if (a > amax)
                amax = a;
        }
        scale[j] = (float)oracle_e4m3_column_scale(amax);
    }
    for (int64_t n = 0; n < N; ++n) {
        for (int64_t j = 0; j < ld_q; ++j) {
            uint8_t q = 0;
            if (j < P)
                q = e4m3_encode((double)X[n * ld_in + j] / (double)scale[j]);
            Q[n * ld_q + j] = q;
        }
    }
    return 0;
}
