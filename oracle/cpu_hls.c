/*
 * Multi-core FP64 CPU baseline: the paper's own CPU design for the
 * log-posterior and its gradient, restated in plain C with OpenMP.
 *
 * TIMED BASELINE ONLY, like the oracle beside it: the benchmark's
 * cpu_baseline leg and the tests call it; the CUDA library never does, and it
 * shares no code with it. It is not the oracle: tests check it against the
 * oracle (glm_oracle.c), which stays the definition.
 *
 * What it follows:
 * - §3.4.1 partial loop fusion (PLF): the rows are split statically into one
 *   contiguous block per thread, and each thread runs the whole pipeline
 *   (LA map, TR map, second LA map) over its own block.
 * - §4.2.1 cache fusion: within its block a thread walks chunks of rows small
 *   enough to stay in cache; for each chunk it forms eta = X beta, applies the
 *   transformation (ell and the residual r, in the stable forms the oracle
 *   uses), and adds r x_n into its gradient while the chunk's rows are still
 *   cached, so X is read from memory once per evaluation.
 * - §4.2.2: every thread keeps a private gradient and log-likelihood and
 *   combines them into the shared result once, at the end.
 * - §3.1.1 / §4.2: Gaussian prior N(0, sigma^2 I) added once after the combine.
 * NUMA placement (§3.4.2) is left to the operating system's first touch.
 * Several coefficient vectors share each cached chunk (the chunk is read
 * once for all K vectors).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HLS_CHUNK 128                 /* rows per cache-fused chunk */
#define HLS_LN_2PI 1.8378770664093454835606594728112

/* log(1 + e^{-|v|}) + max(-v, 0) = log(1 + e^{-v}), overflow-free */
static double softplus_neg(double v)
{
    return (v < 0.0 ? -v : 0.0) + log1p(exp(-fabs(v)));
}

/* 1 / (1 + e^{-v}) without overflow */
static double logistic(double v)
{
    if (v >= 0.0)
        return 1.0 / (1.0 + exp(-v));
    double e = exp(v);
    return e / (1.0 + e);
}

int hls_logpost_grad(const double *X, int64_t N, int32_t P, int64_t ld, const uint8_t *y,
                     const double *beta, int32_t K, double prior_sigma, int32_t threads,
                     double *f_out, double *g_out)
{
    if (N < 0 || P < 1 || ld < P || K < 1 || !(prior_sigma > 0.0) || threads < 1)
        return -1;
    for (int32_t k = 0; k < K; ++k)
        f_out[k] = 0.0;
    memset(g_out, 0, sizeof(double) * (size_t)K * (size_t)P);
    int bad = 0;
#pragma omp parallel num_threads(threads)
    {
        const int t = omp_get_thread_num();
        const int T = omp_get_num_threads();
        const int64_t r0 = N * t / T;
        const int64_t r1 = N * (t + 1) / T;
        double *gp = calloc((size_t)K * (size_t)P, sizeof(double));
        double *fp = calloc((size_t)K, sizeof(double));
        double *eta = malloc(sizeof(double) * HLS_CHUNK);
        if (!gp || !fp || !eta) {
#pragma omp atomic write
            bad = 1;
        } else {
            for (int64_t c0 = r0; c0 < r1; c0 += HLS_CHUNK) {
                const int64_t c1 = (c0 + HLS_CHUNK < r1) ? c0 + HLS_CHUNK : r1;
                const int m = (int)(c1 - c0);
                for (int32_t k = 0; k < K; ++k) {
                    const double *b = beta + (int64_t)k * P;
                    double *g = gp + (int64_t)k * P;
                    /* LA map 1 over the chunk */
                    for (int i = 0; i < m; ++i) {
                        const double *x = X + (c0 + i) * ld;
                        double s = 0.0;
                        for (int32_t j = 0; j < P; ++j)
                            s += x[j] * b[j];
                        eta[i] = s;
                    }
                    /* TR map; eta is overwritten by the residual */
                    double fs = 0.0;
                    for (int i = 0; i < m; ++i) {
                        const double v = eta[i];
                        const double yv = (double)y[c0 + i];
                        fs -= (1.0 - yv) * v + softplus_neg(v);
                        eta[i] = yv - logistic(v);
                    }
                    fp[k] += fs;
                    /* LA map 2 from the same (cached) rows */
                    for (int i = 0; i < m; ++i) {
                        const double *x = X + (c0 + i) * ld;
                        const double r = eta[i];
                        for (int32_t j = 0; j < P; ++j)
                            g[j] += r * x[j];
                    }
                }
            }
            /* one combine per thread */
#pragma omp critical
            {
                for (int32_t k = 0; k < K; ++k) {
                    f_out[k] += fp[k];
                    for (int32_t j = 0; j < P; ++j)
                        g_out[(int64_t)k * P + j] += gp[(int64_t)k * P + j];
                }
            }
        }
        free(gp);
        free(fp);
        free(eta);
    }
    if (bad)
        return -2;
    const double s2 = prior_sigma * prior_sigma;
    for (int32_t k = 0; k < K; ++k) {
        const double *b = beta + (int64_t)k * P;
        double bb = 0.0;
        for (int32_t j = 0; j < P; ++j) {
            bb += b[j] * b[j];
            g_out[(int64_t)k * P + j] -= b[j] / s2;
        }
        f_out[k] += -bb / (2.0 * s2) - 0.5 * (double)P * (HLS_LN_2PI + log(s2));
    }
    return 0;
}

int hls_max_threads(void)
{
    return omp_get_num_procs();
}
