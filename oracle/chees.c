/*
 * chees.c -- oracle ChEES trajectory-length adaptation (Sec. 2.3, Algorithm 2).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 * Pins: the per-particle estimate against a finite difference in log t of the
 * sample ChEES criterion on tiny inputs; Adam and the moving average against
 * hand-computed sequences (tests/test_oracle_chees.py).
 * The Adam constants are not given by the paper: parity unpinned for their
 * values (the recurrences themselves are pinned).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>

int oracle_chees_gradient(const double* theta0, const double* theta1, const double* p,
                          const double* l, const double* alpha, int64_t N, int64_t D,
                          double* ghat, double* g_per_particle) {
    double* m0 = (double*)calloc((size_t)D, sizeof(double));
    double* m1 = (double*)calloc((size_t)D, sizeof(double));
    /* Unweighted population means of the previous and proposed states. */
    for (int64_t j = 0; j < N; ++j)
        for (int64_t d = 0; d < D; ++d) {
            m0[d] += theta0[j * D + d];
            m1[d] += theta1[j * D + d];
        }
    for (int64_t d = 0; d < D; ++d) {
        m0[d] /= (double)N;
        m1[d] /= (double)N;
    }
    double num = 0.0, den = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        double sq0 = 0.0, sq1 = 0.0, proj = 0.0;
        for (int64_t d = 0; d < D; ++d) {
            double e0 = theta0[j * D + d] - m0[d];
            double e1 = theta1[j * D + d] - m1[d];
            sq0 += e0 * e0;
            sq1 += e1 * e1;
            proj += e1 * p[j * D + d];
        }
        double gj = l[j] * (sq1 - sq0) * proj;
        if (g_per_particle) g_per_particle[j] = gj;
        num += alpha[j] * gj;
        den += alpha[j];
    }
    free(m0);
    free(m1);
    if (!(den > 0.0)) return 0;
    double g = num / den;
    if (!isfinite(g)) return 0;
    *ghat = g;
    return 1;
}

void oracle_chees_adam(oracle_chees_state* s, double ghat, double lr, double b1, double b2,
                       double adam_eps, double eps, int32_t max_steps) {
    /* Adam (Kingma & Ba 2015) as gradient ASCENT on log L: ChEES is maximised. */
    s->t += 1;
    s->m = b1 * s->m + (1.0 - b1) * ghat;
    s->v = b2 * s->v + (1.0 - b2) * ghat * ghat;
    double mhat = s->m / (1.0 - pow(b1, (double)s->t));
    double vhat = s->v / (1.0 - pow(b2, (double)s->t));
    s->log_L += lr * mhat / (sqrt(vhat) + adam_eps);
    double lo = log(eps), hi = log((double)max_steps * eps);
    if (s->log_L < lo) s->log_L = lo;
    if (s->log_L > hi) s->log_L = hi;
}

double oracle_harmonic_mean_alpha(const double* alpha, int64_t N) {
    /* N / sum_j 1/alpha_j; a zero acceptance makes the harmonic mean 0 */
    double inv = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        if (!(alpha[j] > 0.0)) return 0.0;
        inv += 1.0 / alpha[j];
    }
    return (double)N / inv;
}

double oracle_step_size_update(double eps, const double* alpha, int64_t N, double rate, double target) {
    const double ah = oracle_harmonic_mean_alpha(alpha, N);
    return exp(log(eps) + rate * (ah - target));
}
