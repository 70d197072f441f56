/*
 * weights.c -- oracle weight normalisation, ESS and fixed-point resampling.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 * Pins: logsumexp against scipy and the special cases ESS = N (equal weights)
 * and ESS = 1 (one-hot); resampling offspring bounds, conservation, and the
 * exact expectation over every distinct U (tests/test_oracle_weights.py).
 */
#include "oracle.h"
#include <math.h>

void oracle_normalise(const double* logw, int64_t N, double* lse, double* ess, double* W) {
    /* Normalised weights w_j / sum w (Sec. 3) computed through the maximum so
     * that exp never overflows; ESS = 1 / sum W_j^2. */
    double m = -INFINITY;
    for (int64_t j = 0; j < N; ++j)
        if (logw[j] > m) m = logw[j];
    if (m == -INFINITY) {
        if (lse) *lse = -INFINITY;
        if (ess) *ess = 0.0;
        if (W)
            for (int64_t j = 0; j < N; ++j) W[j] = 0.0;
        return;
    }
    double s = 0.0;
    for (int64_t j = 0; j < N; ++j) s += exp(logw[j] - m);
    double L = m + log(s);
    double s2 = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        double wj = exp(logw[j] - L);
        if (W) W[j] = wj;
        s2 += wj * wj;
    }
    if (lse) *lse = L;
    if (ess) *ess = 1.0 / s2;
}

static int32_t ceil_log2(int64_t N) {
    int32_t c = 0;
    while (((int64_t)1 << c) < N) ++c;
    return c;
}

int32_t oracle_quantise(const double* W, int64_t N, uint64_t* q) {
    int32_t S = 62 - ceil_log2(N);
    double scale = ldexp(1.0, S);
    for (int64_t j = 0; j < N; ++j) {
        double v = W[j] * scale;
        q[j] = (v > 0.0) ? (uint64_t)v : 0u;   /* truncation = floor for v >= 0 */
    }
    return S;
}

uint64_t oracle_systematic(const uint64_t* q, int64_t N, uint64_t r64, int32_t* ancestors) {
    /* Systematic resampling: one uniform offset shared by N evenly spaced
     * pointers.  In integers, pointer i sits at (i T + U) / (N T) of the mass
     * and particle j owns the cumulative interval (C_{j-1}, C_j] / T. */
    uint64_t T = 0;
    for (int64_t j = 0; j < N; ++j) T += q[j];
    if (T == 0) return 0;
    uint64_t U = (uint64_t)(((unsigned __int128)r64 * (unsigned __int128)T) >> 64);
    int64_t j = 0;
    uint64_t C = q[0];
    for (int64_t i = 0; i < N; ++i) {
        uint64_t P = (uint64_t)i * T + U;
        while ((uint64_t)N * C <= P) {
            ++j;
            C += q[j];
        }
        ancestors[i] = (int32_t)j;
    }
    return T;
}

void oracle_multinomial(const uint64_t* q, int64_t N, const uint64_t* u64, int32_t* ancestors) {
    uint64_t T = 0;
    for (int64_t j = 0; j < N; ++j) T += q[j];
    for (int64_t i = 0; i < N; ++i) {
        uint64_t P = (uint64_t)(((unsigned __int128)u64[i] * (unsigned __int128)T) >> 64);
        uint64_t C = 0;
        int64_t j = 0;
        for (; j < N; ++j) {
            C += q[j];
            if (C > P) break;
        }
        ancestors[i] = (int32_t)(j < N ? j : N - 1);
    }
}

void oracle_moments(const double* theta, const double* logw, int64_t N, int64_t D,
                    double* mean, double* var) {
    /* Realised estimates sum_j W_j f(theta_j) (Sec. 3) for f = theta and
     * f = (theta - mean)^2.  A particle of zero weight is left out: its
     * position may be non-finite (the end of a divergent trajectory). */
    double lse;
    oracle_normalise(logw, N, &lse, 0, 0);
    for (int64_t d = 0; d < D; ++d) {
        double m = 0.0;
        for (int64_t j = 0; j < N; ++j)
            if (logw[j] > -INFINITY) m += exp(logw[j] - lse) * theta[j * D + d];
        double v = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (!(logw[j] > -INFINITY)) continue;
            double e = theta[j * D + d] - m;
            v += exp(logw[j] - lse) * e * e;
        }
        mean[d] = m;
        if (var) var[d] = v;
    }
}
