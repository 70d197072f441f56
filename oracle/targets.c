/*
 * targets.c -- oracle log-targets log pi(theta) = log p(x|theta) + log q0(theta)
 * (Sec. 2) and their gradients, in FP64, one particle at a time.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 * Pins: central finite differences of log pi (tests/test_oracle_targets.py);
 * closed-form evidence of the Gaussian and linear-Gaussian targets through the
 * whole sampler (tests/test_oracle_smc.py).
 */
#include "oracle.h"
#include <math.h>
#include <string.h>

static const double LOG_2PI = 1.8378770664093454835606594728112;

/* log(1 + e^x) without overflow. */
static double softplus(double x) {
    return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

/* 1 / (1 + e^-x) without overflow. */
static double sigmoid(double x) {
    if (x >= 0.0) return 1.0 / (1.0 + exp(-x));
    double e = exp(x);
    return e / (1.0 + e);
}

/* Dense Gaussian: c - 1/2 (theta - mu)' P (theta - mu); gradient -P (theta - mu). */
static double gauss_dense(const oracle_target* t, const double* th, double* g) {
    const int64_t D = t->D;
    double quad = 0.0;
    for (int64_t a = 0; a < D; ++a) {
        double Pd = 0.0;
        for (int64_t b = 0; b < D; ++b) Pd += t->P[a * D + b] * (th[b] - t->mu[b]);
        quad += (th[a] - t->mu[a]) * Pd;
        if (g) g[a] = -Pd;
    }
    return t->c - 0.5 * quad;
}

/* Logistic regression (Sec. 4, German Credit): y_i ~ Bernoulli(sigmoid(x_i' theta)),
 * prior theta ~ N(0, tau^2 I).  log p(y|theta) = sum_i y_i eta_i - log(1 + e^eta_i);
 * gradient X'(y - sigmoid(eta)) - theta / tau^2. */
static double logistic(const oracle_target* t, const double* th, double* g) {
    const int64_t D = t->D, n = t->n;
    const double tau = t->hyper[0];
    double lp = 0.0;
    if (g) memset(g, 0, (size_t)D * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        const double* x = t->X + i * D;
        double eta = 0.0;
        for (int64_t d = 0; d < D; ++d) eta += x[d] * th[d];
        lp += t->y[i] * eta - softplus(eta);
        if (g) {
            double r = t->y[i] - sigmoid(eta);
            for (int64_t d = 0; d < D; ++d) g[d] += r * x[d];
        }
    }
    double sq = 0.0;
    for (int64_t d = 0; d < D; ++d) {
        sq += th[d] * th[d];
        if (g) g[d] -= th[d] / (tau * tau);
    }
    lp += -0.5 * sq / (tau * tau) - 0.5 * (double)D * (LOG_2PI + 2.0 * log(tau));
    return lp;
}

/* Linear-Gaussian regression: y_i ~ N(x_i' theta, sigma^2), theta ~ N(0, tau^2 I). */
static double linear_gauss(const oracle_target* t, const double* th, double* g) {
    const int64_t D = t->D, n = t->n;
    const double sigma = t->hyper[0], tau = t->hyper[1];
    double lp = 0.0;
    if (g) memset(g, 0, (size_t)D * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        const double* x = t->X + i * D;
        double eta = 0.0;
        for (int64_t d = 0; d < D; ++d) eta += x[d] * th[d];
        double r = (t->y[i] - eta) / sigma;
        lp += -0.5 * r * r;
        if (g)
            for (int64_t d = 0; d < D; ++d) g[d] += (r / sigma) * x[d];
    }
    lp += -0.5 * (double)n * (LOG_2PI + 2.0 * log(sigma));
    double sq = 0.0;
    for (int64_t d = 0; d < D; ++d) {
        sq += th[d] * th[d];
        if (g) g[d] -= th[d] / (tau * tau);
    }
    lp += -0.5 * sq / (tau * tau) - 0.5 * (double)D * (LOG_2PI + 2.0 * log(tau));
    return lp;
}

/* Non-centred hierarchical normal.  theta = (mu, log tau, eta_1..eta_G),
 * group effect b_g = mu + tau eta_g, y_gi ~ N(b_g, sigma^2) summarised by the
 * group mean ybar_g, size n_g and within-group sum of squares SS_g.
 * Priors: mu ~ N(0,1), log tau ~ N(0,1), eta_g ~ N(0,1). */
static double hier_normal(const oracle_target* t, const double* th, double* g) {
    const int64_t G = t->n;
    const double sigma = t->hyper[0], s2 = sigma * sigma;
    const double mu = th[0], logtau = th[1], tau = exp(logtau);
    double lp = 0.0, dmu = 0.0, dlogtau = 0.0;
    for (int64_t k = 0; k < G; ++k) {
        double eta = th[2 + k];
        double ng = t->mu[k], ybar = t->y[k], SS = t->P[k];
        double b = mu + tau * eta;
        double dev = ybar - b;
        lp += -0.5 * ng * (LOG_2PI + 2.0 * log(sigma)) - 0.5 * (SS + ng * dev * dev) / s2;
        lp += -0.5 * eta * eta - 0.5 * LOG_2PI;
        double r = ng * dev / s2;           /* d loglik / d b_g */
        dmu += r;
        dlogtau += r * tau * eta;
        if (g) g[2 + k] = r * tau - eta;
    }
    lp += -0.5 * mu * mu - 0.5 * LOG_2PI;
    lp += -0.5 * logtau * logtau - 0.5 * LOG_2PI;
    if (g) {
        g[0] = dmu - mu;
        g[1] = dlogtau - logtau;
    }
    return lp;
}

/* Banana (Sec. 4, Rosenbrock) generalised to D/2 independent pairs:
 * x_o ~ N(0, a), x_e | x_o ~ N(b (x_o^2 - a), 1).  Normalised: log Z = 0. */
static double banana(const oracle_target* t, const double* th, double* g) {
    const int64_t D = t->D;
    const double a = t->hyper[0], b = t->hyper[1];
    double lp = 0.0;
    for (int64_t i = 0; i + 1 < D; i += 2) {
        double xo = th[i], xe = th[i + 1];
        double u = xe - b * (xo * xo - a);
        lp += -0.5 * xo * xo / a - 0.5 * (LOG_2PI + log(a)) - 0.5 * u * u - 0.5 * LOG_2PI;
        if (g) {
            g[i] = -xo / a + u * 2.0 * b * xo;
            g[i + 1] = -u;
        }
    }
    return lp;
}

double oracle_logpi(const oracle_target* t, const double* theta, double* grad) {
    switch (t->kind) {
        case ORACLE_GAUSS_DENSE: return gauss_dense(t, theta, grad);
        case ORACLE_LOGISTIC: return logistic(t, theta, grad);
        case ORACLE_HIER_NORMAL: return hier_normal(t, theta, grad);
        case ORACLE_BANANA: return banana(t, theta, grad);
        case ORACLE_LINEAR_GAUSS: return linear_gauss(t, theta, grad);
        default: return NAN;
    }
}
