/*
 * smc.c -- oracle SMC sampler with the ChEES-HMC proposal (Algorithm 3 with
 * the proposal of Sec. 3.1-3.2), FP64, step by step in the paper's order.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 * Pins: posterior mean, covariance and log evidence of conjugate Gaussian and
 * linear-Gaussian targets within 3 Monte Carlo standard errors; the paper's
 * Table 1 row for 1-d Halton on the 5-d Gaussian as a loose statistical check
 * (tests/test_oracle_smc.py).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double LOG_2PI = 1.8378770664093454835606594728112;

static void set_threads(int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

static double lse(const double* a, int64_t N) {
    double m = -INFINITY;
    for (int64_t j = 0; j < N; ++j)
        if (a[j] > m) m = a[j];
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int64_t j = 0; j < N; ++j) s += exp(a[j] - m);
    return m + log(s);
}

double oracle_smc_init(const oracle_target* t, const oracle_config* c, double* theta,
                       double* grad, double* logpi, double* logw, int32_t nthreads) {
    /* theta_0^j ~ q_init = N(0, s^2 I), or N(m, L L^T) when the config gives
     * a mean or a Cholesky factor; w_1^j = pi(theta_0^j) / q_init(theta_0^j). */
    const int64_t N = c->n_particles, D = t->D;
    const double s = c->init_scale;
    const int general = c->init_mean != 0 || c->init_chol != 0;
    double logdet = 0.0;     /* log |det L| = sum_d log L_dd */
    if (general) {
        if (c->init_chol)
            for (int64_t d = 0; d < D; ++d) logdet += log(c->init_chol[d * D + d]);
        else
            logdet = (double)D * log(s);
    }
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < N; ++j) {
        double* th = theta + j * D;
        oracle_normals(c->seed, ORACLE_TAG_INIT, 0u, (uint32_t)j, D, th);
        double zz = 0.0;
        for (int64_t d = 0; d < D; ++d) zz += th[d] * th[d];
        double logq;
        if (!general) {
            for (int64_t d = 0; d < D; ++d) th[d] *= s;
            logq = -0.5 * zz - 0.5 * (double)D * (LOG_2PI + 2.0 * log(s));
        } else {
            /* theta = m + L z, component d from the highest index down so
             * that z_e (e <= d) is still unmodified when it is read */
            for (int64_t d = D - 1; d >= 0; --d) {
                double acc = c->init_mean ? c->init_mean[d] : 0.0;
                for (int64_t e = 0; e <= d; ++e) {
                    const double l = c->init_chol ? c->init_chol[d * D + e] : (e == d ? s : 0.0);
                    acc += l * th[e];
                }
                th[d] = acc;
            }
            logq = -0.5 * zz - (0.5 * (double)D * LOG_2PI + logdet);
        }
        double lp = oracle_logpi(t, th, grad + j * D);
        logpi[j] = lp;
        logw[j] = c->mcmc ? 0.0 : (isfinite(lp) ? lp - logq : -INFINITY);
    }
    return lse(logw, N) - log((double)N);
}

int oracle_smc_iteration(const oracle_target* t, const oracle_config* c, int64_t k,
                         oracle_iter_io* io, oracle_stats* st, int32_t nthreads) {
    const int64_t N = c->n_particles, D = t->D, K = c->n_iters;
    int status = 0;
    double* z0 = 0;
    double* W = (double*)malloc((size_t)N * sizeof(double));
    int32_t* anc = io->ancestors ? io->ancestors : (int32_t*)malloc((size_t)N * sizeof(int32_t));
    int32_t* S = io->steps ? io->steps : (int32_t*)malloc((size_t)N * sizeof(int32_t));
    double* l = (double*)malloc((size_t)N * sizeof(double));
    double* th1 = (double*)malloc((size_t)(N * D) * sizeof(double));
    double* g1 = (double*)malloc((size_t)(N * D) * sizeof(double));
    double* lp1 = (double*)malloc((size_t)N * sizeof(double));
    double* p0 = io->p0 ? io->p0 : (double*)malloc((size_t)(N * D) * sizeof(double));
    double* p1 = io->p1 ? io->p1 : (double*)malloc((size_t)(N * D) * sizeof(double));
    double* dH = io->dH ? io->dH : (double*)malloc((size_t)N * sizeof(double));
    double* alpha = io->alpha ? io->alpha : (double*)malloc((size_t)N * sizeof(double));
    set_threads(nthreads);

    /* (a) normalise the weights and compute J_eff. */
    double L0, ess;
    oracle_normalise(io->logw, N, &L0, &ess, W);
    if (L0 == -INFINITY) { status = -4; goto done; }
    if (st) st->ess_pre = ess;

    /* (b) resample when J_eff < J/2; reset the weights to 1/J. */
    int resampled = ess < c->ess_frac * (double)N;
    if (resampled) {
        uint64_t* q = (uint64_t*)malloc((size_t)N * sizeof(uint64_t));
        oracle_quantise(W, N, q);
        uint64_t T = 0;
        if (c->resample_scheme == 1) {
            /* multinomial: N independent draws from the fixed-point weights */
            uint64_t* u = (uint64_t*)malloc((size_t)N * sizeof(uint64_t));
            for (int64_t i = 0; i < N; ++i) {
                u[i] = oracle_multinomial_u64(c->seed, (uint32_t)k, (uint32_t)i);
                T += q[i];
            }
            if (T > 0) oracle_multinomial(q, N, u, anc);
            free(u);
        } else {
            T = oracle_systematic(q, N, oracle_resample_r64(c->seed, (uint32_t)k), anc);
        }
        free(q);
        if (T == 0) { status = -4; goto done; }
        double* tmp = (double*)malloc((size_t)(N * D) * sizeof(double));
        double* tmp1 = (double*)malloc((size_t)N * sizeof(double));
        memcpy(tmp, io->theta, (size_t)(N * D) * sizeof(double));
        for (int64_t i = 0; i < N; ++i) memcpy(io->theta + i * D, tmp + (int64_t)anc[i] * D, (size_t)D * sizeof(double));
        memcpy(tmp, io->grad, (size_t)(N * D) * sizeof(double));
        for (int64_t i = 0; i < N; ++i) memcpy(io->grad + i * D, tmp + (int64_t)anc[i] * D, (size_t)D * sizeof(double));
        memcpy(tmp1, io->logpi, (size_t)N * sizeof(double));
        for (int64_t i = 0; i < N; ++i) io->logpi[i] = tmp1[anc[i]];
        free(tmp);
        free(tmp1);
        for (int64_t i = 0; i < N; ++i) {
            io->logw[i] = -log((double)N);
            W[i] = 1.0 / (double)N;
        }
    } else {
        for (int64_t i = 0; i < N; ++i) anc[i] = (int32_t)i;
    }

    /* learned preconditioner: trained on the current weighted particles at
     * warm-up iterations (k - 1) % every == 0 whose tested J_eff is at least
     * flow_min_ess * J (a near-degenerate weighted set holds a few distinct
     * points, and fitting a density to them collapses the map), frozen
     * afterwards */
    oracle_flow flow = {D, io->flow_H, io->flow_L, io->flow_params};
    const int use_flow = io->flow_params != 0;
    if (use_flow && k < c->n_warmup && c->flow_train_every > 0 && (k - 1) % c->flow_train_every == 0 &&
        ess >= c->flow_min_ess * (double)N) {
        const int64_t np = oracle_flow_num_params(D, io->flow_H, io->flow_L);
        double* gradp = (double*)malloc((size_t)np * sizeof(double));
        for (int32_t e = 0; e < c->flow_epochs; ++e) {
            oracle_flow_loss_grad(&flow, io->theta, W, N, gradp);
            *io->flow_t += 1;
            oracle_flow_adam(io->flow_params, gradp, io->flow_m, io->flow_v, np, *io->flow_t, c->flow_lr, 0.9,
                             0.999, 1e-8);
        }
        free(gradp);
    }
    z0 = use_flow ? (double*)malloc((size_t)(N * D) * sizeof(double)) : 0;

    /* the step size of this iteration: fixed, or the adapted value */
    const double eps = io->eps ? *io->eps : c->step_size;

    /* (c) jittered trajectory lengths l_j = h_j L and step counts. */
    const double L = exp(io->chees->log_L);
    for (int64_t j = 0; j < N; ++j) {
        double h = oracle_jitter(c->jitter, c->seed, j, k, N, K);
        l[j] = h * L;
        S[j] = oracle_step_count(h, L, eps, c->max_steps);
    }

    /* (d, e) momentum, leapfrog, energy error and acceptance probability. */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < N; ++j) {
        double* pj = p1 + j * D;
        oracle_normals(c->seed, ORACLE_TAG_MOM, (uint32_t)k, (uint32_t)j, D, pj);
        memcpy(p0 + j * D, pj, (size_t)D * sizeof(double));
        memcpy(th1 + j * D, io->theta + j * D, (size_t)D * sizeof(double));
        memcpy(g1 + j * D, io->grad + j * D, (size_t)D * sizeof(double));
        lp1[j] = io->logpi[j];
        double H0, H1;
        if (!use_flow) {
            H0 = oracle_hamiltonian(pj, D, lp1[j]);
            oracle_leapfrog(t, th1 + j * D, pj, g1 + j * D, lp1 + j, eps, S[j]);
            H1 = oracle_hamiltonian(pj, D, lp1[j]);
        } else {
            /* HMC in z = T^-1(theta) on log pi_z (Algorithm 1 in latent space) */
            double* z = z0 + j * D;
            double ldi;
            oracle_flow_inverse(&flow, io->theta + j * D, z, &ldi);
            double* zz = (double*)malloc((size_t)(3 * D) * sizeof(double));
            double *gz = zz + D, *x = gz + D;
            memcpy(zz, z, (size_t)D * sizeof(double));
            double lpz = oracle_flow_logpi_z(&flow, t, zz, gz, 0, 0, 0);
            H0 = oracle_hamiltonian(pj, D, lpz);
            double lpx = lp1[j];
            for (int32_t l = 0; l < S[j]; ++l) {
                for (int64_t d = 0; d < D; ++d) pj[d] += 0.5 * eps * gz[d];
                for (int64_t d = 0; d < D; ++d) zz[d] += eps * pj[d];
                lpz = oracle_flow_logpi_z(&flow, t, zz, gz, x, g1 + j * D, &lpx);
                for (int64_t d = 0; d < D; ++d) pj[d] += 0.5 * eps * gz[d];
            }
            if (S[j] > 0) {
                memcpy(th1 + j * D, x, (size_t)D * sizeof(double));
                lp1[j] = lpx;
            }
            H1 = oracle_hamiltonian(pj, D, lpz);
            /* keep the latent start for the ChEES statistics; the end in th1 is
             * re-mapped below */
            free(zz);
        }
        double d = H1 - H0;
        if (!isfinite(d)) d = INFINITY;
        dH[j] = d;
        alpha[j] = d <= 0.0 ? 1.0 : exp(-d);
    }

    /* (f) reweight with the momentum L-kernel: log w += -Delta H, and the
     * evidence factor sum_j W_j exp(-Delta H_j). */
    double log_z_inc = 0.0;
    const int mh_select = c->accept_reject || c->mcmc;
    if (!mh_select) {
        double* a = (double*)malloc((size_t)N * sizeof(double));
        for (int64_t j = 0; j < N; ++j) a[j] = log(W[j]) - dH[j];
        log_z_inc = lse(a, N);
        free(a);
        for (int64_t j = 0; j < N; ++j) io->logw[j] -= dH[j];
    }

    /* (g) ChEES adaptation during warm-up, uses the pre-move states (in the
     * latent space when the flow is on: the momenta live there). */
    if (c->adapt && k < c->n_warmup) {
        double ghat;
        const double* pm = c->chees_initial_p ? p0 : p1;
        const double* s0 = io->theta;
        const double* s1 = th1;
        double* z1 = 0;
        if (use_flow) {
            z1 = (double*)malloc((size_t)(N * D) * sizeof(double));
            for (int64_t j = 0; j < N; ++j) oracle_flow_inverse(&flow, th1 + j * D, z1 + j * D, 0);
            s0 = z0;
            s1 = z1;
        }
        int okg = oracle_chees_gradient(s0, s1, pm, l, alpha, N, D, &ghat, 0);
        free(z1);
        if (okg)
            oracle_chees_adam(io->chees, ghat, c->adam_lr, c->adam_b1, c->adam_b2,
                              c->adam_eps, eps, c->max_steps);
        io->chees->Lbar = 0.9 * io->chees->Lbar + 0.1 * exp(io->chees->log_L);
    }
    if (c->adapt && k == c->n_warmup && io->chees->Lbar > 0.0) io->chees->log_L = log(io->chees->Lbar);
    /* optional step-size adaptation during warm-up, after the ChEES update;
     * epsilon stays where it is from M_warmup on */
    if (c->step_adapt_rate > 0.0 && k < c->n_warmup && io->eps)
        *io->eps = oracle_step_size_update(eps, alpha, N, c->step_adapt_rate, c->step_adapt_target);

    /* (h) move: without accept-reject every particle takes its proposal; with
     * it, the Metropolis rule u < alpha decides and the weight is unchanged. */
    for (int64_t j = 0; j < N; ++j) {
        int take = 1;
        if (mh_select) {
            uint32_t ctr[4] = {0u, (uint32_t)j, (uint32_t)k, (uint32_t)ORACLE_TAG_MH}, w[4];
            oracle_philox4x32_10(ctr, c->seed, w);
            take = oracle_u01(w[0], w[1]) < alpha[j];
        }
        if (take) {
            memcpy(io->theta + j * D, th1 + j * D, (size_t)D * sizeof(double));
            memcpy(io->grad + j * D, g1 + j * D, (size_t)D * sizeof(double));
            io->logpi[j] = lp1[j];
        }
    }
    *io->log_z += log_z_inc;

    if (st) {
        double lz2, ess2;
        oracle_normalise(io->logw, N, &lz2, &ess2, 0);
        st->ess = ess2;
        st->log_z_inc = log_z_inc;
        double sa = 0.0;
        int64_t ge = 0;
        int32_t smin = S[0], smax = S[0];
        for (int64_t j = 0; j < N; ++j) {
            sa += alpha[j];
            ge += S[j];
            if (S[j] < smin) smin = S[j];
            if (S[j] > smax) smax = S[j];
        }
        st->mean_alpha = sa / (double)N;
        st->traj_len = L;
        st->grad_evals = ge;
        st->steps_min = smin;
        st->steps_max = smax;
        st->resampled = resampled;
    }

done:
    free(z0);
    free(W);
    if (!io->ancestors) free(anc);
    if (!io->steps) free(S);
    free(l);
    free(th1);
    free(g1);
    free(lp1);
    if (!io->p0) free(p0);
    if (!io->p1) free(p1);
    if (!io->dH) free(dH);
    if (!io->alpha) free(alpha);
    return status;
}

int oracle_smc_run(const oracle_target* t, const oracle_config* c, double* theta_out,
                   double* logw_out, double* log_z, oracle_stats* stats, int32_t nthreads) {
    const int64_t N = c->n_particles, D = t->D;
    double* theta = (double*)malloc((size_t)(N * D) * sizeof(double));
    double* grad = (double*)malloc((size_t)(N * D) * sizeof(double));
    double* logpi = (double*)malloc((size_t)N * sizeof(double));
    double* logw = (double*)malloc((size_t)N * sizeof(double));
    double lz = oracle_smc_init(t, c, theta, grad, logpi, logw, nthreads);
    oracle_chees_state ch = {log(c->traj_len0), 0.0, 0.0, 0, 0.0};
    double lo = log(c->step_size), hi = log((double)c->max_steps * c->step_size);
    if (ch.log_L < lo) ch.log_L = lo;
    if (ch.log_L > hi) ch.log_L = hi;
    double eps = c->step_size;
    int status = 0;
    for (int64_t k = 1; k <= c->n_iters && status == 0; ++k) {
        oracle_iter_io io = {theta, grad, logpi, logw, &ch, &lz, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, &eps};
        status = oracle_smc_iteration(t, c, k, &io, stats ? stats + (k - 1) : 0, nthreads);
    }
    if (theta_out) memcpy(theta_out, theta, (size_t)(N * D) * sizeof(double));
    if (logw_out) memcpy(logw_out, logw, (size_t)N * sizeof(double));
    if (log_z) *log_z = lz;
    free(theta);
    free(grad);
    free(logpi);
    free(logw);
    return status;
}
