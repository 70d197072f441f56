/*
 * oracle.h -- plain, slow, FP64 CPU oracle for SMC with a ChEES-HMC proposal
 * (Millard, Murphy, Frisch, Maskell, "Incorporating the ChEES Criterion into
 * Sequential Monte Carlo Samplers", arXiv 2504.02627).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no source,
 * header, table or helper with the CUDA library; the two sides meet only in
 * the seeded input generators (workloads/), which hold none of the method's
 * arithmetic.
 *
 * Layout: particle-major on the CPU side means particle j's D coordinates are
 * contiguous: theta[j*D + d].  (The GPU library uses the transposed [D x N]
 * layout; tests transpose.)
 *
 * Every floating-point result is FP64.  Compile with -ffp-contract=off so that
 * x86-64 and aarch64 hosts give identical bits.
 *
 * Pins (what fixes each function independently of this code) live in
 * tests/test_oracle_*.py.  Functions without an independent pin say
 * "parity unpinned" below.
 */
#ifndef SMC_ORACLE_H
#define SMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------------------
 * Counter-based random numbers.  Philox4x32-10 as defined by Salmon, Moraes,
 * Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).  The
 * paper under study draws momenta p ~ N(0, M) (Sec. 2.1) and resampling
 * uniforms (Sec. 3); it does not fix a generator.
 * Key  = (seed low 32 bits, seed high 32 bits).
 * Counter = (i, j, k, tag): i = block index inside one particle's stream,
 * j = particle slot, k = SMC iteration, tag = purpose below.
 * ------------------------------------------------------------------------- */
enum { ORACLE_TAG_INIT = 1, ORACLE_TAG_MOM = 2, ORACLE_TAG_RESAMPLE = 3, ORACLE_TAG_MH = 4,
       ORACLE_TAG_JITTER = 5, ORACLE_TAG_SHUFFLE = 6 };

void oracle_philox4x32_10(const uint32_t ctr[4], uint64_t seed, uint32_t out[4]);
/* Uniform on the open interval (0,1) from 52 random bits: (k + 0.5) * 2^-52. */
double oracle_u01(uint32_t w0, uint32_t w1);
/* D standard normals for (tag, k, j) by Box-Muller on consecutive Philox blocks. */
void oracle_normals(uint64_t seed, uint32_t tag, uint32_t k, uint32_t j, int64_t D, double* out);
/* 64-bit uniform integer used by systematic resampling at iteration k. */
uint64_t oracle_resample_r64(uint64_t seed, uint32_t k);
/* Uniform 64-bit integer of output i for multinomial resampling at iteration
 * k: Philox block (1, i, k, RESAMPLE), words 0 and 1 (the systematic draw
 * above uses block (0, 0, k, RESAMPLE)). */
uint64_t oracle_multinomial_u64(uint64_t seed, uint32_t k, uint32_t i);

/* ---------------------------------------------------------------------------
 * Jitter of the trajectory length (Sec. "Random Number Generators", item
 * "1-d Halton"): the base-2 radical inverse of n = j*K + k (0-based slot j,
 * 1-based iteration k), and the step count ceil(h*L/eps) (Alg. 2) clipped
 * to [1, max_steps].
 * ------------------------------------------------------------------------- */
double oracle_halton2(uint32_t n);

/* Jitter schemes of Sec. 3.2.1 for particle j (0-based: the paper's j - 1) at
 * iteration k (1-based) of J particles and K iterations:
 *   0 none (1);  1 1-d Halton, base 2, of n = jK + k;  2 uniform, the FP64
 *   uniform of Philox block (0, j, k, JITTER);  3 N-d Halton: radical
 *   inverse of j + 1 in base P_k (the k-th prime);  4 N-d inverse Halton:
 *   base P_{K+1-k};  5 N-d primes: frac((j + 1) sqrt(P_k));  6 N-d inverse
 *   primes: P_{K+1-k};  7 1-d golden ratio: frac((jK + k)(sqrt(5) - 1)/2);
 *   8 equidistant: (pi_k(j) + 1) / J, pi_k the shuffle of iteration k;
 *   9 offset equidistant: that plus 0.1 u, u the FP64 uniform of Philox block
 *   (1, j, k, JITTER);  10 1-d Sobol: radical inverse base 2 of the Gray
 *   code g = n ^ (n >> 1) of n = jK + k (the first Sobol dimension in Gray-
 *   code order);  11 1-d Halton, base 2, of n = (k - 1) J + j + 1 (the J x K
 *   matrix of scheme 1 read iteration-major).
 * Schemes 3-6 reuse their K dimensions cyclically past iteration K.
 * Every value is a correctly rounded FP64 operation sequence: radical
 * inverses as one division of two exact integers, sqrt, products and frac
 * each rounded once. */
double oracle_jitter(int32_t scheme, uint64_t seed, int64_t j, int64_t k, int64_t J, int64_t K);
/* the m-th prime (m >= 1; m <= 65536) */
int64_t oracle_nth_prime(int64_t m);
/* radical inverse of n in base b: the base-b digits of n reversed behind the
 * point (Halton 1960), as the exact fraction rev / b^digits rounded once */
double oracle_radical_inverse(uint64_t n, uint64_t b);
/* shuffle of iteration k: a bijection of {0..J-1}, the four-round Feistel
 * network on 2 ceil(log4 J) bits with round function F_r(x) = word 0 of
 * Philox block (x, r, k, SHUFFLE) masked to half the bits, applied to j
 * repeatedly until the result is below J (cycle walking) */
uint32_t oracle_shuffle_index(uint64_t seed, uint32_t k, uint32_t j, uint32_t J);
int32_t oracle_step_count(double h, double L, double eps, int32_t max_steps);

/* ---------------------------------------------------------------------------
 * Targets: log pi(theta) = log p(x|theta) + log q0(theta) (Sec. 2) and its
 * gradient.  All densities are normalised unless stated, so that the SMC
 * evidence estimate targets the marginal likelihood.
 * ------------------------------------------------------------------------- */
enum {
    ORACLE_GAUSS_DENSE = 0,   /* c - 1/2 (t-mu)' P (t-mu); P = precision            */
    ORACLE_LOGISTIC = 1,      /* Sec. 4 "German Credit": Bernoulli(sigmoid(x'theta)), prior N(0, tau^2 I) */
    ORACLE_HIER_NORMAL = 2,   /* non-centred hierarchical normal, sufficient statistics  */
    ORACLE_BANANA = 3,        /* Sec. 4 "Rosenbrock": pairs x_o ~ N(0,a), x_e ~ N(b(x_o^2-a),1) */
    ORACLE_LINEAR_GAUSS = 4   /* y ~ N(X theta, sigma^2 I), theta ~ N(0, tau^2 I)     */
};

typedef struct {
    int32_t kind;
    int64_t D;          /* parameter dimension                                    */
    int64_t n;          /* observations (LOGISTIC, LINEAR_GAUSS) or groups (HIER)   */
    const double* X;    /* n x D row-major                                         */
    const double* y;    /* n labels / responses; HIER: group means ybar           */
    const double* mu;   /* GAUSS_DENSE mean; HIER: group sizes n_g                  */
    const double* P;    /* GAUSS_DENSE precision D x D; HIER: within-group SS_g     */
    double c;           /* GAUSS_DENSE additive constant                            */
    double hyper[4];    /* LOGISTIC: tau; LINEAR: sigma, tau; HIER: sigma; BANANA: a, b */
} oracle_target;

/* log pi(theta); writes grad (length D) when grad != NULL. */
double oracle_logpi(const oracle_target* t, const double* theta, double* grad);

/* ---------------------------------------------------------------------------
 * HMC (Sec. 2.1): Hamiltonian H = 1/2 |p|^2 - log pi(theta) (the sign printed
 * in the paper's second line is read as a typo; exp(-H) must be the joint
 * density), and S leapfrog steps (Eqs. for p_{l+1/2}, theta_{l+1}, p_{l+1};
 * Algorithm 1).  theta, p, grad and *logpi are updated in place; on entry grad
 * and *logpi must hold the values at theta.
 * ------------------------------------------------------------------------- */
double oracle_hamiltonian(const double* p, int64_t D, double logpi);
void oracle_leapfrog(const oracle_target* t, double* theta, double* p, double* grad,
                     double* logpi, double eps, int32_t steps);

/* ---------------------------------------------------------------------------
 * Weights (Sec. 3, Eqs. for the normalised weights and J_eff): log-sum-exp,
 * normalised weights W (may be NULL) and ESS = 1 / sum W^2.
 * ------------------------------------------------------------------------- */
void oracle_normalise(const double* logw, int64_t N, double* lse, double* ess, double* W);

/* ---------------------------------------------------------------------------
 * Systematic resampling in 64-bit fixed point.  The paper resamples when
 * J_eff < J/2 (Sec. 3) with the multinomial scheme; the systematic scheme is
 * the one it cites as optimally parallelisable.  q_j = floor(W_j 2^S) with
 * S = 62 - ceil(log2 N); T = sum q; U = floor(r64 T / 2^64); ancestor of
 * output i = smallest j with N*C_j > i*T + U where C is the inclusive prefix.
 * Returns S from quantise, T from resample (0 means degenerate).
 * ------------------------------------------------------------------------- */
int32_t oracle_quantise(const double* W, int64_t N, uint64_t* q);
uint64_t oracle_systematic(const uint64_t* q, int64_t N, uint64_t r64, int32_t* ancestors);
/* Multinomial variant (the paper's own scheme, Sec. 3): N independent
 * 64-bit uniforms u_i; position P_i = floor(u_i T / 2^64); ancestor of output
 * i = smallest j with C_j > P_i, so P(ancestor = j) = q_j / T up to 2^-64. */
void oracle_multinomial(const uint64_t* q, int64_t N, const uint64_t* u64, int32_t* ancestors);

/* ---------------------------------------------------------------------------
 * ChEES (Sec. 2.3, Algorithm 2): per-particle gradient estimates
 *   g_j = l_j (|t1_j - mean t1|^2 - |t0_j - mean t0|^2) (t1_j - mean t1)' p_j
 * and their acceptance-weighted mean sum a_j g_j / sum a_j.  p is the final
 * momentum by default (see the reading list); use_initial selects p0.
 * Returns 0 when sum a_j == 0 or the mean is not finite (no update).
 * ------------------------------------------------------------------------- */
int oracle_chees_gradient(const double* theta0, const double* theta1, const double* p,
                          const double* l, const double* alpha, int64_t N, int64_t D,
                          double* ghat, double* g_per_particle);

typedef struct {
    double log_L;   /* log trajectory length (time units)       */
    double m, v;    /* Adam first and second moments            */
    int32_t t;      /* Adam step counter                        */
    double Lbar;    /* moving average 0.9 Lbar + 0.1 L          */
} oracle_chees_state;

/* One Adam ascent step on log L with gradient ghat, then clamp L to
 * [eps, max_steps*eps].  The moving average Lbar <- 0.9 Lbar + 0.1 L of
 * Algorithm 2 is applied by the iteration after this call. */
void oracle_chees_adam(oracle_chees_state* s, double ghat, double lr, double b1, double b2,
                       double adam_eps, double eps, int32_t max_steps);

/* Optional step-size adaptation (not in the paper, which fixes epsilon per
 * experiment and names its adaptation as future work, Sec. 5): after the
 * ChEES update of a warm-up iteration, log epsilon moves by
 * rate * (a_h - target), where a_h = N / sum_j 1/alpha_j is the harmonic mean
 * of the acceptance probabilities (0 when some alpha_j is 0) and the target
 * is the asymptotically optimal HMC acceptance 0.651 (Beskos et al., 2013).
 * Returns the new epsilon. */
double oracle_harmonic_mean_alpha(const double* alpha, int64_t N);
double oracle_step_size_update(double eps, const double* alpha, int64_t N, double rate, double target);

/* ---------------------------------------------------------------------------
 * The SMC sampler (Algorithm 3) with the ChEES-HMC proposal and the
 * momentum change-of-variable L-kernel (Sec. 3.1), so the incremental
 * log-weight is -Delta H, without accept-reject by default (Sec. 3.1).
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t n_particles;    /* J                                             */
    int64_t n_iters;        /* K                                             */
    int64_t n_warmup;       /* M_warmup                                      */
    double step_size;       /* epsilon                                       */
    double traj_len0;       /* L_0 (time units)                              */
    int32_t max_steps;      /* leapfrog cap                                  */
    double ess_frac;        /* resample when ESS < ess_frac * J (0.5)        */
    uint64_t seed;
    int32_t jitter;         /* 0: h = 1; 1: 1-d Halton base 2               */
    int32_t accept_reject;  /* 0: paper's SMC-ChEES; 1: MH select, weight 1  */
    int32_t adapt;          /* 1: ChEES adaptation of L during warm-up       */
    int32_t chees_initial_p;/* 0: final momentum in g_j (default); 1: initial */
    double adam_lr, adam_b1, adam_b2, adam_eps;
    double init_scale;      /* q_init = N(0, init_scale^2 I)                 */
    int32_t flow_train_every; /* train the flow at warm-up iterations k with (k-1) % every == 0 */
    int32_t flow_epochs;    /* full-batch Adam steps per training event      */
    double flow_lr;
    double flow_min_ess;    /* train only when the tested J_eff >= flow_min_ess * J */
    double step_adapt_rate; /* kappa: 0 keeps epsilon fixed (the paper); > 0 applies
                               oracle_step_size_update during warm-up        */
    double step_adapt_target; /* harmonic-mean acceptance target (0.651)      */
    int32_t resample_scheme;  /* 0: systematic (fixed point, the default); 1:
                                 multinomial, the paper's choice (Sec. 3), with
                                 the uniforms of oracle_multinomial_u64         */
    int32_t mcmc;             /* 1: Algorithm 2 as J independent chains: no
                                 importance weights (log w = 0 from the start,
                                 so J_eff = J and nothing resamples), the
                                 Metropolis select of accept_reject, log Z = 0 */
    /* A general Gaussian initial distribution q_init = N(m, L L^T) (the paper
     * leaves q_init to the user; its experiments use N(0, I), Sec. 4).  Either
     * pointer may be NULL: m = 0, L = init_scale * I.  With either given,
     * theta_0 = m + L z with z the same standard normals as the isotropic
     * draw, each component summed in the order m_d + L_d0 z_0 + ... + L_dd z_d,
     * and log q_init = -|z|^2 / 2 - (D/2 log 2 pi + sum_d log L_dd), the
     * log-determinant summed over d in order. */
    const double* init_mean;  /* [D], or NULL                                   */
    const double* init_chol;  /* [D x D] row-major, lower-triangular, positive
                                 diagonal (the upper triangle is not read), or NULL */
} oracle_config;

typedef struct {
    double ess;             /* J_eff after this iteration's reweighting      */
    double ess_pre;         /* J_eff tested for resampling at its start      */
    double log_z_inc;
    double mean_alpha;
    double traj_len;        /* L used for this iteration's jitter            */
    int64_t grad_evals;     /* sum_j S_j                                     */
    int32_t steps_min, steps_max, resampled, pad;
} oracle_stats;

/* Runs the whole sampler.  theta_out: N*D (may be NULL), logw_out: N (may be
 * NULL), stats: n_iters entries (may be NULL).  Returns 0, or -4 when all
 * weights are -inf.  nthreads <= 0 uses every OpenMP thread (when built with
 * OpenMP). */
int oracle_smc_run(const oracle_target* t, const oracle_config* c, double* theta_out,
                   double* logw_out, double* log_z, oracle_stats* stats, int32_t nthreads);

/* One SMC iteration k (1-based) on caller-owned state, for parity tests that
 * feed the GPU state back in.  theta/grad/logpi: N*D, N*D, N; logw: N.
 * Outputs (may be NULL): ancestors N, steps N, p0 N*D (initial momentum),
 * p1 N*D (final), dH N, alpha N. */
typedef struct {
    double* theta; double* grad; double* logpi; double* logw;
    oracle_chees_state* chees; double* log_z;
    int32_t* ancestors; int32_t* steps; double* p0; double* p1; double* dH; double* alpha;
    /* learned preconditioner (NULL: HMC in theta space) and its Adam state */
    double* flow_params; double* flow_m; double* flow_v; int32_t* flow_t; int64_t flow_H, flow_L;
    /* current step size, updated in place when step_adapt_rate > 0 (NULL:
     * step_size, fixed) */
    double* eps;
} oracle_iter_io;
int oracle_smc_iteration(const oracle_target* t, const oracle_config* c, int64_t k,
                         oracle_iter_io* io, oracle_stats* st, int32_t nthreads);

/* Initial draw (Eqs. for theta_0 ~ q0 and w_1 = pi/q0): fills theta, grad,
 * logpi, logw (all N entries) and returns log Z_0 = LSE(logw) - log N. */
double oracle_smc_init(const oracle_target* t, const oracle_config* c, double* theta,
                       double* grad, double* logpi, double* logw, int32_t nthreads);

/* ---------------------------------------------------------------------------
 * Learned preconditioner: affine-coupling flow theta = T(z) (flow.c).  HMC
 * runs on log pi_z(z) = log pi(T(z)) + log|det dT/dz|; the move is exact for
 * any fixed T, and the weight takes -Delta H in z-space.
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t D, H, L;        /* dimension (even), hidden width, coupling layers */
    const double* params;   /* oracle_flow_num_params(D, H, L) doubles         */
} oracle_flow;
int64_t oracle_flow_num_params(int64_t D, int64_t H, int64_t L);
void oracle_flow_forward(const oracle_flow* f, const double* z, double* x, double* logdet);
void oracle_flow_inverse(const oracle_flow* f, const double* x, double* z, double* logdet_inv);
double oracle_flow_logpi_z(const oracle_flow* f, const oracle_target* t, const double* z, double* gz,
                           double* x_out, double* gx_out, double* logpi_x_out);
double oracle_flow_loss_grad(const oracle_flow* f, const double* theta, const double* W, int64_t N,
                             double* grad);
void oracle_flow_adam(double* params, const double* grad, double* m, double* v, int64_t n, int32_t t,
                      double lr, double b1, double b2, double eps);

/* Weighted moments (Eq. for realised estimates): mean and variance per dim. */
void oracle_moments(const double* theta, const double* logw, int64_t N, int64_t D,
                    double* mean, double* var);

#ifdef __cplusplus
}
#endif
#endif
