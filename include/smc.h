/*
 * smc.h -- C ABI of libsmcchees, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of an SMC sampler with a ChEES-HMC proposal
 * (Millard, Murphy, Frisch, Maskell, "Incorporating the ChEES Criterion into
 * Sequential Monte Carlo Samplers", arXiv 2504.02627).
 *
 * Conventions for every entry point:
 *  - Plain C types only; sizes are int64_t, floating scalars are double.
 *  - Every call returns smc_status; no exception or abort crosses the ABI.
 *  - "stream" is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  The caller owns the stream and keeps it alive while a handle that
 *    uses it exists.
 *  - Device arrays on the GPU side are particle-major [D x N]: element (d, j)
 *    lives at d * ld + j, with ld >= N, so consecutive particles are
 *    consecutive in memory.
 *  - The library allocates its own device memory (stream-ordered) in the
 *    *_create / smc_init calls; the kernel-level smc_k_* calls allocate
 *    nothing beyond what their comment states and write only their outputs.
 *  - Model data passed at creation are host FP64 arrays, copied (and cast) by
 *    the library; the caller may free them when the call returns.
 *  - Calls on one handle are not thread-safe; separate handles are independent.
 *  - Results are a deterministic function of (config, model, seed).
 */
#ifndef SMC_CHEES_H
#define SMC_CHEES_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SMC_OK = 0,
    SMC_E_INVAL = -1,       /* bad argument or unsupported configuration          */
    SMC_E_NOMEM = -2,       /* device allocation failed                           */
    SMC_E_CUDA = -3,        /* a CUDA call failed; smc_last_error has the text    */
    SMC_E_DEGENERATE = -4,  /* every weight is zero (all log-weights -inf)        */
    SMC_E_TIMEOUT = -5,     /* a bounded device wait gave up (scan look-back)     */
    SMC_E_STATE = -6        /* handle is in a sticky error state                  */
} smc_status;

/* ------------------------------------------------------------------ models
 * The target pi(theta) = p(x | theta) q0(theta) (Sec. 2).  Densities are
 * normalised (except GAUSS_DENSE, which adds the constant c), so that the
 * evidence estimate is the marginal likelihood.
 *  GAUSS_DENSE  log pi = c - 1/2 (theta - mu)' P (theta - mu); mu [dim],
 *               prec P [dim x dim] row-major.
 *  LOGISTIC     y_i ~ Bernoulli(sigmoid(x_i' theta)), theta ~ N(0, tau^2 I)
 *               (Sec. 4, German Credit); X [n_obs x dim] row-major, y [n_obs]
 *               in {0,1}; hyper[0] = tau.
 *  HIER_NORMAL  theta = (mu, log tau, eta_1..eta_G), dim = G + 2; group
 *               effect mu + tau eta_g, y_gi ~ N(., sigma^2) given by the
 *               sufficient statistics group_mean, group_n, group_ss [G];
 *               priors N(0,1) on mu, log tau, eta; hyper[0] = sigma; n_obs = G.
 *  BANANA       dim/2 independent pairs (Sec. 4, Rosenbrock):
 *               x_o ~ N(0, a), x_e ~ N(b (x_o^2 - a), 1); hyper = {a, b}.
 *  LINEAR_GAUSS y_i ~ N(x_i' theta, sigma^2), theta ~ N(0, tau^2 I);
 *               X, y as LOGISTIC; hyper = {sigma, tau}.
 */
typedef enum {
    SMC_MODEL_GAUSS_DENSE = 0,
    SMC_MODEL_LOGISTIC = 1,
    SMC_MODEL_HIER_NORMAL = 2,
    SMC_MODEL_BANANA = 3,
    SMC_MODEL_LINEAR_GAUSS = 4
} smc_model_kind;

typedef struct {
    int32_t kind;               /* smc_model_kind                                 */
    int32_t pad;
    int64_t dim;                /* D                                              */
    int64_t n_obs;              /* n (LOGISTIC, LINEAR_GAUSS) or G (HIER_NORMAL)  */
    const double* X;            /* host, n_obs x dim row-major                    */
    const double* y;            /* host, n_obs                                    */
    const double* mu;           /* host, dim                                      */
    const double* prec;         /* host, dim x dim row-major                      */
    const double* group_mean;   /* host, G                                        */
    const double* group_n;      /* host, G                                        */
    const double* group_ss;     /* host, G                                        */
    double c;                   /* additive constant (GAUSS_DENSE)                */
    double hyper[4];
} smc_model;

/* Likelihood arithmetic for the GEMM-shaped models (LOGISTIC, LINEAR_GAUSS). */
typedef enum {
    SMC_PREC_FP32 = 0,      /* FP32 SIMT, FP32 everywhere on the trajectory       */
    SMC_PREC_BF16X3 = 1,    /* tensor cores, every operand split into BF16 hi + lo,
                               three products (lo*lo dropped), FP32 accumulation;
                               dim <= 32: warp-level MMAs with X in one CTA's
                               shared memory, else the tcgen05 cluster kernel     */
    SMC_PREC_BF16 = 2,      /* tensor cores, BF16 operands, FP32 accumulation (same
                               kernels; data that do not fit on chip are streamed,
                               see BF16X2)                                        */
    SMC_PREC_BF16X2 = 3,    /* tcgen05, streamed data (any n, dim <= 128): X rounded
                               once to BF16, theta and the residuals r split into
                               BF16 hi + lo (two products per GEMM), FP32
                               accumulation                                      */
    SMC_PREC_BF16C = 4      /* tcgen05, streamed data (any n, dim <= 128), centred:
                               before each move every run's reference point
                               theta_ref (the mean of its particles) and the
                               reference quantities X theta_ref, sigmoid of it and
                               X'(y - sigmoid) are evaluated with the FP32 data and
                               FP64 sums; the trajectory's products then carry only
                               the deviations theta - theta_ref and the residual
                               changes, one BF16 product per GEMM with FP32
                               accumulation.  The gradient at the start point is
                               re-evaluated with the move's reference (so a move
                               costs S_j + 1 gradients).  At most 16 runs per
                               handle.  (Sec. 2 of the paper fixes no precision;
                               the end-point energies in the weights stay FP32 data
                               with FP64 sums, as for every precision.)          */
} smc_precision;

/* ------------------------------------------------------------------ config
 * Algorithm 3 (SMC) with the proposal of Algorithm 2 (ChEES-HMC).
 * Defaults used by the Python binding: ess_frac 0.5 (J_eff < J/2, Sec. 3),
 * jitter 1 (1-d Halton, Sec. 3.2), accept_reject 0 (no accept-reject,
 * Sec. 3.1), adapt 1; the Adam constants are this library's choice.
 */
typedef struct {
    int64_t n_particles;    /* J for this run                                     */
    int64_t n_iters;        /* K (also the Halton index stride)                   */
    int64_t n_warmup;       /* M_warmup: ChEES adapts while k < M_warmup          */
    double step_size;       /* epsilon                                            */
    double traj_len0;       /* L_0 in time units, clamped to [eps, max_steps*eps] */
    int32_t max_steps;      /* leapfrog cap (>= 1)                                */
    int32_t jitter;         /* trajectory-length jitter h (Sec. 3.2.1; smc_k_jitter):
                               0 none (h = 1); 1 1-d Halton of n = j*K + k; 2
                               uniform; 3 N-d Halton; 4 N-d inverse Halton; 5 N-d
                               primes; 6 N-d inverse primes; 7 1-d golden ratio;
                               8 equidistant; 9 offset equidistant; 10 1-d Sobol;
                               11 1-d Halton of n = (k-1)*J + j + 1 (the J x K
                               matrix read iteration-major).  3-6 need
                               n_iters <= 65536                                */
    double ess_frac;        /* resample when ESS < ess_frac * J                   */
    uint64_t seed;          /* Philox4x32-10 key                                  */
    int32_t accept_reject;  /* 0: the paper's SMC-ChEES (every particle moves, log w
                               += -Delta H); 1: Metropolis select u < alpha after
                               the move (Eqs. for alpha and the select rule), weight
                               unchanged; ChEES statistics use the proposals     */
    int32_t adapt;          /* 1: ChEES adaptation of L during warm-up            */
    double adam_lr, adam_b1, adam_b2, adam_eps;
    double init_scale;      /* q_init = N(0, init_scale^2 I)                      */
    int32_t precision;      /* smc_precision                                      */
    int32_t pad;
    /* Optional step-size adaptation (not in the paper, which fixes epsilon and
     * names its adaptation as future work, Sec. 5).  0 keeps epsilon fixed.
     * rate > 0: after the ChEES update of each warm-up iteration (k <
     * M_warmup), log epsilon += rate * (a_h - step_adapt_target), a_h = J /
     * sum_j 1/alpha_j the harmonic mean of the acceptance probabilities (0 if
     * some alpha_j = 0); epsilon is frozen from M_warmup on.  The current
     * epsilon is the ninth double of smc_get_buffer(SMC_BUF_RUNSTATE).      */
    double step_adapt_rate;
    double step_adapt_target;   /* in (0, 1); 0.651 in the Python binding          */
    int32_t resample_scheme;    /* 0: systematic (fixed point, the default); 1:
                                   multinomial, the paper's scheme (Sec. 3): output
                                   i takes the first particle j whose inclusive
                                   prefix C_j of the fixed-point weights exceeds
                                   floor(u_i T / 2^64), u_i the 64-bit word pair of
                                   Philox block (1, i, k, RESAMPLE)             */
    int32_t mcmc;               /* 1: Algorithm 2 as J independent ChEES-HMC
                                   chains: the initial draw carries no importance
                                   weight (log w = 0, J_eff = J, nothing resamples),
                                   every move takes the Metropolis select of
                                   accept_reject, log Z stays 0               */
    /* Optional Gaussian initial distribution q_init = N(m, L L') (Algorithm 3
     * weights the first population by w_1 = pi / q_init; the paper's
     * experiments use N(0, I), Sec. 4).  Host pointers, read and copied by
     * smc_init / smc_init_batch only (the caller keeps ownership; later calls,
     * smc_reset included, use the copies).  NULL: m = 0, L = init_scale * I.
     * With either given, theta_0 = m + L z (z the same standard normals as the
     * isotropic draw; component d summed as m_d + L_d0 z_0 + ... + L_dd z_d in
     * FP64, then rounded to FP32) and log q_init = -|z|^2/2 - (dim/2 log 2 pi
     * + sum_d log L_dd).  Errors (SMC_E_INVAL): a non-finite mean, or a factor
     * whose diagonal is not positive and finite or whose lower triangle is
     * not finite.  The upper triangle is not read. */
    const double* init_mean;    /* [dim] f64, or NULL                              */
    const double* init_chol;    /* [dim x dim] f64 row-major lower-triangular, or NULL */
} smc_config;

typedef struct {
    double ess;             /* J_eff after this iteration's reweighting (Eq. ESS) */
    double ess_pre;         /* J_eff tested for resampling                        */
    double log_z_inc;       /* log sum_j W_j exp(-Delta H_j)                      */
    double mean_alpha;      /* mean HMC acceptance probability                    */
    double traj_len;        /* L used for this iteration's jitter                 */
    int64_t grad_evals;     /* sum_j S_j (gradients evaluated on the trajectory)  */
    int32_t steps_min, steps_max;
    int32_t resampled;
    int32_t pad;
} smc_stats;

typedef struct smc_handle smc_handle;   /* opaque; owned by the library */

/* Creates a sampler, allocates its device state on `stream`, draws theta_0 ~
 * q_init and sets w_1 = pi / q_init (Algorithm 3, first two lines; Eqs. for
 * theta_0 and w_1).  Errors: SMC_E_INVAL (bad config/model), SMC_E_NOMEM,
 * SMC_E_CUDA.  On error *out is NULL. */
smc_status smc_init(smc_handle** out, const smc_config* cfg, const smc_model* model,
                    void* stream);

/* Creates n_runs independent samplers over the same model in one handle; run
 * r uses cfg[r] (particle counts may differ; K, M_warmup and precision must
 * agree).  Kernels process all runs in each launch. */
smc_status smc_init_batch(smc_handle** out, int64_t n_runs, const smc_config* cfg,
                          const smc_model* model, void* stream);

/* One SMC iteration (the loop body of Algorithm 3): normalise, ESS test,
 * systematic resampling, jittered ChEES-HMC move of every particle, reweight
 * by -Delta H, ChEES adaptation.  stats (n_runs entries) may be NULL; when
 * non-NULL the call synchronises the stream and copies the statistics. */
smc_status smc_step(smc_handle* h, smc_stats* stats);

/* n_iters calls of smc_step; per_iter (n_iters * n_runs, iteration-major) may
 * be NULL, in which case nothing synchronises until the caller asks. */
smc_status smc_run(smc_handle* h, int64_t n_iters, smc_stats* per_iter);

/* log Z estimate per run (n_runs doubles, host).  Synchronises the stream. */
smc_status smc_log_evidence(const smc_handle* h, double* out);

/* Copies particles out: theta [dim x N_total] FP32 particle-major (ld =
 * N_total) and log-weights [N_total] FP64.  device_ptrs = 1: the pointers are
 * device pointers on the handle's device; 0: host pointers.  Either may be
 * NULL.  Synchronises the stream. */
smc_status smc_get_particles(const smc_handle* h, float* theta, double* logw,
                             int32_t device_ptrs);

/* Weighted posterior mean and variance (Eq. for realised estimates) of run 0
 * (host arrays of dim doubles). */
smc_status smc_moments(const smc_handle* h, double* mean, double* var);

/* Internal per-particle buffers of the last completed iteration, for
 * inspection and parity tests.  Copies `bytes` bytes into dst (device_ptrs as
 * above).  Buffer ids: */
typedef enum {
    SMC_BUF_THETA = 0,      /* f32 [dim x ld]   current positions                 */
    SMC_BUF_GRAD = 1,       /* f32 [dim x ld]   grad log pi at THETA              */
    SMC_BUF_LOGPI = 2,      /* f64 [N]          log pi at THETA                   */
    SMC_BUF_LOGW = 3,       /* f64 [N]          log-weights                       */
    SMC_BUF_W = 4,          /* f64 [N]          normalised weights before resampling */
    SMC_BUF_ANCESTORS = 5,  /* i32 [N]          ancestors (run-local) if resampled */
    SMC_BUF_STEPS = 6,      /* i32 [N]          leapfrog steps S_j                */
    SMC_BUF_P_FINAL = 7,    /* f32 [dim x ld]   final momenta                     */
    SMC_BUF_DH = 8,         /* f64 [N]          Delta H                           */
    SMC_BUF_ALPHA = 9,      /* f64 [N]          acceptance probabilities          */
    SMC_BUF_THETA_PREV = 10,/* f32 [dim x ld]   positions before the move (after resampling) */
    SMC_BUF_RUNSTATE = 11,  /* f64 [n_runs x 9] log_z, log_L, adam_m, adam_v, Lbar, adam_t, L of the last iteration, its ESS,
                               the step size of the next iteration */
    SMC_BUF_Z0 = 12,        /* f32 [dim x ld]   latent start points z0 = T^-1(theta) of the last move (transport map on) */
    SMC_BUF_Z1 = 13,        /* f32 [dim x ld]   latent end points z' of the last move (transport map on) */
    SMC_BUF_ORDER = 14      /* i32 [N]          launch order of the last move: slot t holds particle
                               perm[t] (handle-wide), step counts non-increasing
                               along the slots; particles with equal counts in
                               any order (a counting sort with atomic slots)   */
} smc_buffer;
smc_status smc_get_buffer(const smc_handle* h, int32_t which, void* dst, int64_t bytes,
                          int32_t device_ptrs);
/* Leading dimension ld of the [dim x ld] buffers, total particle count, runs. */
smc_status smc_get_layout(const smc_handle* h, int64_t* ld, int64_t* n_total, int64_t* n_runs);

/* Restarts every run of the handle from a fresh initial draw (Algorithm 3,
 * first two lines) with seed + r for run r, reusing the device memory:
 * nothing is allocated.  Clears the adaptation state, the evidence and the
 * summary counters; keeps the configuration. */
smc_status smc_reset(smc_handle* h, uint64_t seed);

/* Cumulative counters per run since smc_init / smc_reset. */
typedef struct {
    int64_t iterations;         /* completed SMC iterations                         */
    int64_t grad_evals;         /* sum over iterations of sum_j S_j                 */
    double ess_sum;             /* sum over iterations of J_eff after reweighting   */
    double ess_sum_post_warmup; /* the same over iterations k > M_warmup            */
    double log_z;               /* current log evidence estimate                    */
    int64_t resamples;          /* iterations that resampled                        */
} smc_summary;
smc_status smc_get_summary(const smc_handle* h, smc_summary* per_run);

/* Trajectory-kernel timing with CUDA events recorded on the handle's stream
 * around every trajectory launch while enabled (enable = 1 also clears the
 * totals).  smc_get_profile synchronises and returns the summed device time
 * of those launches in ms, their count, and the number of kernels the library
 * launched while profiling was on. */
smc_status smc_profile(smc_handle* h, int32_t enable);
smc_status smc_get_profile(smc_handle* h, double* traj_ms, int64_t* traj_launches,
                           int64_t* kernel_launches);

/* Launch plan of the trajectory kernel.  smc_init / smc_init_batch run an
 * autotuner once, after the initial draw: every launch-configuration variant
 * of the model's trajectory kernel (CTA size, register cap, one-shot or
 * persistent launch of the thread-per-particle kernels: the persistent form
 * runs as many CTAs as fit at once, each taking tiles of length-sorted
 * particles from a device counter) runs a 16-step trajectory of the handle's own
 * initial particles into the scratch half of the state, timed with CUDA
 * events (best of three), and the fastest is kept.  Variants run the same
 * arithmetic in the same order, so the choice changes speed only, never a
 * result.  smc_get_plan returns the variant in use, the number of variants
 * (1: nothing to tune for this model and precision) and, when tile_ms is not
 * NULL, the measured times in ms (n_tiles values; 0 when not measured). */
smc_status smc_get_plan(const smc_handle* h, int32_t* traj_tile, int32_t* n_tiles, double* tile_ms);

/* Forces variant traj_tile (0 <= traj_tile < n_tiles) from the next iteration
 * on (the captured graph is dropped).  Errors: SMC_E_INVAL. */
smc_status smc_set_plan(smc_handle* h, int32_t traj_tile);

/* Copies the last error text (NUL-terminated, truncated to len). */
smc_status smc_last_error(const smc_handle* h, char* buf, int64_t len);

/* Frees the handle and its device memory (stream-ordered). NULL is a no-op. */
void smc_destroy(smc_handle* h);

/* ------------------------------------------------------------------ transport map
 * A learned preconditioner: an affine-coupling flow theta = T(z) used as a
 * transport map under HMC.  The move of Algorithm 2 runs in the latent space:
 * z0 = T^-1(theta), Algorithm 1 on log pi_z(z) = log pi(T(z)) + log|det dT/dz|
 * with the momentum of Algorithm 2 drawn in z, theta' = T(z').  The energy
 * error Delta H is taken in z and includes the log-determinant, so -Delta H
 * remains the exact incremental log-weight of Sec. 3.1.  ChEES statistics
 * (Algorithm 2) use z0 and z'.  The paper has no learned map; it is this
 * library's preconditioner, and a zero last layer (T = identity) gives back
 * the paper's identity-metric sampler.
 *
 * T = layer_{L-1} o ... o layer_0.  Layer l keeps half A (even l: coordinates
 * 0 .. D/2-1; odd l: D/2 .. D-1) and maps the other half b -> b exp(s) + t,
 * (s_raw, t) = W3 tanh(W2 tanh(W1 a + b1) + b2) + b3, s = 2 tanh(s_raw)
 * (smooth, so that grad log pi_z is continuous).
 * Parameters, per layer, row-major (out x in): W1 [H x D/2], b1 [H],
 * W2 [H x H], b2 [H], W3 [D x H] (rows < D/2 give s_raw, the rest t), b3 [D];
 * smc_flow_num_params values in all.  FP32 on the device.
 *
 * Training: at warm-up iterations k < M_warmup with (k - 1) % train_every ==
 * 0 whose tested J_eff is at least min_ess_frac * J (a near-degenerate
 * weighted set holds a few distinct points, and fitting a density to them
 * collapses the map), after resampling and before the move, `epochs` Adam
 * steps (beta1 0.9,
 * beta2 0.999, eps 1e-8, step lr) descend the weighted negative
 * log-likelihood of the particles under the flow density (without the
 * constant D/2 log 2 pi)
 *     sum_j W_j ( 1/2 |T^-1(theta_j)|^2 - log|det dT^-1/dtheta (theta_j)| ),
 * W_j = 1/J after resampling; particles of zero weight are left out.  The map
 * is frozen from k = M_warmup on.
 */
typedef struct {
    int32_t hidden;         /* H: multiple of 4 in [4, 128], at least dim / 2
                               rounded up to a multiple of 4                      */
    int32_t layers;         /* L: [1, 8]                                          */
    int32_t train_every;    /* train at k - 1 = 0, train_every, ... (0: never)     */
    int32_t epochs;         /* Adam steps per training iteration (0: never train) */
    double lr;              /* Adam step size (> 0)                               */
    double min_ess_frac;    /* train only when J_eff >= min_ess_frac * J, [0, 1]  */
    int32_t precision;      /* conditioner products of the trajectories:
                               SMC_PREC_FP32 (0), or SMC_PREC_BF16 (2): BF16
                               weights and activations on warp-level tensor-core
                               MMAs with FP32 accumulation (hidden a multiple of
                               16)                                                */
    int32_t train_precision;/* products of the training gradient: SMC_PREC_FP32
                               (0), or SMC_PREC_BF16 (2): the conditioner, its
                               transposed products and the weight gradients
                               (sums over particles) on BF16 warp MMAs with FP32
                               accumulation (hidden a multiple of 16); the
                               master weights, bias gradients, the coupling
                               arithmetic and Adam stay FP32                      */
} smc_flow_config;

/* Number of parameters of the flow (0 for an invalid shape). */
int64_t smc_flow_num_params(int64_t dim, int32_t hidden, int32_t layers);

/* Turns the transport map on for a single-run FP32 handle before its first
 * iteration (also restored, with zero Adam moments, by smc_reset).  params:
 * host FP64, smc_flow_num_params(dim, hidden, layers) values, copied and cast
 * to FP32.  Models: GAUSS_DENSE and BANANA with even dim <= 128.
 * Allocates the parameters, Adam moments, gradient, work copies, per-CTA
 * gradient partials and the two latent buffers on the handle's stream.
 * Errors: SMC_E_INVAL (unsupported model / shape / handle state / non-finite
 * parameter; message in smc_last_error), SMC_E_CUDA. */
smc_status smc_flow_enable(smc_handle* h, const smc_flow_config* fc, const double* params);

/* Current (possibly trained) parameters into params (host FP64, n values =
 * smc_flow_num_params).  Synchronises the stream. */
smc_status smc_flow_get_params(const smc_handle* h, double* params, int64_t n);

/* ------------------------------------------------------------------ kernels
 * Kernel-level entry points on caller-owned DEVICE buffers.  They run single
 * stages of the path for parity tests and for callers that drive their own
 * loop.  None allocates device memory except smc_model_create and the two
 * smc_k_flow_* calls (stream-ordered temporaries, freed before returning).
 */
typedef struct smc_dev_model smc_dev_model;

/* Uploads model data to the device (the target of Sec. 2). */
smc_status smc_model_create(smc_dev_model** out, const smc_model* model, void* stream);
void smc_model_destroy(smc_dev_model* m);

/* Philox4x32-10 (Salmon et al., SC'11) blocks: ctr [n x 4] u32 -> out [n x 4]. */
smc_status smc_k_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t n,
                        void* stream);

/* Standard normals of particle slots j = 0..N-1 for (tag, k): out [D x ld] f64,
 * Box-Muller on Philox blocks (i, j, k, tag), i = d / 2.  tag 1: initial draw,
 * 2: momentum (Sec. 2.1, p ~ N(0, I)). */
smc_status smc_k_normals(uint64_t seed, uint32_t tag, uint32_t k, int64_t N, int64_t D,
                         double* out, int64_t ld, void* stream);

/* Jittered step counts (Algorithm 2: ceil(h L / eps), clipped to [1, max]):
 * h_j = radical inverse base 2 of n = j*K + k (jitter = 1) or 1 (jitter = 0;
 * the other schemes: smc_k_jitter);
 * out_h [N] f64 (may be NULL), out_steps [N] i32. */
smc_status smc_k_steps(int64_t N, int64_t K, int64_t k, double L, double eps,
                       int32_t max_steps, int32_t jitter, double* out_h, int32_t* out_steps,
                       void* stream);

/* Jitter h of particles j = 0..J-1 (the paper's j - 1) at iteration k (1 <= k
 * <= K) under scheme 0..11 (Sec. 3.2.1; the list at smc_config.jitter), as the
 * sampler computes it: out_h [J] f64, device.  For j (0-based), iteration k:
 *   1 1-d Halton: radical inverse base 2 of n = j*K + k;
 *   2 uniform: (m + 1/2) 2^-52, m the 52-bit integer of words 0, 1 of Philox
 *     block (0, j, k, 5);
 *   3 / 4 N-d Halton / inverse: radical inverse of j + 1 in base P_k /
 *     P_{K+1-k} (P_m the m-th prime), the exact fraction rounded once;
 *   5 / 6 N-d primes / inverse: frac((j + 1) sqrt(P_k)) / with P_{K+1-k};
 *   7 golden ratio: frac((j*K + k)(sqrt(5) - 1)/2);
 *   8 equidistant: (s_k(j) + 1) / J, s_k the shuffle of iteration k: the
 *     four-round Feistel network on 2 ceil(log4 J) bits whose round r xors
 *     word 0 of Philox block (x, r, k, 6) (masked to half the bits) into the
 *     other half, applied until the value is below J;
 *   9 offset equidistant: that + 0.1 u, u the uniform of block (1, j, k, 5);
 *   10 1-d Sobol: radical inverse base 2 of g = n ^ (n >> 1), n = j*K + k;
 *   11 1-d Halton of n = (k-1)*J + j + 1 (the J x K index matrix of 1 read
 *      iteration-major).
 * Every FP64 operation rounds once, in the order written.  Errors:
 * SMC_E_INVAL (scheme, sizes, J*K + k >= 2^32, K > 65536 for 3-6). */
smc_status smc_k_jitter(int32_t scheme, uint64_t seed, int64_t J, int64_t K, int64_t k, double* out_h,
                        void* stream);

/* log pi and grad log pi (Sec. 2) at theta [D x ld] f32: logpi [N] f64,
 * grad [D x ld] f32. */
smc_status smc_k_target(const smc_dev_model* m, const float* theta, int64_t N, int64_t ld,
                        double* logpi, float* grad, int32_t precision, void* stream);

/* steps[j] leapfrog steps (Eqs. for p_{l+1/2}, theta_{l+1}, p_{l+1};
 * Algorithm 1) with step size eps, in place on theta, p, grad [D x ld] f32 and
 * logpi [N] f64 (which must hold grad log pi and log pi at the start).  On
 * return logpi holds log pi at the end point. */
smc_status smc_k_leapfrog(const smc_dev_model* m, float* theta, float* p, float* grad,
                          double* logpi, const int32_t* steps, double eps, int64_t N,
                          int64_t ld, int32_t precision, void* stream);

/* The preconditioned move of smc_flow_enable for N particles with given
 * latent momenta: params device FP32 (smc_flow_num_params values); theta,
 * grad (= grad log pi at theta), p (latent momenta) f32 [dim x ld] and logpi
 * f64 [N] are updated in place (theta' = T(z'), its gradient and log pi, the
 * final latent momenta); steps i32 [N] (>= 1); z0, z1 (f32 [dim x ld], may be
 * NULL) receive T^-1(theta) and z'; dH (f64 [N], may be NULL) the energy
 * error in z.  precision: SMC_PREC_FP32 or SMC_PREC_BF16 (conditioner products
 * on BF16 warp MMAs, as smc_flow_config.precision).  Allocates (stream-ordered)
 * and frees the padded work copies of the weights. */
smc_status smc_k_flow_leapfrog(const smc_dev_model* m, int32_t hidden, int32_t layers,
                               const float* params, float* theta, float* p, float* grad,
                               double* logpi, const int32_t* steps, double eps, int64_t N,
                               int64_t ld, float* z0, float* z1, double* dH, int32_t precision,
                               void* stream);

/* Gradient of the weighted training loss of smc_flow_enable with respect to
 * every parameter: grad (device f32, smc_flow_num_params values) from params
 * (device f32), theta f32 [dim x ld] and W f64 [N] (used as given, not
 * normalised).  precision: SMC_PREC_FP32, or SMC_PREC_BF16 (the products on
 * BF16 warp MMAs, as smc_flow_config.train_precision).  Per-CTA partial
 * gradients are summed in a fixed order, so the result is deterministic.
 * Allocates (stream-ordered) and frees the work copies, the BF16 fragments
 * and the partials (ceil(N / 32) x n_params floats).  Errors: SMC_E_INVAL
 * (shape, precision, null pointers, ld < N), SMC_E_NOMEM, SMC_E_CUDA. */
smc_status smc_k_flow_loss_grad(int64_t dim, int32_t hidden, int32_t layers, const float* params,
                                const float* theta, const double* W, int64_t N, int64_t ld,
                                float* grad, int32_t precision, void* stream);

/* Normalised weights (Sec. 3): lse, ess (device scalars, f64) and W [N] f64
 * from logw [N] f64. */
smc_status smc_k_normalise(const double* logw, int64_t N, double* W, double* lse,
                           double* ess, void* stream);

/* Fixed-point systematic resampling: q_j = floor(W_j 2^S), S = 62 -
 * ceil(log2 N); T = sum q (exact, uint64); U = floor(r64 T / 2^64); ancestor
 * of output i = smallest j with N C_j > i T + U (C = inclusive prefix of q,
 * by a decoupled look-back scan).  W is read-only; writes q [N] u64,
 * ancestors [N] i32 and *status_out (device i32: 0 ok, -4 T == 0, -5 the
 * look-back wait gave up).  Uses `scratch` (device, caller-allocated, at least
 * smc_k_resample_scratch_bytes(N) bytes, 256-byte aligned) for the tile
 * descriptors; its contents on entry do not matter.  N <= 2^30. */
int64_t smc_k_resample_scratch_bytes(int64_t N);
smc_status smc_k_resample(const double* W, int64_t N, uint64_t r64, uint64_t* q,
                          int32_t* ancestors, int32_t* status_out, void* scratch,
                          void* stream);

/* Failure detection of the resampling scan's bounded wait (the paper has no
 * counterpart: it concerns this library's look-back scan for the resampling
 * step of Algorithm 3).  Runs the scan's look-back for tile 1 of a two-tile
 * run whose tile 0 never publishes its prefix, giving up after poll_limit
 * polls without progress (about 64 ns each; the sampler uses 2^22).  Writes
 * *status_out (device i32): -5 when the wait gave up, as the sampler reports
 * SMC_E_TIMEOUT for a run.  scratch: device, at least 64 bytes, 16-byte
 * aligned, overwritten.  Returns SMC_E_INVAL for poll_limit outside
 * [1, 2^40] or null pointers, SMC_E_CUDA if the launch fails; the GPU
 * context stays usable. */
smc_status smc_k_lookback_wait_check(int64_t poll_limit, int32_t* status_out, void* scratch, void* stream);

/* Systematic resampling exactly as smc_k_resample, for callers that cannot
 * allocate device memory where they resample (a host framework that owns the
 * whole device memory budget, or a latency-critical loop that cannot afford
 * the device synchronisation implied by cudaMalloc / cudaFree).  The paper has
 * no counterpart: it is an interface convenience of this library.
 * Allocates nothing: the scan descriptors live in a fixed 64 KiB device array
 * inside the library (present on every device that loads it, until the
 * process exits), so N is limited to SMC_NOALLOC_MAX_N; larger N returns
 * SMC_E_INVAL with a message on stderr.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current) and caches it; make that first call before any stream capture.
 * The cached address belongs to the device's primary context: after
 * cudaDeviceReset, or anything else that destroys that context, the library
 * must be unloaded and loaded again before the next call.
 * Every call shares the one array, and each call clears the part it uses
 * before reading it; calls whose work overlaps on the GPU (other streams,
 * other host threads) race on it and must be serialised by the caller.
 * Arguments, outputs and status codes are those of smc_k_resample. */
#define SMC_NOALLOC_MAX_N 4194304
smc_status smc_k_resample_noalloc(const double* W, int64_t N, uint64_t r64, uint64_t* q,
                                  int32_t* ancestors, int32_t* status_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
