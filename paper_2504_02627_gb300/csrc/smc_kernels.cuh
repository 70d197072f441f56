// smc_kernels.cuh -- launchers of the per-iteration SMC kernels (smc_kernels.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"

namespace smc {

// Decoupled look-back descriptor of one scan tile: aggregate and inclusive
// prefix (uint64), published with an epoch-tagged flag.
struct TileDesc {
    unsigned long long agg;
    unsigned long long incl;
    unsigned int flag;      // (epoch << 2) | {0: not ready, 1: aggregate, 2: prefix}
    unsigned int pad;
};
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Partial results of one particle slice, combined in a fixed order.
struct SlicePart {
    double za_m, za_s;      // log-sum-exp pieces of log W_j - Delta H_j
    double w_m, w_e1, w_e2; // max, sum exp, sum exp^2 of the new log-weights
    double alpha_sum;
    double inv_alpha_sum;   // sum 1/alpha_j (step-size rule; +inf if some alpha_j = 0)
    double g_num, g_den;    // ChEES: sum alpha_j g_j, sum alpha_j
    long long steps_sum;
    int smin, smax;
};

// Per-iteration buffers shared by the stage kernels.
struct StepBufs {
    const RunParams* runs;
    RunState* rstate;
    const int32_t* run_of;      // particle -> run
    const int32_t* tile_run;    // scan tile -> run
    int64_t n_runs, N, ld, D;
    double* logw;               // [N]
    double* W;                  // [N]
    unsigned long long* q;      // [N]
    unsigned long long* cprefix;  // [N] inclusive prefix of q within each multinomial run (scan output)
    const int32_t* primes;      // the first K primes (N-d jitter schemes), else nullptr
    int32_t* anc;               // [N] run-local ancestor of each output slot
    int32_t* src;               // [N] global source index of each particle
    int32_t* steps;             // [N]
    int32_t* perm;              // [N] slot -> particle (sorted by steps, descending)
    int32_t* hist;              // [max_steps + 1]
    unsigned int* counter;      // dynamic tile counter + sort scratch
    TileDesc* tiles;
    int64_t n_tiles;
    int32_t max_steps_all;
    int32_t any_multinomial;    // some run resamples multinomially
    // particle slices of the weight / statistics kernels
    const int32_t* slice_run;   // slice -> run
    const int32_t* slice_start; // slice -> first run-local particle
    int64_t n_slices;
    SlicePart* parts;           // [n_slices]
    double* colsum;             // [n_slices x 2D] ChEES column sums
    unsigned int* done;         // [n_runs] slice tickets
    // trajectory results
    const float* theta_prev;    // positions before the move (source buffer)
    float* theta_new;           // proposals (replaced by the start state when rejected)
    const float* grad_prev;
    float* grad_new;
    const double* logpi_prev;
    double* logpi_new;
    const float* p_final;
    const double* dH;
    const double* alpha;
    // latent start / end points [D x ld] of the preconditioned move (indexed
    // by particle); when set, the ChEES statistics use them instead of theta
    const float* chees0;
    const float* chees1;
};

// One iteration = weights_steps, resample_scan, sort, trajectory kernel,
// move_stats (each launch covers every run).
cudaError_t launch_init_draw(const StepBufs& b, float* theta, cudaStream_t s);
cudaError_t launch_init_finish(const StepBufs& b, const double* logpi, cudaStream_t s);
cudaError_t launch_weights_steps(const StepBufs& b, cudaStream_t s);
cudaError_t launch_resample_scan(const StepBufs& b, cudaStream_t s);
cudaError_t launch_lookback_wait_check(long long limit, TileDesc* tiles, int* status, cudaStream_t s);
cudaError_t launch_sort(const StepBufs& b, cudaStream_t s);
cudaError_t launch_move_stats(const StepBufs& b, cudaStream_t s);
constexpr int KERNELS_PER_ITERATION = 7;   // kernels launched by one smc_step
constexpr int MAX_CHEES_DIM = 256;         // D handled by the fused ChEES statistics

// Kernel-level entry points (stand-alone buffers).
cudaError_t launch_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t n, cudaStream_t s);
cudaError_t launch_normals(uint64_t seed, uint32_t tag, uint32_t k, int64_t N, int64_t D, double* out,
                           int64_t ld, cudaStream_t s);
cudaError_t launch_jitter_only(int32_t scheme, uint64_t seed, int64_t J, int64_t K, int64_t k,
                               const int32_t* primes, double* out_h, cudaStream_t s);
cudaError_t launch_steps_only(int64_t N, int64_t K, int64_t k, double L, double eps, int32_t max_steps,
                              int32_t jitter, double* out_h, int32_t* out_steps, cudaStream_t s);
cudaError_t launch_normalise_flat(const double* logw, int64_t N, double* W, double* lse, double* ess,
                                  cudaStream_t s);
// Stand-alone resampling: scratch layout = [RunParams][RunState][TileDesc x tiles][counter].
int64_t resample_scratch_bytes(int64_t N);
cudaError_t launch_resample_flat(const double* W, int64_t N, uint64_t r64, unsigned long long* q,
                                 int32_t* anc, int32_t* status, void* scratch, cudaStream_t s);

}  // namespace smc
