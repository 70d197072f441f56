// traj.cuh -- interfaces between the host driver and the trajectory kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"

namespace smc {

enum ModelKind : int32_t { GAUSS_DENSE = 0, LOGISTIC = 1, HIER_NORMAL = 2, BANANA = 3, LINEAR_GAUSS = 4 };

// Device-resident target (Sec. 2 of the paper).  FP32 copies of the data;
// X is row-major [n x Dp] with Dp = D rounded up to a multiple of 4 and
// zero padding.  lconst holds the additive FP64 constant of log pi that does
// not depend on theta (normalisers), computed once on the host.
struct DevModel {
    int32_t kind, D, Dp, n;
    const float* X;       // [n x Dp]
    const float* y;       // [n]
    const float* mu;      // [D]         GAUSS_DENSE
    const float* P;       // [D x D]     GAUSS_DENSE
    const float* gmean;   // [n]         HIER_NORMAL group means
    const float* gn;      // [n]         group sizes
    const float* gss;     // [n]         within-group sums of squares
    const uint16_t* Xbf;  // [n x Dp] bf16 (high part), tensor-core paths
    const uint16_t* Xbf_lo; // [n x Dp] bf16 residual x - bf16(x)
    // D <= 32: X hi and lo as two [n16][32] bf16 row blocks (rows padded to a
    // multiple of 16, dims to 32, zeros) in the warp-MMA kernel's swizzled
    // shared-memory order, so staging them is a straight 16-byte copy
    const uint16_t* xmma_img;
    double h0, h1;        // LOGISTIC: tau; LINEAR: sigma, tau; HIER: sigma; BANANA: a, b
    double lconst;        // theta-independent part of log pi
    // Streamed tensor-core operands (GEMM-shaped models with D <= 128): X in
    // BF16 as per-chunk shared-memory images of STREAM_CHUNK observations,
    // already in the 128-byte-swizzled K-major layouts the MMAs read, so one
    // contiguous bulk copy per chunk stages them:
    //   xk_img chunk c: 2 atoms x [STREAM_CHUNK obs rows x 64 dims] (16 KB)
    //   xt_img chunk c: [dkr dim rows x STREAM_CHUNK obs] (dkr x 128 bytes)
    //   y_img  chunk c: STREAM_CHUNK floats (zero past n)
    const uint16_t* xk_img;
    const uint16_t* xt_img;
    const float* y_img;
    int32_t dk;           // D rounded up to 16 (MMA K of the first product, N of the second)
    int32_t n_chunks;
    // Centred tensor-core path: X in BF16 as tiles of CENTRED_CHUNK
    // observations, [ceil(dk / 64) atoms][CENTRED_CHUNK obs rows][128 B], an
    // atom holding 64 dimensions in the 128-byte swizzle (16-byte unit u of
    // row r at unit u ^ (r & 7)); zeros past n and past D.
    const uint16_t* xc_img;
    int32_t n_tiles128;
};
constexpr int STREAM_CHUNK = 64;
constexpr int CENTRED_CHUNK = 128;
constexpr int CENTRED_MAX_RUNS = 16;   // runs of one handle the centred path serves

// What a trajectory launch reads and writes.  Slot t of the launch handles
// particle j = perm ? perm[t] : t; it starts from source index src[j] (the
// resampled ancestor) or j; outputs go to index j.
struct TrajArgs {
    const float* theta_in; const float* grad_in; const double* logpi_in;
    float* theta_out; float* grad_out; double* logpi_out;
    const float* p_in;      // momenta given by the caller (nullptr: draw from Philox)
    float* p_out;           // final momenta (may be nullptr)
    double* dH;             // Delta H (may be nullptr)
    double* alpha;          // min(1, exp(-Delta H)) (may be nullptr)
    const int32_t* steps;   // S_j
    const int32_t* perm;    // slot -> particle (may be nullptr)
    const int32_t* src;     // particle -> source index (may be nullptr)
    const int32_t* run_of;  // particle -> run (may be nullptr: run 0)
    const RunParams* runs;  // per-run parameters (may be nullptr if eps_fixed used)
    const RunState* rstate; // per-run state: k for the momentum counter
    double eps_fixed;       // step size when runs == nullptr
    int64_t N, ld;
    int32_t eval_only;      // 1: compute log pi and grad at theta_in, no move
    int32_t tile;           // launch-configuration variant of the model's kernel (0: default)
    int* dev_err;           // set to 1 when a bounded device wait gives up (may be nullptr)
    unsigned int* work;     // tile counter of the persistent launch variants (may be nullptr)
    // centred tensor-core path only: per-move reference quantities of each
    // run (written by the launcher before the trajectory kernel)
    float* c_centre;        // [c_runs][dk] reference points theta_ref
    float* c_gref;          // [c_runs][dk] reference gradients X'(y - s)
    float2* c_refs;         // [n_tiles128][c_runs][CENTRED_CHUNK / 2] observation pairs, each as the floats
                            // (c0, c1, s0, s1): c = -log2(e) eta_ref, s = sigmoid(eta_ref)
    double* c_part;         // [n_tiles128][c_runs][dk] per-tile parts of c_gref
    int32_t c_runs;         // runs in these arrays (1 when runs == nullptr)
    int32_t c_split;        // CTAs per particle tile (observation split), set by the launcher
    // optional [D x c_sld] f32 buffers for the move's theta and p in slot
    // order (so the per-pass update reads and writes them coalesced);
    // nullptr: the move keeps its state in theta_out / p_out at the
    // particles' indices
    float* c_sth;
    float* c_sp;
    int64_t c_sld;
    // several runs: every particle tile holds one run's particles.  Run r's
    // particles take the slots [c_padoff[r], c_padoff[r] + n_r) in the order
    // of perm (a stable partition of it, written into c_perm by the
    // launcher; the slots up to the next multiple of 128 hold -1), and tile b
    // covers the 128 slots from c_tiles[b].y, all of run c_tiles[b].x.
    // nullptr: tiles are the slots of perm in order (one run).
    const int2* c_tiles;
    int32_t* c_perm;
    const int32_t* c_padoff;
    int32_t* c_pcnt;        // partition scratch: [ceil(N / 1024)][c_runs] counts, then bases
    int64_t c_ntiles;       // tiles of the launch when c_tiles is set
};

// Run of particle j: step size, Philox key, iteration and run-local index.
__device__ __forceinline__ void particle_run(const TrajArgs& a, int64_t j, int& r, double& eps,
                                             uint64_t& seed, uint32_t& kk, uint32_t& jl) {
    r = a.run_of ? a.run_of[j] : 0;
    if (a.runs) {
        eps = a.rstate ? a.rstate[r].eps : a.runs[r].eps;
        seed = a.runs[r].seed;
        jl = (uint32_t)(j - a.runs[r].off);
    } else {
        eps = a.eps_fixed;
        seed = 0;
        jl = (uint32_t)j;
    }
    kk = a.rstate ? (uint32_t)a.rstate[r].k : 0u;
}

// Launchers (kernels in traj_simt.cu / traj_tc.cu).  Return cudaError_t of
// the launch; `supported` reports whether the model/shape has a kernel.
bool traj_supported(const DevModel& m, int32_t precision);
// warp-MMA GLM kernel's X image (DevModel::xmma_img): elements to allocate for
// n observations, and the kernel that fills it from the BF16 hi / lo rows
int64_t glm_mma_image_elems(int64_t n);
cudaError_t build_glm_mma_image(const uint16_t* xh, const uint16_t* xl, int64_t n, int D, int Dp,
                                uint16_t* img, cudaStream_t s);
// Launch-configuration variants of the model's trajectory kernel that the
// host autotuner may choose between (1: nothing to choose).  Every variant
// runs the same arithmetic in the same order, so the choice never changes a
// result, only its speed.
int32_t traj_tile_count(const DevModel& m, int32_t precision);
// thread-per-particle kernels (traj_thread.cu): dense Gaussian D <= 32,
// banana, hierarchical normal; FP32
cudaError_t launch_traj_thread(const DevModel& m, const TrajArgs& a, cudaStream_t s);
int32_t traj_thread_tiles(const DevModel& m);
cudaError_t launch_traj(const DevModel& m, const TrajArgs& a, int32_t precision, cudaStream_t s);
// tensor-core path (traj_tc.cu): logistic / linear regression, BF16 or BF16x3
bool traj_tc_supported(const DevModel& m);
cudaError_t launch_traj_tc(const DevModel& m, const TrajArgs& a, bool x3, cudaStream_t s);
// streamed tensor-core path (traj_tc_stream.cu): any n, D <= 128; np = 1
// (BF16 state operands) or 2 (state operands split into BF16 hi + lo)
// FP32 SIMT path for regression data that do not fit in shared memory
// (traj_glm_stream.cu): X streamed in chunks, D <= 128
bool traj_glm_stream_supported(const DevModel& m);
// warp-level BF16 tensor-core path with X resident in shared memory
// (traj_glm_mma.cu): D <= 32, n up to about 1300 (x3) / 2400 (BF16)
bool traj_glm_mma_supported(const DevModel& m, bool x3);
// warp-level BF16 tensor-core path for the dense Gaussian (traj_gauss_mma.cu): D <= 128
bool traj_gauss_mma_supported(const DevModel& m);
cudaError_t launch_traj_gauss_mma(const DevModel& m, const TrajArgs& a, bool x3, cudaStream_t s);
cudaError_t launch_traj_glm_mma(const DevModel& m, const TrajArgs& a, bool x3, cudaStream_t s);
cudaError_t launch_traj_glm_stream(const DevModel& m, const TrajArgs& a, cudaStream_t s);
bool traj_stream_supported(const DevModel& m);
cudaError_t launch_traj_stream(const DevModel& m, const TrajArgs& a, int np, cudaStream_t s);
// centred tensor-core path (traj_centred.cu): any n, D <= 128, precision 4;
// the caller provides the TrajArgs::c_* arrays (sizes below)
bool traj_centred_supported(const DevModel& m);
int64_t centred_refs_elems(const DevModel& m, int n_runs);
int64_t centred_part_elems(const DevModel& m, int n_runs);
cudaError_t launch_traj_centred(const DevModel& m, const TrajArgs& a, cudaStream_t s);

}  // namespace smc
