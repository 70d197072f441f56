// flow.cuh -- learned preconditioner: an affine-coupling flow theta = T(z)
// used as a transport map under HMC, and its training on weighted particles.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "smc_kernels.cuh"
#include "traj.cuh"

namespace smc {

// Device copy of the flow.  `params` is the canonical FP32 vector (per layer,
// row-major out x in: W1 [H x Dh], b1 [H], W2 [H x H], b2 [H], W3 [D x H],
// b3 [D]; rows 0..Dh-1 of W3 give s_raw, rows Dh..D-1 give t).  The work
// copies below are rebuilt from it after every update, padded so that every
// row is 16-byte aligned (Dh4 = Dh rounded up to 4, O4 = 2 Dh4 output rows).
struct DevFlow {
    int32_t D, H, L, Dh, Dh4, O4;
    int64_t n_params;            // canonical parameter count
    int64_t layer_work;          // floats per layer of the work copies
    float* params;               // [n_params]
    float* adam_m;               // [n_params]
    float* adam_v;               // [n_params]
    float* grad;                 // [n_params]
    float* work;                 // [L x layer_work]
    int32_t* adam_t;             // device Adam step count (steps taken)
};

// Training gate: a training epoch runs only when the run's tested ESS is at
// least frac * n (rs == nullptr: always).  Evaluated on the device, so a
// training iteration needs no host round trip.
struct FlowGate {
    const RunState* rs;
    const RunParams* rp;
    double frac;
    __device__ bool open() const { return rs == nullptr || rs->ess_pre >= frac * (double)rp->n; }
};

// Offsets inside one layer of the work copies.
struct FlowLayerOff {
    int64_t W1t, W1, b1, W2t, W2, b2, W3t, W3, b3;
};
__host__ __device__ inline FlowLayerOff flow_layer_off(int H, int Dh, int Dh4, int O4) {
    FlowLayerOff o;
    o.W1t = 0;                       // [Dh][H]   forward  (K = Dh, out = H)
    o.W1 = o.W1t + (int64_t)Dh * H;  // [H][Dh4]  backward (K = H,  out = Dh4)
    o.b1 = o.W1 + (int64_t)H * Dh4;  // [H]
    o.W2t = o.b1 + H;                // [H][H]
    o.W2 = o.W2t + (int64_t)H * H;   // [H][H]
    o.b2 = o.W2 + (int64_t)H * H;    // [H]
    o.W3t = o.b2 + H;                // [H][O4]   forward  (K = H,  out = O4)
    o.W3 = o.W3t + (int64_t)H * O4;  // [O4][H]   backward (K = O4, out = H)
    o.b3 = o.W3 + (int64_t)O4 * H;   // [O4]
    (void)Dh4;
    return o;
}
inline int64_t flow_layer_work(int H, int Dh, int Dh4, int O4) {
    return (int64_t)Dh * H + (int64_t)H * Dh4 + H + 2 * (int64_t)H * H + H + 2 * (int64_t)H * O4 + O4;
}

inline int64_t flow_num_params(int64_t D, int64_t H, int64_t L) {
    return L * (H * (D / 2) + H + H * H + H + D * H + D);
}
// Shapes with a kernel: D even in [2, 128], H a multiple of 4 in [4, 128], L in [1, 8].
bool flow_shape_ok(int64_t D, int64_t H, int64_t L);
bool flow_supported(const DevModel& m, int H, int L);
// Sizes of a flow of this shape; the pointers are left null.
DevFlow flow_shape(int D, int H, int L);
size_t flow_smem_bytes(int D, int H, int L, int O4);
// Rebuild the padded / transposed work copies from params.  With `bump`, the
// launch also counts the Adam step that preceded it (when the gate was open).
cudaError_t flow_refresh(const DevFlow& f, cudaStream_t s, bool bump = false, FlowGate gate = FlowGate{});
// HMC in z = T^-1(theta) with the frozen map (trajectory kernel); z0 and z1
// (may be nullptr) receive the latent start and end points [D x ld].
cudaError_t launch_traj_flow(const DevModel& m, const DevFlow& f, const TrajArgs& a, float* z0, float* z1,
                             cudaStream_t s);
// Gradient of the weighted NLL of the particles (theta gathered through src,
// weights 1/n after resampling, else W) into f.grad, using `partials`
// (n_blocks x n_params floats) for a fixed-order reduction.
int64_t flow_partials_floats(const DevFlow& f, int64_t N);
// gate.rs / gate.rp describe the single run of the handle (nullptr: weights W
// as given, always open).
cudaError_t flow_loss_grad(const DevFlow& f, const float* theta, int64_t ld, const int32_t* src, const double* W,
                           FlowGate gate, int64_t N, float* partials, cudaStream_t s);
// One Adam step (descent) on f.params from f.grad, step number *f.adam_t + 1
// (the following flow_refresh with bump counts it).
cudaError_t flow_adam(const DevFlow& f, double lr, FlowGate gate, cudaStream_t s);

}  // namespace smc
