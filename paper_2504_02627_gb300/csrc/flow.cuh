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
// For the BF16 form the six conditioner matrices of every layer (W1, W2, W3
// and their transposes for the backward products) are also kept as BF16
// operand fragments of the m16n8k16 MMA: per 16 x 16 tile, 32 lanes x 16
// bytes in the order the lanes load them (kp1 = Dh and o4p = O4 rounded up to
// 16 are the padded tile extents).
struct DevFlow {
    int32_t D, H, L, Dh, Dh4, O4;
    int32_t kp1, o4p;            // Dh, O4 rounded up to 16
    int32_t bf16;                // 1: conditioner products on warp-level BF16 MMAs
    int32_t train_bf16;          // 1: the training gradient's products on warp-level BF16 MMAs
    int64_t n_params;            // canonical parameter count
    int64_t layer_work;          // floats per layer of the work copies
    int64_t layer_frag;          // 16-byte fragments per layer of the BF16 copies
    float* params;               // [n_params]
    float* adam_m;               // [n_params]
    float* adam_v;               // [n_params]
    float* grad;                 // [n_params]
    float* work;                 // [L x layer_work]
    uint4* frag;                 // [L x layer_frag]
    int32_t* adam_t;             // device Adam step count (steps taken)
};

// Offsets (in fragments) of the six BF16 operand matrices inside one layer:
// W1 [H x kp1], W2 [H x H], W3 [o4p x H] (rows in the padded output order),
// W1t [kp1 x H], W2t [H x H], W3t [H x o4p]; each 32 x (rows/16) x (cols/16).
struct FlowFragOff {
    int64_t W1, W2, W3, W1t, W2t, W3t, total;
};
__host__ __device__ inline FlowFragOff flow_frag_off(int H, int kp1, int o4p) {
    const int64_t h = H / 16, k = kp1 / 16, o = o4p / 16;
    FlowFragOff f;
    f.W1 = 0;
    f.W2 = f.W1 + 32 * h * k;
    f.W3 = f.W2 + 32 * h * h;
    f.W1t = f.W3 + 32 * o * h;
    f.W2t = f.W1t + 32 * k * h;
    f.W3t = f.W2t + 32 * h * h;
    f.total = f.W3t + 32 * h * o;
    return f;
}
// The BF16 form needs H a multiple of 16, at most 128.
inline bool flow_bf16_ok(int H) { return H % 16 == 0 && H >= 16 && H <= 128; }

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
// Shapes with a kernel: D even in [2, 128], H a multiple of 4 in [4, 128] and at
// least D/2 rounded up to 4, L in [1, 8].
bool flow_shape_ok(int64_t D, int64_t H, int64_t L);
bool flow_supported(const DevModel& m, int H, int L);
// ... and the BF16 form of it (H a multiple of 16, room for its operand buffer)
bool flow_bf16_supported(int64_t D, int H, int L);
// ... and BF16 training (H a multiple of 16, room for the BF16 operands of the
// weight-gradient products)
bool flow_train_bf16_supported(int64_t D, int H, int L);
// Sizes of a flow of this shape; the pointers are left null.
DevFlow flow_shape(int D, int H, int L);
size_t flow_smem_bytes(int D, int H, int L, int O4);
// Rebuild the padded / transposed work copies (and the BF16 fragments, when
// f.frag is set) from params.  With `bump`, the launch also counts the Adam
// step that preceded it (when the gate was open).
cudaError_t flow_refresh(const DevFlow& f, cudaStream_t s, bool bump = false, FlowGate gate = FlowGate{});
// HMC in z = T^-1(theta) with the frozen map (trajectory kernel); z0 and z1
// (may be nullptr) receive the latent start and end points [D x ld].
cudaError_t launch_traj_flow(const DevModel& m, const DevFlow& f, const TrajArgs& a, float* z0, float* z1,
                             cudaStream_t s);
// Gradient of the weighted NLL of the particles (theta gathered through src,
// weights 1/n after resampling, else W) into f.grad, using `partials`
// (n_blocks x n_params floats) for a fixed-order reduction; with f.train_bf16
// the conditioner, transposed and weight-gradient products run on BF16 warp
// MMAs (f.frag must hold the fragments of the current params).
int64_t flow_partials_floats(const DevFlow& f, int64_t N);
// gate.rs / gate.rp describe the single run of the handle (nullptr: weights W
// as given, always open).
cudaError_t flow_loss_grad(const DevFlow& f, const float* theta, int64_t ld, const int32_t* src, const double* W,
                           FlowGate gate, int64_t N, float* partials, cudaStream_t s);
// One Adam step (descent) on f.params from f.grad, step number *f.adam_t + 1
// (the following flow_refresh with bump counts it).
cudaError_t flow_adam(const DevFlow& f, double lr, FlowGate gate, cudaStream_t s);

}  // namespace smc
