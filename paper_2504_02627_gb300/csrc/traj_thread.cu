// traj_thread.cu -- thread-per-particle leapfrog trajectories (Algorithm 1)
// for targets whose gradient is cheap per particle: the dense Gaussian with
// D <= 32, the banana and the non-centred hierarchical normal.  One thread
// carries theta, p and grad of its particle in registers for the whole
// trajectory, draws its momentum from the (seed, i, j, k, MOM) Philox stream
// and returns the end-point energy error Delta H and min(1, exp(-Delta H)).
#include <algorithm>
#include <cstdio>
#include <math_constants.h>
#include "traj.cuh"

namespace smc {

// ============================================================ thread models
template <int DM>
struct GaussDenseM {
    static size_t smem_bytes(const DevModel& m) { return (size_t)(m.D * m.D + m.D) * sizeof(float); }
    __device__ static void load(const DevModel& m, float* sm) {
        for (int i = threadIdx.x; i < m.D * m.D; i += blockDim.x) sm[i] = m.P[i];
        for (int i = threadIdx.x; i < m.D; i += blockDim.x) sm[m.D * m.D + i] = m.mu[i];
    }
    // grad log pi = -P (theta - mu)
    __device__ static void grad(const DevModel& m, const float* sm, const float (&th)[DM], float (&g)[DM]) {
        const int D = m.D;
        const float* P = sm;
        const float* mu = sm + D * D;
        float dl[DM];
#pragma unroll
        for (int d = 0; d < DM; ++d) dl[d] = d < D ? th[d] - mu[d] : 0.0f;
#pragma unroll
        for (int a = 0; a < DM; ++a) {
            float acc = 0.0f;
            if (a < D) {
#pragma unroll
                for (int b = 0; b < DM; ++b)
                    if (b < D) acc = fmaf(P[a * D + b], dl[b], acc);
            }
            g[a] = -acc;
        }
    }
    // log pi = c - 1/2 (theta - mu)' P (theta - mu) = c + 1/2 (theta - mu)' g
    // with g = -P (theta - mu) the FP32 gradient at theta: FP32 products,
    // FP64 accumulation (the FP64 quadratic form costs D^2 operations at the
    // FP64 rate, a small fraction of the FP32 rate here)
    __device__ static double logpi(const DevModel& m, const float* sm, const float (&th)[DM],
                                   const float (&g)[DM]) {
        const float* mu = sm + m.D * m.D;
        double q = 0.0;
#pragma unroll
        for (int d = 0; d < DM; ++d)
            if (d < m.D) q += (double)((th[d] - mu[d]) * g[d]);
        return m.lconst + 0.5 * q;
    }
};

// Banana pairs (Sec. 4, Rosenbrock): x_o ~ N(0, a), x_e ~ N(b (x_o^2 - a), 1).
template <int DM>
struct BananaM {
    static size_t smem_bytes(const DevModel&) { return 0; }
    __device__ static void load(const DevModel&, float*) {}
    __device__ static void grad(const DevModel& m, const float*, const float (&th)[DM], float (&g)[DM]) {
        const float a = (float)m.h0, b = (float)m.h1, inva = (float)(1.0 / m.h0);
#pragma unroll
        for (int i = 0; i + 1 < DM; i += 2) {
            if (i + 1 < m.D) {
                float xo = th[i], xe = th[i + 1];
                float u = xe - b * (xo * xo - a);
                g[i] = -xo * inva + 2.0f * b * u * xo;
                g[i + 1] = -u;
            } else {
                g[i] = 0.0f;
                g[i + 1] = 0.0f;
            }
        }
        if (DM & 1) g[DM - 1] = 0.0f;
    }
    // FP32 terms per pair, FP64 accumulation
    __device__ static double logpi(const DevModel& m, const float*, const float (&th)[DM], const float (&)[DM]) {
        const float a = (float)m.h0, b = (float)m.h1, half_inva = (float)(0.5 / m.h0);
        double s = 0.0;
#pragma unroll
        for (int i = 0; i + 1 < DM; i += 2) {
            if (i + 1 < m.D) {
                const float xo = th[i], xe = th[i + 1];
                const float u = xe - b * (xo * xo - a);
                s += (double)(-half_inva * xo * xo - 0.5f * u * u);
            }
        }
        return s + m.lconst;
    }
};

// Non-centred hierarchical normal with group sufficient statistics:
// theta = (mu, log tau, eta_1..eta_G), b_g = mu + tau eta_g.
template <int DM>
struct HierM {
    // shared memory: (ybar_g, n_g / sigma^2) pairs for the gradient (one 8-byte
    // load per group), then n_g and the within-group sums of squares
    static size_t smem_bytes(const DevModel& m) { return (size_t)4 * m.n * sizeof(float); }
    __device__ static void load(const DevModel& m, float* sm) {
        const float inv_s2 = (float)(1.0 / (m.h0 * m.h0));
        for (int i = threadIdx.x; i < m.n; i += blockDim.x) {
            sm[2 * i] = m.gmean[i];
            sm[2 * i + 1] = m.gn[i] * inv_s2;
            sm[2 * m.n + i] = m.gn[i];
            sm[3 * m.n + i] = m.gss[i];
        }
    }
    __device__ static void grad(const DevModel& m, const float* sm, const float (&th)[DM], float (&g)[DM]) {
        const float2* st = reinterpret_cast<const float2*>(sm);
        const float mu = th[0], logtau = th[1], tau = expf(logtau);
        float dmu = 0.0f, dlt = 0.0f;
#pragma unroll
        for (int d = 2; d < DM; ++d) {
            float gd = 0.0f;
            if (d < m.D) {
                const float2 yn = st[d - 2];               // ybar_g, n_g / sigma^2
                const float eta = th[d];
                const float r = yn.y * (yn.x - fmaf(tau, eta, mu));
                dmu += r;
                dlt = fmaf(r * tau, eta, dlt);
                gd = fmaf(r, tau, -eta);
            }
            g[d] = gd;
        }
        g[0] = dmu - mu;
        g[1] = dlt - logtau;
    }
    // FP32 terms per group, FP64 accumulation (as the GEMM-shaped models'
    // end points): FP64 runs at a small fraction of the FP32 rate here
    __device__ static double logpi(const DevModel& m, const float* sm, const float (&th)[DM], const float (&)[DM]) {
        const float inv_2s2 = (float)(0.5 / (m.h0 * m.h0));
        const float mu = th[0], logtau = th[1], tau = expf(logtau);
        double s = -0.5 * (double)mu * (double)mu - 0.5 * (double)logtau * (double)logtau;
#pragma unroll
        for (int d = 2; d < DM; ++d) {
            if (d < m.D) {
                const int k = d - 2;
                const float eta = th[d];
                const float dev = sm[2 * k] - fmaf(tau, eta, mu);
                const float term = -fmaf(sm[2 * m.n + k] * dev, dev, sm[3 * m.n + k]) * inv_2s2 - 0.5f * eta * eta;
                s += (double)term;
            }
        }
        return s + m.lconst;
    }
};

// The move of the particle in slot t (Algorithm 1 for its S_j steps, the
// end-point energy and Delta H), the model's data already in shared memory.
template <template <int> class MT, int DM>
__device__ __forceinline__ void particle_move(const DevModel& m, const TrajArgs& a, const float* sm, int64_t t) {
    using M = MT<DM>;
    const int64_t j = a.perm ? a.perm[t] : t;
    const int64_t src = a.src ? a.src[j] : j;
    const int D = m.D;
    int r;
    double eps;
    uint64_t seed;
    uint32_t kk, jl;
    particle_run(a, j, r, eps, seed, kk, jl);

    float th[DM], g[DM], p[DM];
#pragma unroll
    for (int d = 0; d < DM; ++d) th[d] = d < D ? a.theta_in[(int64_t)d * a.ld + src] : 0.0f;

    if (a.eval_only) {
        M::grad(m, sm, th, g);
        double lp = M::logpi(m, sm, th, g);
#pragma unroll
        for (int d = 0; d < DM; ++d)
            if (d < D) a.grad_out[(int64_t)d * a.ld + j] = g[d];
        a.logpi_out[j] = lp;
        return;   // from the particle's move
    }

#pragma unroll
    for (int d = 0; d < DM; ++d) g[d] = d < D ? a.grad_in[(int64_t)d * a.ld + src] : 0.0f;
    const double lp0 = a.logpi_in[src];
    if (a.p_in) {
#pragma unroll
        for (int d = 0; d < DM; ++d) p[d] = d < D ? a.p_in[(int64_t)d * a.ld + j] : 0.0f;
    } else {
#pragma unroll
        for (int d = 0; d < DM; d += 2) {
            float z0 = 0.0f, z1 = 0.0f;
            if (d < D) normal_pair_f32(seed, (uint32_t)(d >> 1), jl, kk, TAG_MOM, z0, z1);
            p[d] = d < D ? z0 : 0.0f;
            if (d + 1 < DM) p[d + 1] = d + 1 < D ? z1 : 0.0f;
        }
    }
    double kin0 = 0.0;
#pragma unroll
    for (int d = 0; d < DM; ++d) kin0 += (double)p[d] * (double)p[d];
    const double H0 = 0.5 * kin0 - lp0;

    const int S = a.steps[j];
    const float ef = (float)eps, he = (float)(0.5 * eps);
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int d = 0; d < DM; ++d) p[d] = fmaf(he, g[d], p[d]);
#pragma unroll
        for (int d = 0; d < DM; ++d) th[d] = fmaf(ef, p[d], th[d]);
        M::grad(m, sm, th, g);
#pragma unroll
        for (int d = 0; d < DM; ++d) p[d] = fmaf(he, g[d], p[d]);
    }
    const double lp1 = M::logpi(m, sm, th, g);
    double kin1 = 0.0;
#pragma unroll
    for (int d = 0; d < DM; ++d) kin1 += (double)p[d] * (double)p[d];
    double dH = (0.5 * kin1 - lp1) - H0;
    if (!isfinite(dH)) dH = CUDART_INF;
#pragma unroll
    for (int d = 0; d < DM; ++d) {
        if (d < D) {
            a.theta_out[(int64_t)d * a.ld + j] = th[d];
            a.grad_out[(int64_t)d * a.ld + j] = g[d];
            if (a.p_out) a.p_out[(int64_t)d * a.ld + j] = p[d];
        }
    }
    a.logpi_out[j] = lp1;
    if (a.dH) a.dH[j] = dH;
    if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
}

// One particle per thread, one CTA per NT slots.
template <template <int> class MT, int DM, int NT = 128, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) traj_thread_kernel(DevModel m, TrajArgs a) {
    extern __shared__ __align__(16) float sm[];
    MT<DM>::load(m, sm);
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.N) particle_move<MT, DM>(m, a, sm, t);
}

// Persistent form: as many CTAs as fit on the GPU at once, each loading the
// model's data once and then taking tiles of NT slots from a device counter
// (zeroed by the launcher) in slot order, i.e. longest trajectories first.
// Every particle's arithmetic is that of traj_thread_kernel.
template <template <int> class MT, int DM, int NT = 128, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) traj_thread_persist_kernel(DevModel m, TrajArgs a, int64_t ntiles) {
    extern __shared__ __align__(16) float sm[];
    __shared__ unsigned int tile_s;
    MT<DM>::load(m, sm);
    for (;;) {
        if (threadIdx.x == 0) tile_s = atomicAdd(a.work, 1u);
        __syncthreads();
        const int64_t tile = tile_s;
        __syncthreads();   // every thread has the tile before the next one is taken
        if (tile >= ntiles) break;
        const int64_t t = tile * NT + threadIdx.x;
        if (t < a.N) particle_move<MT, DM>(m, a, sm, t);
    }
}


namespace {

template <template <int> class MT, int DM, int NT, int MINB>
cudaError_t launch_thread_v(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const size_t sm = MT<DM>::smem_bytes(m);
    auto kern = traj_thread_kernel<MT, DM, NT, MINB>;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    const int64_t grid = (a.N + NT - 1) / NT;
    if (grid == 0) return cudaSuccess;
    kern<<<(unsigned)grid, NT, sm, s>>>(m, a);
    return cudaGetLastError();
}

template <template <int> class MT, int DM, int NT, int MINB>
cudaError_t launch_thread_persist(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const size_t sm = MT<DM>::smem_bytes(m);
    auto kern = traj_thread_persist_kernel<MT, DM, NT, MINB>;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    const int64_t ntiles = (a.N + NT - 1) / NT;
    if (ntiles == 0) return cudaSuccess;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
    e = cudaMemsetAsync(a.work, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, NT, sm, s>>>(m, a, ntiles);
    return cudaGetLastError();
}

// Variants of the thread-per-particle kernel for the autotuner: CTA size
// (the granularity with which length-sorted slots are dealt to the SMs), a
// register cap that trades spills for a third resident CTA, and for each of
// these the persistent form (4-7: tiles from a device counter; they need
// TrajArgs::work, else the launch falls back to the one-shot form).  Same
// code, same arithmetic.  Small particles (DM < 16) have only the default.
constexpr int32_t THREAD_TILES = 8;
template <template <int> class MT, int DM>
cudaError_t launch_thread(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    if constexpr (DM >= 16) {
        const int v = (a.tile >= 4 && !a.work) ? a.tile - 4 : a.tile;
        switch (v) {
            case 1: return launch_thread_v<MT, DM, 64, 1>(m, a, s);
            case 2: return launch_thread_v<MT, DM, 256, 1>(m, a, s);
            case 3: return launch_thread_v<MT, DM, 128, 3>(m, a, s);
            case 4: return launch_thread_persist<MT, DM, 128, 1>(m, a, s);
            case 5: return launch_thread_persist<MT, DM, 64, 1>(m, a, s);
            case 6: return launch_thread_persist<MT, DM, 256, 1>(m, a, s);
            case 7: return launch_thread_persist<MT, DM, 128, 3>(m, a, s);
            default: break;
        }
    }
    return launch_thread_v<MT, DM, 128, 1>(m, a, s);
}

template <template <int> class MT>
cudaError_t dispatch_thread(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const int D = m.D;
    if (D <= 2) return launch_thread<MT, 2>(m, a, s);
    if (D <= 4) return launch_thread<MT, 4>(m, a, s);
    if (D <= 8) return launch_thread<MT, 8>(m, a, s);
    if (D <= 12) return launch_thread<MT, 12>(m, a, s);
    if (D <= 16) return launch_thread<MT, 16>(m, a, s);
    if (D <= 32) return launch_thread<MT, 32>(m, a, s);
    return cudaErrorInvalidValue;
}

template <template <int> class MT>
cudaError_t dispatch_thread_wide(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const int D = m.D;
    if (D <= 32) return dispatch_thread<MT>(m, a, s);
    if (D <= 52) return launch_thread<MT, 52>(m, a, s);
    if (D <= 64) return launch_thread<MT, 64>(m, a, s);
    return cudaErrorInvalidValue;
}

}  // namespace

int32_t traj_thread_tiles(const DevModel& m) { return m.D > 12 ? THREAD_TILES : 1; }

cudaError_t launch_traj_thread(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    switch (m.kind) {
        case GAUSS_DENSE: return m.D <= 32 ? dispatch_thread<GaussDenseM>(m, a, s) : cudaErrorInvalidValue;
        case BANANA: return dispatch_thread_wide<BananaM>(m, a, s);
        case HIER_NORMAL: return dispatch_thread_wide<HierM>(m, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace smc
