// traj_glm_stream.cu -- FP32 SIMT leapfrog trajectories (Algorithm 1) for
// Bayesian logistic / linear-Gaussian regression whose data do not fit in
// shared memory: the plain FP32 counterpart of the streamed tensor-core
// kernel.  Per leapfrog step the gradient X'(y - sigmoid(X theta)) - theta/tau^2
// of 64 particles is accumulated over chunks of 64 observations that stream
// through a double-buffered shared-memory ring (cp.async).
//
// Thread layout: 256 threads; lanes 4k .. 4k + 3 of warp w hold particle
// 8w + k, each lane a quarter of the dimensions (HQ of them, zero padded), so
// one observation costs a quarter dot product per lane, two shuffles, one
// residual and a quarter gradient update, and the gradient of a particle needs
// no cross-warp reduction.  Positions stay in registers; momenta live in
// a.p_out during the trajectory.  The end-point log pi (the importance
// weight's energy) is an FP32 product with FP64 accumulation, as in every
// trajectory kernel of the library.
#include <math_constants.h>
#include "tc_ptx.cuh"
#include "traj.cuh"

namespace smc {
namespace {

constexpr int GS_P = 64;           // particles per CTA
constexpr int GS_T = 256;          // threads per CTA
constexpr int GS_C = 64;           // observations per chunk

template <bool LOGIT>
__device__ __forceinline__ float gs_resid(float y, float eta, float inv_s2) {
    if (LOGIT) return y - __fdividef(1.0f, 1.0f + __expf(-eta));
    return (y - eta) * inv_s2;
}

template <bool LOGIT>
__device__ __forceinline__ float gs_term(float y, float eta, float inv_s) {
    if (LOGIT) {
        const float sp = eta > 0.0f ? eta + log1pf(expf(-eta)) : log1pf(expf(eta));
        return y * eta - sp;
    }
    const float z = (y - eta) * inv_s;
    return -0.5f * z * z;
}

template <bool LOGIT, int HQ>
__global__ void __launch_bounds__(GS_T, 2) traj_glm_stream_kernel(DevModel m, TrajArgs a) {
    constexpr int XS = 4 * HQ;                        // shared row stride (floats)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* xs = reinterpret_cast<float*>(smem_raw);   // [2][GS_C][XS]
    __shared__ int smax_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int qq = lane & 3;                          // quarter of the dimensions
    const int pq = wid * 8 + (lane >> 2);             // particle within the CTA
    const int D = m.D, Dp = m.Dp, n = m.n;
    const int nch = (n + GS_C - 1) / GS_C;
    const int d0 = qq * HQ;
    const float inv_tau2 = LOGIT ? (float)(1.0 / (m.h0 * m.h0)) : (float)(1.0 / (m.h1 * m.h1));
    const double inv_tau2_d = LOGIT ? 1.0 / (m.h0 * m.h0) : 1.0 / (m.h1 * m.h1);
    const float inv_s2 = LOGIT ? 0.0f : (float)(1.0 / (m.h0 * m.h0));
    const float inv_s = LOGIT ? 0.0f : (float)(1.0 / m.h0);

    // padding columns [Dp, XS) of both buffers are zero and never copied over
    for (int e = tid; e < 2 * GS_C * XS; e += GS_T)
        if (e % XS >= Dp) xs[e] = 0.0f;
    if (tid == 0) smax_s = 0;

    // ---- particle state
    int64_t j = -1, src = -1;
    int S = 0;
    float ef = 0.0f;
    const int64_t t = (int64_t)blockIdx.x * GS_P + pq;
    uint64_t seed = 0;
    uint32_t kk = 0, jl = 0;
    if (t < a.N) {
        j = a.perm ? a.perm[t] : t;
        src = a.src ? a.src[j] : j;
        S = a.eval_only ? 0 : a.steps[j];
        int r;
        double eps;
        particle_run(a, j, r, eps, seed, kk, jl);
        ef = (float)eps;
    }
    const float hf = 0.5f * ef;
    float th[HQ];
    double kin = 0.0;
#pragma unroll
    for (int i = 0; i < HQ; i += 2) {
        const int d = d0 + i;
        th[i] = th[i + 1] = 0.0f;
        if (j < 0 || d >= D) continue;
        float pv[2] = {0.0f, 0.0f};
        if (!a.eval_only) {
            if (a.p_in) {
                pv[0] = a.p_in[(int64_t)d * a.ld + j];
                pv[1] = d + 1 < D ? a.p_in[(int64_t)(d + 1) * a.ld + j] : 0.0f;
            } else {
                double z0, z1;
                normal_pair(seed, (uint32_t)(d >> 1), jl, kk, TAG_MOM, z0, z1);
                pv[0] = (float)z0;
                pv[1] = d + 1 < D ? (float)z1 : 0.0f;
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (d + q >= D) continue;
            float tv = a.theta_in[(int64_t)(d + q) * a.ld + src];
            if (!a.eval_only) {
                kin += (double)pv[q] * (double)pv[q];
                if (S >= 1) {   // first half kick and drift from the cached gradient
                    const float g0 = a.grad_in[(int64_t)(d + q) * a.ld + src];
                    pv[q] = fmaf(hf, g0, pv[q]);
                    tv = fmaf(ef, pv[q], tv);
                }
                a.p_out[(int64_t)(d + q) * a.ld + j] = pv[q];
            }
            th[i + q] = tv;
        }
    }
    kin += __shfl_xor_sync(0xffffffffu, kin, 1);
    kin += __shfl_xor_sync(0xffffffffu, kin, 2);
    const double H0 = (j >= 0 && !a.eval_only) ? 0.5 * kin - a.logpi_in[src] : 0.0;
    __syncthreads();
    if (qq == 0 && S > 0) atomicMax(&smax_s, S);
    __syncthreads();
    const int nsteps = a.eval_only ? 1 : smax_s;

    // chunk c of X -> buffer b (cp.async; rows past n are not copied and are
    // skipped by the loops below)
    const int pieces = Dp / 4;
    auto issue = [&](int c, int b) {
        const int row0 = c * GS_C;
        const int rows = min(GS_C, n - row0);
        float* dst = xs + b * GS_C * XS;
        const float* srcx = m.X + (int64_t)row0 * Dp;
        for (int v = tid; v < rows * pieces; v += GS_T) {
            const int r = v / pieces, q = v - r * pieces;
            tc::cp_async16(dst + r * XS + 4 * q, srcx + (int64_t)r * Dp + 4 * q);
        }
        tc::cp_async_commit();
    };

    // ---- leapfrog steps: a flat sequence of (step, chunk) iterations, with
    // the next chunk in flight while the current one is used
    const int64_t total = (int64_t)nsteps * nch;
    float acc[HQ];
#pragma unroll
    for (int i = 0; i < HQ; ++i) acc[i] = 0.0f;
    if (total > 0) issue(0, 0);
    int c = 0, s = 1;
    for (int64_t it = 0; it < total; ++it) {
        const int b = (int)(it & 1);
        if (it + 1 < total) issue(c + 1 < nch ? c + 1 : 0, b ^ 1);
        else tc::cp_async_commit();
        tc::cp_async_wait<1>();
        __syncthreads();
        const float* xb = xs + b * GS_C * XS + d0;
        const int row0 = c * GS_C;
        const int rows = min(GS_C, n - row0);
        for (int o = 0; o < rows; ++o) {
            const float4* xr = reinterpret_cast<const float4*>(xb + o * XS);
            float xv[HQ];
#pragma unroll
            for (int q = 0; q < HQ / 4; ++q) {
                const float4 v = xr[q];
                xv[4 * q] = v.x;
                xv[4 * q + 1] = v.y;
                xv[4 * q + 2] = v.z;
                xv[4 * q + 3] = v.w;
            }
            float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, e3 = 0.0f;
#pragma unroll
            for (int i = 0; i < HQ; i += 4) {
                e0 = fmaf(xv[i], th[i], e0);
                e1 = fmaf(xv[i + 1], th[i + 1], e1);
                e2 = fmaf(xv[i + 2], th[i + 2], e2);
                e3 = fmaf(xv[i + 3], th[i + 3], e3);
            }
            float eta = (e0 + e1) + (e2 + e3);
            eta += __shfl_xor_sync(0xffffffffu, eta, 1);
            eta += __shfl_xor_sync(0xffffffffu, eta, 2);
            const float rr = gs_resid<LOGIT>(__ldg(m.y + row0 + o), eta, inv_s2);
#pragma unroll
            for (int i = 0; i < HQ; ++i) acc[i] = fmaf(rr, xv[i], acc[i]);
        }
        __syncthreads();   // buffer b is refilled by the next iteration's issue
        if (++c == nch) {
            // ---- step end: gradient, closing half kick, opening kick + drift
            c = 0;
            const bool live = j >= 0 && (a.eval_only || s <= S);
#pragma unroll
            for (int i = 0; i < HQ; ++i) {
                const int d = d0 + i;
                if (live && d < D) {
                    const int64_t o = (int64_t)d * a.ld + j;
                    const float g = acc[i] - th[i] * inv_tau2;
                    if (a.eval_only || s == S) a.grad_out[o] = g;
                    if (!a.eval_only) {
                        float pv = fmaf(hf, g, a.p_out[o]);
                        if (s + 1 <= S) {
                            pv = fmaf(hf, g, pv);
                            th[i] = fmaf(ef, pv, th[i]);
                        }
                        a.p_out[o] = pv;
                    }
                }
                acc[i] = 0.0f;
            }
            ++s;
        }
    }

    // ---- end point: log pi in FP64 accumulation (FP32 eta)
    double ll = 0.0;
    issue(0, 0);
    for (int cc = 0; cc < nch; ++cc) {
        const int b = cc & 1;
        if (cc + 1 < nch) issue(cc + 1, b ^ 1);
        else tc::cp_async_commit();
        tc::cp_async_wait<1>();
        __syncthreads();
        const float* xb = xs + b * GS_C * XS + d0;
        const int row0 = cc * GS_C;
        const int rows = min(GS_C, n - row0);
        for (int o = 0; o < rows; ++o) {
            const float4* xr = reinterpret_cast<const float4*>(xb + o * XS);
            float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, e3 = 0.0f;
#pragma unroll
            for (int q = 0; q < HQ / 4; ++q) {
                const float4 v = xr[q];
                e0 = fmaf(v.x, th[4 * q], e0);
                e1 = fmaf(v.y, th[4 * q + 1], e1);
                e2 = fmaf(v.z, th[4 * q + 2], e2);
                e3 = fmaf(v.w, th[4 * q + 3], e3);
            }
            float eta = (e0 + e1) + (e2 + e3);
            eta += __shfl_xor_sync(0xffffffffu, eta, 1);
            eta += __shfl_xor_sync(0xffffffffu, eta, 2);
            if (qq == 0) ll += (double)gs_term<LOGIT>(__ldg(m.y + row0 + o), eta, inv_s);
        }
        __syncthreads();
    }
    double sq = 0.0;
#pragma unroll
    for (int i = 0; i < HQ; ++i) sq += (double)th[i] * (double)th[i];
    sq += __shfl_xor_sync(0xffffffffu, sq, 1);
    sq += __shfl_xor_sync(0xffffffffu, sq, 2);
    double kin1 = 0.0;
    if (j >= 0 && !a.eval_only)
#pragma unroll
        for (int i = 0; i < HQ; ++i) {
            const int d = d0 + i;
            if (d < D) {
                const double pv = a.p_out[(int64_t)d * a.ld + j];
                kin1 += pv * pv;
            }
        }
    kin1 += __shfl_xor_sync(0xffffffffu, kin1, 1);
    kin1 += __shfl_xor_sync(0xffffffffu, kin1, 2);
    if (j < 0) return;
    if (!a.eval_only)
#pragma unroll
        for (int i = 0; i < HQ; ++i) {
            const int d = d0 + i;
            if (d < D) a.theta_out[(int64_t)d * a.ld + j] = th[i];
        }
    if (qq == 0) {
        const double lp1 = ll - 0.5 * sq * inv_tau2_d + m.lconst;
        a.logpi_out[j] = lp1;
        if (!a.eval_only) {
            double dH = (0.5 * kin1 - lp1) - H0;
            if (!isfinite(dH)) dH = CUDART_INF;
            if (a.dH) a.dH[j] = dH;
            if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
        }
    }
}

template <bool LOGIT, int HQ>
cudaError_t launch_gs(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const int64_t grid = (a.N + GS_P - 1) / GS_P;
    if (grid == 0) return cudaSuccess;
    const size_t sm = sizeof(float) * 2 * GS_C * 4 * HQ;
    auto kern = traj_glm_stream_kernel<LOGIT, HQ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, GS_T, sm, s>>>(m, a);
    return cudaGetLastError();
}

template <bool LOGIT>
cudaError_t dispatch_gs(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const int hq = ((m.Dp + 3) / 4 + 3) & ~3;     // quarter width, a multiple of 4
    if (hq <= 8) return launch_gs<LOGIT, 8>(m, a, s);
    if (hq <= 16) return launch_gs<LOGIT, 16>(m, a, s);
    if (hq <= 28) return launch_gs<LOGIT, 28>(m, a, s);
    return launch_gs<LOGIT, 32>(m, a, s);
}

}  // namespace

bool traj_glm_stream_supported(const DevModel& m) {
    return (m.kind == LOGISTIC || m.kind == LINEAR_GAUSS) && m.D >= 1 && m.D <= 128 && m.n >= 1 && m.X;
}

cudaError_t launch_traj_glm_stream(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    if (!traj_glm_stream_supported(m)) return cudaErrorInvalidValue;
    if (!a.eval_only && !a.p_out) return cudaErrorInvalidValue;   // the momenta live in p_out
    return m.kind == LOGISTIC ? dispatch_gs<true>(m, a, s) : dispatch_gs<false>(m, a, s);
}

}  // namespace smc
