// traj_tc_stream.cu -- tensor-core (tcgen05) leapfrog trajectories for
// GEMM-shaped likelihoods whose data do not fit on chip (Bayesian logistic or
// linear-Gaussian regression with many observations).  Per leapfrog step
// (Algorithm 1) the gradient X'r(X theta) of a tile of 128 particles is
//
//   GEMM1  eta^T [128 x 64 obs] = Theta^T [128 x dk] . X_c^T      (per chunk c)
//   GEMM2  G^T   [128 x dk]    += R_c^T [128 x 64 obs] . X_c      (accumulated)
//
// over chunks of 64 observations; eta is never stored beyond one chunk.  The
// chunks stream through a ring of shared-memory stages filled by the TMA unit
// from per-chunk images that already hold the swizzled K-major operand
// layouts (one contiguous bulk copy per operand), so X, resident in L2 when
// it fits, is read once per tile and step.
//
// Roles (320 threads): warp 8 lane 0 issues the bulk copies; warp 9 lane 0
// issues the MMAs (GEMM1 of chunk c before GEMM2 of chunk c-1, so the tensor
// core works while the residuals of the previous chunk are formed); warps 0-7
// form the residuals r = y - sigmoid(eta) (or (y - eta)/sigma^2) from TMEM
// and hold the particle state: warp w owns TMEM lanes 32 (w % 4) .. + 31
// (one particle per lane) and dimensions 64 (w / 4) .. + 63.  Every wait on
// an mbarrier is bounded (then *dev_err is set and the kernel still runs to
// its end).
//
// Precision: X is rounded once to BF16 (a fixed perturbation of the data the
// integrator sees); with np = 2 the state operands Theta and r are split into
// BF16 hi + lo parts (two products per GEMM), with np = 1 they are BF16.
// Accumulation is FP32 in TMEM.  The end-point energy that enters the
// importance weight is recomputed with the FP32 data and FP64 accumulation,
// so the reduced-precision gradient changes the integrator only: leapfrog with
// any fixed gradient map stays volume preserving and reversible.
#include <cuda_bf16.h>
#include <math_constants.h>
#include "tc_ptx.cuh"
#include "traj.cuh"

namespace smc {
namespace {

constexpr int SP = 128;                       // particles per CTA (MMA M)
constexpr int SC = STREAM_CHUNK;              // observations per chunk
constexpr int S_EPI_WARPS = 8;
constexpr int S_THREADS = 32 * (S_EPI_WARPS + 2);
constexpr int S_PRODUCER_WARP = 8, S_MMA_WARP = 9;
constexpr int TH_ATOM = SP * 128;             // 128 particle rows x 64 BF16 (one 128-byte swizzle atom)
constexpr int R_PART = SP * 128;              // R^T part: 128 particle rows x 64 obs
constexpr int XK_BYTES = 2 * SC * 128;        // X chunk, K-major over dims: 2 atoms of 64 obs rows
constexpr uint32_t S_TMEM_COLS = 256;
constexpr uint32_t S_COL_ETA = 0;             // two eta buffers of 64 columns
constexpr uint32_t S_COL_G = 128;             // gradient accumulator, dk columns
constexpr int S_SMEM_MAX = 232448;            // opt-in shared memory per CTA

struct SLayout {
    int dkr, stages, xt_bytes, stage_bytes;
    int off_th, off_r, off_stage, off_y, off_misc, off_bar, total;
};

// Byte layout of the dynamic shared memory (from a 1024-aligned base).
__host__ __device__ inline SLayout s_layout(int dk, int np, int stages) {
    SLayout L;
    L.dkr = dk;                                   // dk is a multiple of 16: whole 8-row swizzle groups
    L.stages = stages;
    L.xt_bytes = L.dkr * 128;
    L.stage_bytes = XK_BYTES + L.xt_bytes;        // multiple of 1024
    L.off_th = 0;                                 // [np][2 atoms]
    L.off_r = L.off_th + np * 2 * TH_ATOM;        // [2 buffers][np]
    L.off_stage = L.off_r + 2 * np * R_PART;      // [stages]
    L.off_y = L.off_stage + stages * L.stage_bytes;   // [stages][64] f32
    L.off_misc = L.off_y + stages * SC * 4;       // kin, sq, ll: [2][128] f64 each
    L.off_bar = L.off_misc + 6 * SP * 8;          // mbarriers, TMEM base, step maximum
    L.total = L.off_bar + 256 + 1024;             // + alignment slack of the base
    return L;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float bf16_round(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

// 8 consecutive values -> one 16-byte unit of a BF16 row (hi), and the
// residual unit (lo) when split.
__device__ __forceinline__ void pack_unit(const float* v, uint4& hi, uint4& lo) {
    float h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        h[e] = bf16_round(v[e]);
        l[e] = v[e] - h[e];
    }
    hi = make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
    lo = make_uint4(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]), pack_bf16(l[4], l[5]), pack_bf16(l[6], l[7]));
}

template <bool LOGIT>
__device__ __forceinline__ float residual(float y, float eta, float inv_s2) {
    if (LOGIT) return y - 1.0f / (1.0f + __expf(-eta));
    return (y - eta) * inv_s2;
}

template <bool LOGIT, int NP>
__global__ void __launch_bounds__(S_THREADS, 1) traj_stream_kernel(DevModel m, TrajArgs a, int stages) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const SLayout L = s_layout(m.dk, NP, stages);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int D = m.D, dk = m.dk, nch = m.n_chunks;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.off_bar);   // [4] stage filled
    uint64_t* empty = full + 4;                                      // [4] stage consumed by both GEMMs
    uint64_t* eta_full = empty + 4;                                  // [2] GEMM1 done
    uint64_t* eta_empty = eta_full + 2;                              // [2] eta read by the epilogue
    uint64_t* r_full = eta_empty + 2;                                // [2] R^T written
    uint64_t* r_empty = r_full + 2;                                  // [2] GEMM2 done with R^T
    uint64_t* g_full = r_empty + 2;                                  // step's gradient complete
    uint64_t* th_full = g_full + 1;                                  // next step's Theta^T written
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(th_full + 1);
    int* smax_s = reinterpret_cast<int*>(tmem_s + 1);
    double* kin_s = reinterpret_cast<double*>(sm + L.off_misc);      // [2][128] |p|^2 halves
    double* sq_s = kin_s + 2 * SP;                                   // [2][128] |theta|^2 halves
    double* ll_s = sq_s + 2 * SP;                                    // [2][128] log-likelihood halves
    float* y_s = reinterpret_cast<float*>(sm + L.off_y);
    const uint32_t s_base = tc::smem_u32(sm);
    int* err = a.dev_err;

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&eta_full[i], 1);
            tc::mbar_init(&eta_empty[i], S_EPI_WARPS);
            tc::mbar_init(&r_full[i], S_EPI_WARPS);
            tc::mbar_init(&r_empty[i], 1);
        }
        tc::mbar_init(g_full, 1);
        tc::mbar_init(th_full, S_EPI_WARPS);
        tc::fence_mbar_init();
        *smax_s = 0;
    }
    if (wid == 0) {
        tc::tmem_alloc(tmem_s, S_TMEM_COLS);
        tc::tmem_relinquish();
    }

    // ---------------------------------------------------------------- particle state (warps 0-7)
    const bool epi = wid < S_EPI_WARPS;
    const int quarter = wid & 3, dh = (wid >> 2) & 1;
    const int prow = 32 * quarter + lane;
    const int d0 = 64 * dh;                          // first dimension of this thread
    const float inv_tau2 = LOGIT ? (float)(1.0 / (m.h0 * m.h0)) : (float)(1.0 / (m.h1 * m.h1));
    const double inv_tau2_d = LOGIT ? 1.0 / (m.h0 * m.h0) : 1.0 / (m.h1 * m.h1);
    const float inv_s2 = LOGIT ? 0.0f : (float)(1.0 / (m.h0 * m.h0));
    const float inv_s = LOGIT ? 0.0f : (float)(1.0 / m.h0);
    // theta lives in registers; the momenta live in a.p_out during the
    // trajectory (read and written once per step), which keeps the epilogue
    // within the register budget of 320 threads
    float th[64];
    int64_t j = -1, src = -1;
    int S = 0;
    float ef = 0.0f;
    {
        const int64_t t = (int64_t)blockIdx.x * SP + prow;
        if (epi && t < a.N) {
            j = a.perm ? a.perm[t] : t;
            src = a.src ? a.src[j] : j;
            S = a.eval_only ? 0 : a.steps[j];
            int r;
            double eps;
            uint64_t seed;
            uint32_t kk, jl;
            particle_run(a, j, r, eps, seed, kk, jl);
            ef = (float)eps;
            double kin = 0.0;
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                const int d = d0 + i;
                th[i] = d < D ? a.theta_in[(int64_t)d * a.ld + src] : 0.0f;
            }
            if (!a.eval_only) {
                const float hf = 0.5f * ef;
                // momentum (given, or Philox + Box-Muller), first half kick and drift
#pragma unroll
                for (int i = 0; i < 64; i += 2) {
                    const int d = d0 + i;
                    if (d < D) {
                        float pv[2];
                        if (a.p_in) {
                            pv[0] = a.p_in[(int64_t)d * a.ld + j];
                            pv[1] = d + 1 < D ? a.p_in[(int64_t)(d + 1) * a.ld + j] : 0.0f;
                        } else {
                            double z0, z1;
                            normal_pair(seed, (uint32_t)(d >> 1), jl, kk, TAG_MOM, z0, z1);
                            pv[0] = (float)z0;
                            pv[1] = d + 1 < D ? (float)z1 : 0.0f;
                        }
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            if (d + e < D) {
                                kin += (double)pv[e] * (double)pv[e];
                                if (S >= 1) {
                                    const float g0 = a.grad_in[(int64_t)(d + e) * a.ld + src];
                                    pv[e] = fmaf(hf, g0, pv[e]);
                                    th[i + e] = fmaf(ef, pv[e], th[i + e]);
                                }
                                a.p_out[(int64_t)(d + e) * a.ld + j] = pv[e];
                            }
                        }
                    }
                }
            }
            kin_s[dh * SP + prow] = kin;
        } else {
#pragma unroll
            for (int i = 0; i < 64; ++i) th[i] = 0.0f;
            if (epi) kin_s[dh * SP + prow] = 0.0;
        }
    }
    __syncthreads();
    if (epi && S > 0) atomicMax(smax_s, S);
    // Theta^T operand rows of this thread's atom (dims d0 .. d0 + 63)
    auto write_theta = [&]() {
        unsigned char* hi = sm + L.off_th + dh * TH_ATOM + prow * 128;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            uint4 vh, vl;
            pack_unit(th + 8 * u, vh, vl);
            const int phys = (u ^ (prow & 7)) << 4;
            *reinterpret_cast<uint4*>(hi + phys) = vh;
            if (NP == 2) *reinterpret_cast<uint4*>(hi + 2 * TH_ATOM + phys) = vl;
        }
    };
    if (epi) write_theta();
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_s;
    const int smax = *smax_s;
    const int nsteps = a.eval_only ? 1 : smax;
    double H0 = 0.0;
    if (epi && dh == 0 && j >= 0 && !a.eval_only) H0 = 0.5 * (kin_s[prow] + kin_s[SP + prow]) - a.logpi_in[src];

    const uint32_t IDESC1 = tc::idesc_bf16_f32(SP, SC);
    const uint32_t IDESC2 = tc::idesc_bf16_f32(SP, (uint32_t)dk);
    const int ksteps1 = dk / 16;
    const int64_t total = (int64_t)nsteps * nch;

    if (wid == S_PRODUCER_WARP) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)(XK_BYTES + L.xt_bytes + SC * 4);
            for (int64_t it = 0; it < total; ++it) {
                const int c = (int)(it % nch);
                const int st = (int)(it % stages);
                const uint32_t ph = (uint32_t)((it / stages) & 1);
                tc::mbar_wait(&empty[st], ph ^ 1u, err);
                tc::mbar_arrive_expect_tx(&full[st], bytes);
                unsigned char* dst = sm + L.off_stage + st * L.stage_bytes;
                tc::bulk_g2s(dst, m.xk_img + (int64_t)c * (XK_BYTES / 2), XK_BYTES, &full[st]);
                tc::bulk_g2s(dst + XK_BYTES, m.xt_img + (int64_t)c * (L.xt_bytes / 2), (uint32_t)L.xt_bytes,
                             &full[st]);
                tc::bulk_g2s(y_s + st * SC, m.y_img + (int64_t)c * SC, SC * 4, &full[st]);
            }
            // every copy has landed before the stage memory is reused or the CTA exits
            for (int64_t it = total > stages ? total - stages : 0; it < total; ++it)
                tc::mbar_wait(&full[it % stages], (uint32_t)((it / stages) & 1), err);
        }
    } else if (wid == S_MMA_WARP) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            auto gemm2 = [&](int64_t i) {
                const int st = (int)(i % stages), b = (int)(i & 1);
                const int ci = (int)(i % nch);
                tc::mbar_wait(&r_full[b], (uint32_t)((i >> 1) & 1), err);
                tc::fence_after_sync();
                const uint32_t xt = s_base + L.off_stage + st * L.stage_bytes + XK_BYTES;
                for (int q = 0; q < NP; ++q)
                    for (int kk = 0; kk < SC / 16; ++kk) {
                        const uint64_t ad = tc::smem_desc(s_base + L.off_r + (b * NP + q) * R_PART + kk * 32, 16, 1024,
                                                          tc::SWZ_128B);
                        const uint64_t bd = tc::smem_desc(xt + kk * 32, 16, 1024, tc::SWZ_128B);
                        tc::mma_bf16(tmem + S_COL_G, ad, bd, IDESC2, (ci > 0 || q > 0 || kk > 0) ? 1u : 0u);
                    }
                tc::mma_commit(&r_empty[b]);
                tc::mma_commit(&empty[st]);
            };
            for (int s = 1; s <= nsteps; ++s) {
                if (s >= 2) tc::mbar_wait(th_full, (uint32_t)((s - 2) & 1), err);
                tc::fence_after_sync();
                for (int c = 0; c < nch; ++c) {
                    const int64_t it = (int64_t)(s - 1) * nch + c;
                    const int st = (int)(it % stages), b = (int)(it & 1);
                    tc::mbar_wait(&full[st], (uint32_t)((it / stages) & 1), err);
                    tc::mbar_wait(&eta_empty[b], (uint32_t)(((it >> 1) & 1) ^ 1), err);
                    tc::fence_after_sync();
                    const uint32_t xk = s_base + L.off_stage + st * L.stage_bytes;
                    for (int q = 0; q < NP; ++q)
                        for (int kk = 0; kk < ksteps1; ++kk) {
                            const int atom = kk >> 2, ko = (kk & 3) * 32;
                            const uint64_t ad = tc::smem_desc(s_base + L.off_th + (q * 2 + atom) * TH_ATOM + ko, 16,
                                                              1024, tc::SWZ_128B);
                            const uint64_t bd = tc::smem_desc(xk + atom * (SC * 128) + ko, 16, 1024, tc::SWZ_128B);
                            tc::mma_bf16(tmem + S_COL_ETA + b * SC, ad, bd, IDESC1, (q > 0 || kk > 0) ? 1u : 0u);
                        }
                    tc::mma_commit(&eta_full[b]);
                    if (c > 0) gemm2(it - 1);
                }
                gemm2((int64_t)s * nch - 1);
                tc::mma_commit(g_full);
            }
        }
    } else {
        // ------------------------------------------------------------ residuals and state (warps 0-7)
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        const float hf = 0.5f * ef;
        for (int s = 1; s <= nsteps; ++s) {
            for (int c = 0; c < nch; ++c) {
                const int64_t it = (int64_t)(s - 1) * nch + c;
                const int st = (int)(it % stages), b = (int)(it & 1);
                const uint32_t ph = (uint32_t)((it >> 1) & 1);
                tc::mbar_wait(&eta_full[b], ph, err);
                tc::fence_after_sync();
                float eta[32];
                tc::tmem_ld32(tmem + lane_base + S_COL_ETA + b * SC + 32 * dh, eta);
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&eta_empty[b]);
                // the stage's y was written by the bulk copy: acquire its barrier
                // phase (still current: the stage is refilled only after this
                // chunk's GEMM2, which waits for these residuals)
                tc::mbar_wait(&full[st], (uint32_t)((it / stages) & 1), err);
                const float* yv = y_s + st * SC + 32 * dh;
                float* r = eta;   // residuals overwrite eta in place
#pragma unroll
                for (int e = 0; e < 32; ++e) r[e] = residual<LOGIT>(yv[e], eta[e], inv_s2);
                tc::mbar_wait(&r_empty[b], ph ^ 1u, err);
                unsigned char* row = sm + L.off_r + b * NP * R_PART + prow * 128;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    uint4 vh, vl;
                    pack_unit(r + 8 * u, vh, vl);
                    const int phys = ((4 * dh + u) ^ (prow & 7)) << 4;
                    *reinterpret_cast<uint4*>(row + phys) = vh;
                    if (NP == 2) *reinterpret_cast<uint4*>(row + R_PART + phys) = vl;
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&r_full[b]);
            }
            // the step's gradient: G - theta / tau^2, then the leapfrog update
            tc::mbar_wait(g_full, (uint32_t)((s - 1) & 1), err);
            tc::fence_after_sync();
            const bool live = j >= 0 && (a.eval_only || s <= S);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float gv[32];
                tc::tmem_ld32(tmem + lane_base + S_COL_G + d0 + 32 * h, gv);
                if (live) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const int i = 32 * h + e, d = d0 + i;
                        if (d < D) {
                            const float g = gv[e] - th[i] * inv_tau2;
                            if (a.eval_only || s == S) a.grad_out[(int64_t)d * a.ld + j] = g;
                            if (!a.eval_only) {
                                float* pp = a.p_out + (int64_t)d * a.ld + j;
                                float pv = fmaf(hf, g, *pp);
                                if (s + 1 <= S) {
                                    pv = fmaf(hf, g, pv);
                                    th[i] = fmaf(ef, pv, th[i]);
                                }
                                *pp = pv;
                            }
                        }
                    }
                }
            }
            if (s < nsteps) {
                write_theta();
                tc::fence_proxy_async_smem();
            }
            tc::fence_before_sync();
            __syncwarp();
            if (s < nsteps && lane == 0) tc::mbar_arrive(th_full);
        }
    }

    // ---------------------------------------------------------------- end point energy
    // theta^T in FP32 over the drained stage ring, FP32 eta from the FP32 data,
    // FP64 accumulation of the log-likelihood
    __syncthreads();
    float* thT = reinterpret_cast<float*>(sm + L.off_stage);   // [dk][128]
    if (epi) {
        double sq = 0.0, kin = 0.0;
#pragma unroll
        for (int i = 0; i < 64; ++i) {
            const int d = d0 + i;
            if (d < dk) thT[d * SP + prow] = th[i];
            sq += (double)th[i] * (double)th[i];
            if (j >= 0 && d < D && !a.eval_only) {
                const double pv = a.p_out[(int64_t)d * a.ld + j];
                kin += pv * pv;
            }
        }
        sq_s[dh * SP + prow] = sq;
        kin_s[dh * SP + prow] = kin;     // the initial halves were consumed by H0
    }
    __syncthreads();
    {
        const int pp = tid & (SP - 1), half = tid >> 7;   // threads 256 .. 319 idle
        if (half < 2) {
            double ll = 0.0;
            for (int i = half; i < m.n; i += 2) {
                const float* x = m.X + (int64_t)i * m.Dp;
                float e0 = 0.0f, e1 = 0.0f;
                int d = 0;
                for (; d + 1 < D; d += 2) {
                    e0 = fmaf(__ldg(x + d), thT[d * SP + pp], e0);
                    e1 = fmaf(__ldg(x + d + 1), thT[(d + 1) * SP + pp], e1);
                }
                if (d < D) e0 = fmaf(__ldg(x + d), thT[d * SP + pp], e0);
                const float eta = e0 + e1, yv = __ldg(m.y + i);
                float term;
                if (LOGIT) {
                    const float sp = eta > 0.0f ? eta + log1pf(expf(-eta)) : log1pf(expf(eta));
                    term = yv * eta - sp;
                } else {
                    const float z = (yv - eta) * inv_s;
                    term = -0.5f * z * z;
                }
                ll += (double)term;
            }
            ll_s[half * SP + pp] = ll;
        }
    }
    __syncthreads();
    if (epi && j >= 0) {
#pragma unroll
        for (int i = 0; i < 64; ++i) {
            const int d = d0 + i;
            if (d < D && !a.eval_only) a.theta_out[(int64_t)d * a.ld + j] = th[i];
        }
        if (dh == 0) {
            const double sq = sq_s[prow] + sq_s[SP + prow];
            const double lp1 = ll_s[prow] + ll_s[SP + prow] - 0.5 * sq * inv_tau2_d + m.lconst;
            a.logpi_out[j] = lp1;
            if (!a.eval_only) {
                const double kin = kin_s[prow] + kin_s[SP + prow];
                double dH = (0.5 * kin - lp1) - H0;
                if (!isfinite(dH)) dH = CUDART_INF;
                if (a.dH) a.dH[j] = dH;
                if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (wid == 0) tc::tmem_dealloc(tmem, S_TMEM_COLS);
}

template <bool LOGIT, int NP>
cudaError_t launch_stream(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const int tiles = (int)((a.N + SP - 1) / SP);
    if (tiles == 0) return cudaSuccess;
    int stages = 4;
    while (stages > 2 && s_layout(m.dk, NP, stages).total > S_SMEM_MAX) --stages;
    const int bytes = s_layout(m.dk, NP, stages).total;
    if (bytes > S_SMEM_MAX) return cudaErrorInvalidValue;
    auto kern = traj_stream_kernel<LOGIT, NP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)tiles, S_THREADS, (size_t)bytes, s>>>(m, a, stages);
    return cudaGetLastError();
}

}  // namespace

bool traj_stream_supported(const DevModel& m) {
    return (m.kind == LOGISTIC || m.kind == LINEAR_GAUSS) && m.D >= 1 && m.D <= 128 && m.xk_img && m.xt_img &&
           m.y_img && m.n_chunks >= 1;
}

cudaError_t launch_traj_stream(const DevModel& m, const TrajArgs& a, int np, cudaStream_t s) {
    if (!traj_stream_supported(m) || (np != 1 && np != 2)) return cudaErrorInvalidValue;
    if (!a.eval_only && !a.p_out) return cudaErrorInvalidValue;   // the momenta live in p_out
    const bool logit = m.kind == LOGISTIC;
    if (logit) return np == 2 ? launch_stream<true, 2>(m, a, s) : launch_stream<true, 1>(m, a, s);
    return np == 2 ? launch_stream<false, 2>(m, a, s) : launch_stream<false, 1>(m, a, s);
}

}  // namespace smc
