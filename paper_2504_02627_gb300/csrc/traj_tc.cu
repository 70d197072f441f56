// traj_tc.cu -- tensor-core (tcgen05) leapfrog trajectories for the
// GEMM-shaped likelihoods: Bayesian logistic regression (Sec. 4, German
// Credit) and linear-Gaussian regression.  Per leapfrog step (Algorithm 1)
// the gradient X'r(X theta) of 128 particles is two dense contractions:
//
//   GEMM1  eta^T [128 particles x obs] = Theta^T [128 x 32] . X^T [32 x obs]
//   GEMM2  G^T   [128 particles x 32]  = R^T [128 x obs] . X [obs x 32]
//
// with r = y - sigmoid(eta) (or (y - eta)/sigma^2) formed in between from
// TMEM.  BF16 operands, FP32 accumulation in TMEM; in the x3 mode every
// operand is split a = a_hi + a_lo (both BF16) and the products
// hi*hi + lo*hi + hi*lo are accumulated (the lo*lo term is dropped).
//
// Layout of the work: a cluster of CS CTAs shares one tile of 128 particles;
// CTA rank r owns observations [r*nloc, (r+1)*nloc) (nloc <= 256) with its
// slice of X resident in shared memory for the whole trajectory, as two
// K-major operand copies (X rows for GEMM1, X^T rows for GEMM2).  The
// per-CTA partial gradients are summed in rank order through distributed
// shared memory once per step, so every CTA of the cluster holds identical
// particle state.  The energy of the trajectory end point (which enters the
// importance weight) is recomputed in FP32 with FP64 accumulation, so the
// reduced-precision gradient only changes the integrator, never the target:
// leapfrog with any fixed gradient map is still volume preserving and
// reversible, and the weight -Delta H uses the exact log pi.
#include <cuda_bf16.h>
#include <math_constants.h>
#include "tc_ptx.cuh"
#include "traj.cuh"

namespace smc {
namespace {

constexpr int TC_P = 128;          // particles per tile (MMA M)
constexpr int TC_DK = 32;          // padded dimension (K of GEMM1, N of GEMM2)
constexpr int TC_NC = 128;         // observations per chunk (N of GEMM1, K of GEMM2)
constexpr int TC_NLOC = 256;       // observations per CTA (two chunks)
constexpr int TC_MAXCH = TC_NLOC / TC_NC;
constexpr int TC_THREADS = 256;    // 8 warps
constexpr int TC_GSTRIDE = 36;     // floats per row of the partial-gradient buffer
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr uint32_t TC_COL_G = 256; // TMEM column of the gradient accumulator

// Shared-memory layout (bytes from a 1024-aligned base).
constexpr int XK_BYTES = TC_NC * 64;            // one chunk of X, K-major SW64 rows: 8 KB
constexpr int XK_PART = TC_NLOC * 64;           // 16 KB
constexpr int XT_ATOM = TC_DK * 128;            // X^T, K-major SW128 atom (32 rows x 64 obs): 4 KB
constexpr int XT_BYTES = 2 * XT_ATOM;           // one chunk of X^T: 8 KB
constexpr int XT_PART = TC_MAXCH * XT_BYTES;    // 16 KB
constexpr int TH_BYTES = TC_P * 64;             // Theta^T, K-major SW64: 8 KB
constexpr int RT_ATOM = TC_P * 128;             // R^T, K-major SW128 atom (128 rows x 64 obs): 16 KB
constexpr int RT_BYTES = 2 * RT_ATOM;           // one chunk of R^T: 32 KB
constexpr int OFF_XK = 0;                                   // [part][256 rows]
constexpr int OFF_XT = OFF_XK + 2 * XK_PART;                // [part][chunk]
constexpr int OFF_TH = OFF_XT + 2 * XT_PART;                // [part]
constexpr int OFF_RT = OFF_TH + 2 * TH_BYTES;               // x3: [part]; BF16: [buffer]
constexpr int OFF_GP = OFF_RT + 2 * RT_BYTES;               // [2][128][36] f32
constexpr int OFF_Y = OFF_GP + 2 * TC_P * TC_GSTRIDE * 4;   // [256] f32
constexpr int OFF_LL = OFF_Y + TC_NLOC * 4;                 // [128] f64
constexpr int OFF_BAR = OFF_LL + TC_P * 8;                  // mbarriers + tmem base
constexpr int TC_SMEM = OFF_BAR + 64 + 1024;                // + alignment slack

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float bf16_round(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

// Logistic function on the SFU.  x3 mode: 1 / (1 + 2^(-x log2 e)) with the
// hardware base-2 exponential and reciprocal (relative error ~2^-22).
// Plain BF16 mode: (1 + tanh(x / 2)) / 2 with the hardware tanh (absolute
// error ~2^-11, below the BF16 rounding of the residual it feeds).
template <bool X3>
__device__ __forceinline__ float sigmoid_sfu(float x) {
    if (X3) return tc::rcp_approx(1.0f + tc::ex2_approx(-1.4426950408889634f * x));
    return fmaf(0.5f, tc::tanh_approx(0.5f * x), 0.5f);
}

template <bool LOGIT, bool X3>
__global__ void __launch_bounds__(TC_THREADS, 1) traj_tc_kernel(DevModel m, TrajArgs a, int cs, int nloc) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int quarter = wid & 3, colhalf = wid >> 2;
    const int prow = 32 * quarter + lane;            // particle row of this thread (TMEM lane)
    const uint32_t rank = tc::cluster_rank();
    const int tile = blockIdx.x / cs;
    const int D = m.D, n = m.n;
    const int obs0 = (int)rank * nloc;
    const int nmine = max(0, min(nloc, n - obs0));   // observations owned by this CTA
    const int nch = max(1, (nmine + TC_NC - 1) / TC_NC);

    uint64_t* bar_g1 = reinterpret_cast<uint64_t*>(sm + OFF_BAR);   // [4] GEMM1 chunk done
    uint64_t* bar_g2 = bar_g1 + TC_MAXCH;                            // [4] GEMM2 chunk done
    uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(bar_g1 + 2 * TC_MAXCH);
    float* y_s = reinterpret_cast<float*>(sm + OFF_Y);
    double* ll_s = reinterpret_cast<double*>(sm + OFF_LL);
    const uint32_t s_base = tc::smem_u32(sm);

    // ---------------------------------------------------------------- setup
    if (tid == 0) {
        for (int c = 0; c < TC_MAXCH; ++c) {
            tc::mbar_init(&bar_g1[c], 1);
            tc::mbar_init(&bar_g2[c], 1);
        }
        tc::fence_mbar_init();
    }
    if (wid == 0) {
        tc::tmem_alloc(tmem_base_s, TC_TMEM_COLS);
        tc::tmem_relinquish();
    }
    // X slice -> K-major SW64 rows (GEMM1 B) and K-major SW128 X^T rows (GEMM2 B)
    for (int e = tid; e < TC_NLOC * TC_DK; e += TC_THREADS) {
        const int i = e / TC_DK, d = e % TC_DK;
        const int c = i / TC_NC, r = i % TC_NC;   // chunk, row within the chunk
        uint16_t hi = 0, lo = 0;
        if (i < nmine && d < D) {
            hi = m.Xbf[(int64_t)(obs0 + i) * m.Dp + d];
            lo = m.Xbf_lo[(int64_t)(obs0 + i) * m.Dp + d];
        }
        const int xk = i * 64 + (((d >> 3) ^ ((i >> 1) & 3)) << 4) + (d & 7) * 2;
        const int w = r & 63;
        const int xt = c * XT_BYTES + (r >> 6) * XT_ATOM + d * 128 + (((w >> 3) ^ (d & 7)) << 4) + (w & 7) * 2;
        *reinterpret_cast<uint16_t*>(sm + OFF_XK + xk) = hi;
        *reinterpret_cast<uint16_t*>(sm + OFF_XT + xt) = hi;
        if (X3) {
            *reinterpret_cast<uint16_t*>(sm + OFF_XK + XK_PART + xk) = lo;
            *reinterpret_cast<uint16_t*>(sm + OFF_XT + XT_PART + xt) = lo;
        }
    }
    for (int i = tid; i < TC_NLOC; i += TC_THREADS) y_s[i] = i < nmine ? m.y[obs0 + i] : 0.0f;
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_base_s;
    tc::cluster_sync();   // every CTA of the cluster is running before any remote access

    // ---------------------------------------------------------------- particle state
    const float inv_tau2 = LOGIT ? (float)(1.0 / (m.h0 * m.h0)) : (float)(1.0 / (m.h1 * m.h1));
    const double inv_tau2_d = LOGIT ? 1.0 / (m.h0 * m.h0) : 1.0 / (m.h1 * m.h1);
    const float inv_s2 = LOGIT ? 0.0f : (float)(1.0 / (m.h0 * m.h0));
    const float inv_s = LOGIT ? 0.0f : (float)(1.0 / m.h0);
    const bool owner = wid < 4;     // warps 0-3 hold particle prow's state
    float th[TC_DK], p[TC_DK], g[TC_DK];
    int64_t j = -1, src = -1;
    int S = 0;
    float ef = 0.0f;
    double H0 = 0.0;
    {
        const int64_t t = (int64_t)tile * TC_P + prow;
        if (owner && t < a.N) {
            j = a.perm ? a.perm[t] : t;
            src = a.src ? a.src[j] : j;
            S = a.eval_only ? 0 : a.steps[j];
            int r;
            double eps;
            uint64_t seed;
            uint32_t kk, jl;
            particle_run(a, j, r, eps, seed, kk, jl);
            ef = (float)eps;
#pragma unroll
            for (int d = 0; d < TC_DK; ++d) {
                th[d] = d < D ? a.theta_in[(int64_t)d * a.ld + src] : 0.0f;
                g[d] = (d < D && !a.eval_only) ? a.grad_in[(int64_t)d * a.ld + src] : 0.0f;
                p[d] = 0.0f;
            }
            if (!a.eval_only) {
                if (a.p_in) {
#pragma unroll
                    for (int d = 0; d < TC_DK; ++d) p[d] = d < D ? a.p_in[(int64_t)d * a.ld + j] : 0.0f;
                } else {
#pragma unroll
                    for (int d = 0; d < TC_DK; d += 2) {
                        if (d < D) {
                            double z0, z1;
                            normal_pair(seed, (uint32_t)(d >> 1), jl, kk, TAG_MOM, z0, z1);
                            p[d] = (float)z0;
                            p[d + 1] = d + 1 < D ? (float)z1 : 0.0f;
                        }
                    }
                }
                double kin = 0.0;
#pragma unroll
                for (int d = 0; d < TC_DK; ++d) kin += (double)p[d] * (double)p[d];
                H0 = 0.5 * kin - a.logpi_in[src];
            }
        } else {
#pragma unroll
            for (int d = 0; d < TC_DK; ++d) th[d] = g[d] = p[d] = 0.0f;
        }
    }
    // uniform step count of the cluster: max S over the tile (identical in every CTA)
    __shared__ int smax_s;
    if (tid == 0) smax_s = 0;
    __syncthreads();
    if (owner && S > 0) atomicMax(&smax_s, S);
    __syncthreads();
    const int smax = smax_s;
    const int nsteps = a.eval_only ? 1 : smax;
    const float hf = 0.5f * ef;
    if (owner && S >= 1) {
#pragma unroll
        for (int d = 0; d < TC_DK; ++d) {
            p[d] = fmaf(hf, g[d], p[d]);
            th[d] = fmaf(ef, p[d], th[d]);
        }
    }

    constexpr uint32_t IDESC1 = tc::idesc_bf16_f32(TC_P, TC_NC);
    constexpr uint32_t IDESC2 = tc::idesc_bf16_f32(TC_P, TC_DK);
    int* err = a.dev_err;
    for (int s = 1; s <= nsteps; ++s) {
        // ---- Theta^T operand rows (hi, lo) from the current positions
        if (owner) {
            unsigned char* th_hi = sm + OFF_TH + prow * 64;
            unsigned char* th_lo = sm + OFF_TH + TH_BYTES + prow * 64;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                float hv[8], lv[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float x = th[8 * u + e];
                    hv[e] = bf16_round(x);
                    lv[e] = x - hv[e];
                }
                const int phys = (u ^ ((prow >> 1) & 3)) << 4;
                *reinterpret_cast<uint4*>(th_hi + phys) = make_uint4(
                    pack_bf16(hv[0], hv[1]), pack_bf16(hv[2], hv[3]), pack_bf16(hv[4], hv[5]), pack_bf16(hv[6], hv[7]));
                if (X3)
                    *reinterpret_cast<uint4*>(th_lo + phys) = make_uint4(
                        pack_bf16(lv[0], lv[1]), pack_bf16(lv[2], lv[3]), pack_bf16(lv[4], lv[5]), pack_bf16(lv[6], lv[7]));
            }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        // ---- GEMM1 for every chunk: eta^T = Theta^T X^T (TMEM columns [64c, 64c + 64))
        if (tid == 0) {
            tc::fence_after_sync();
            for (int c = 0; c < nch; ++c) {
                const uint32_t d_t = tmem + (uint32_t)(c * TC_NC);
                const int nparts = X3 ? 3 : 1;
                for (int q = 0; q < nparts; ++q) {
                    const int pa = (q == 1) ? 1 : 0;   // Theta part: hi, lo, hi
                    const int pb = (q == 2) ? 1 : 0;   // X part:     hi, hi, lo
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t ad = tc::smem_desc(s_base + OFF_TH + pa * TH_BYTES + kk * 32, 16, 512, tc::SWZ_64B);
                        const uint64_t bd = tc::smem_desc(s_base + OFF_XK + pb * XK_PART + c * XK_BYTES + kk * 32, 16, 512,
                                                          tc::SWZ_64B);
                        tc::mma_bf16(d_t, ad, bd, IDESC1, (q > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&bar_g1[c]);
            }
        }
        // ---- per chunk: residuals from TMEM -> R^T operand, GEMM2 accumulates.
        // x3 keeps one R^T buffer (hi + lo), plain BF16 one buffer per chunk.
        constexpr int NBUF = X3 ? 1 : 2;
        for (int c = 0; c < nch; ++c) {
            // every barrier completes exactly once per step: parity (s - 1) & 1
            tc::mbar_wait(&bar_g1[c], (uint32_t)((s - 1) & 1), err);
            if (c >= NBUF) tc::mbar_wait(&bar_g2[c - NBUF], (uint32_t)((s - 1) & 1), err);
            tc::fence_after_sync();
            const int rbuf = X3 ? 0 : (c & 1) * RT_BYTES;
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) {
                float eta[32];
                const uint32_t col = (uint32_t)(c * TC_NC + 64 * colhalf + 32 * blk);
                tc::tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + col, eta);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float hv[8], lv[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int i = c * TC_NC + 64 * colhalf + 32 * blk + 8 * u + e;
                        const float et = eta[8 * u + e];
                        float r;
                        if (LOGIT) r = y_s[i] - sigmoid_sfu<X3>(et);
                        else r = (y_s[i] - et) * inv_s2;
                        r = i < nmine ? r : 0.0f;
                        hv[e] = bf16_round(r);
                        lv[e] = r - hv[e];
                    }
                    const int chunk16 = 4 * blk + u;                    // within the 64-obs atom
                    const int off = rbuf + colhalf * RT_ATOM + prow * 128 + ((chunk16 ^ (prow & 7)) << 4);
                    *reinterpret_cast<uint4*>(sm + OFF_RT + off) = make_uint4(
                        pack_bf16(hv[0], hv[1]), pack_bf16(hv[2], hv[3]), pack_bf16(hv[4], hv[5]), pack_bf16(hv[6], hv[7]));
                    if (X3)
                        *reinterpret_cast<uint4*>(sm + OFF_RT + RT_BYTES + off) = make_uint4(
                            pack_bf16(lv[0], lv[1]), pack_bf16(lv[2], lv[3]), pack_bf16(lv[4], lv[5]),
                            pack_bf16(lv[6], lv[7]));
                }
            }
            tc::fence_proxy_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const int nparts = X3 ? 3 : 1;
                for (int q = 0; q < nparts; ++q) {
                    const int pr = (q == 1) ? 1 : 0;   // R part: hi, lo, hi
                    const int px = (q == 2) ? 1 : 0;   // X part: hi, hi, lo
                    for (int kk = 0; kk < TC_NC / 16; ++kk) {
                        const int atom = kk >> 2, ko = (kk & 3) * 32;
                        const uint64_t ad = tc::smem_desc(s_base + OFF_RT + rbuf + pr * RT_BYTES + atom * RT_ATOM + ko, 16,
                                                          1024, tc::SWZ_128B);
                        const uint64_t bd = tc::smem_desc(s_base + OFF_XT + px * XT_PART + c * XT_BYTES + atom * XT_ATOM + ko,
                                                          16, 1024, tc::SWZ_128B);
                        tc::mma_bf16(tmem + TC_COL_G, ad, bd, IDESC2, (c > 0 || q > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&bar_g2[c]);
            }
        }
        // ---- partial gradient of this CTA -> shared memory, cluster reduction
        const int gbuf = s & 1;
        float* gp = reinterpret_cast<float*>(sm + OFF_GP) + gbuf * TC_P * TC_GSTRIDE;
        for (int c = max(0, nch - NBUF); c < nch; ++c) tc::mbar_wait(&bar_g2[c], (uint32_t)((s - 1) & 1), err);
        tc::fence_after_sync();
        if (owner) {
            float gv[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + TC_COL_G, gv);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                *reinterpret_cast<float4*>(gp + prow * TC_GSTRIDE + 4 * u) =
                    make_float4(gv[4 * u], gv[4 * u + 1], gv[4 * u + 2], gv[4 * u + 3]);
        }
        tc::fence_before_sync();
        tc::cluster_sync();
        if (owner) {
            float gs[TC_DK];
#pragma unroll
            for (int d = 0; d < TC_DK; ++d) gs[d] = 0.0f;
            const uint32_t local = tc::smem_u32(gp + prow * TC_GSTRIDE);
            const int nu = (D + 3) >> 2;    // float4 groups holding the D live components
            for (int rr = 0; rr < cs; ++rr) {
                const uint32_t ra = tc::map_to_rank(local, (uint32_t)rr);
                float4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = u < nu ? tc::ld_cluster_f4(ra + 16 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    gs[4 * u] += v[u].x;
                    gs[4 * u + 1] += v[u].y;
                    gs[4 * u + 2] += v[u].z;
                    gs[4 * u + 3] += v[u].w;
                }
            }
#pragma unroll
            for (int d = 0; d < TC_DK; ++d) gs[d] = d < D ? gs[d] - th[d] * inv_tau2 : 0.0f;
            if (a.eval_only) {
#pragma unroll
                for (int d = 0; d < TC_DK; ++d) g[d] = gs[d];
            } else if (s <= S) {
#pragma unroll
                for (int d = 0; d < TC_DK; ++d) {
                    g[d] = gs[d];
                    p[d] = fmaf(hf, g[d], p[d]);
                    if (s + 1 <= S) {
                        p[d] = fmaf(hf, g[d], p[d]);
                        th[d] = fmaf(ef, p[d], th[d]);
                    }
                }
            }
        }
    }

    // ---------------------------------------------------------------- end point energy
    // FP32 eta, FP64 accumulation of the log-likelihood over this CTA's observations
    float* thT = reinterpret_cast<float*>(sm + OFF_RT);   // [32][128], R^T is no longer read
    tc::fence_before_sync();
    __syncthreads();
    if (owner)
#pragma unroll
        for (int d = 0; d < TC_DK; ++d) thT[d * TC_P + prow] = th[d];
    __syncthreads();
    {
        const int pp = tid & (TC_P - 1), half = tid >> 7;
        double ll = 0.0;
        for (int i = half; i < nmine; i += 2) {
            const float* x = m.X + (int64_t)(obs0 + i) * m.Dp;
            float e0 = 0.0f, e1 = 0.0f;
            for (int d = 0; d + 1 < D; d += 2) {
                e0 = fmaf(__ldg(x + d), thT[d * TC_P + pp], e0);
                e1 = fmaf(__ldg(x + d + 1), thT[(d + 1) * TC_P + pp], e1);
            }
            if (D & 1) e0 = fmaf(__ldg(x + D - 1), thT[(D - 1) * TC_P + pp], e0);
            const float eta = e0 + e1, yv = y_s[i];
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
        __syncthreads();
        if (half == 1) ll_s[pp] = ll;
        __syncthreads();
        if (half == 0) ll_s[pp] += ll;
    }
    tc::cluster_sync();
    if (rank == 0 && owner && j >= 0) {
        double tot = 0.0;
        const uint32_t local = tc::smem_u32(ll_s + prow);
        for (int rr = 0; rr < cs; ++rr) tot += tc::ld_cluster_f64(tc::map_to_rank(local, (uint32_t)rr));
        double sq = 0.0;
#pragma unroll
        for (int d = 0; d < TC_DK; ++d) sq += (double)th[d] * (double)th[d];   // padding is zero
        const double lp1 = tot - 0.5 * sq * inv_tau2_d + m.lconst;
#pragma unroll
        for (int d = 0; d < TC_DK; ++d) {
            if (d < D) {
                if (!a.eval_only) a.theta_out[(int64_t)d * a.ld + j] = th[d];
                a.grad_out[(int64_t)d * a.ld + j] = g[d];
                if (a.p_out && !a.eval_only) a.p_out[(int64_t)d * a.ld + j] = p[d];
            }
        }
        a.logpi_out[j] = lp1;
        if (!a.eval_only) {
            double kin = 0.0;
#pragma unroll
            for (int d = 0; d < TC_DK; ++d) kin += (double)p[d] * (double)p[d];
            double dH = (0.5 * kin - lp1) - H0;
            if (!isfinite(dH)) dH = CUDART_INF;
            if (a.dH) a.dH[j] = dH;
            if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
        }
    }
    tc::cluster_sync();   // no CTA leaves while a peer may still read its shared memory
    tc::fence_after_sync();
    if (wid == 0) tc::tmem_dealloc(tmem, TC_TMEM_COLS);
}

template <bool LOGIT, bool X3>
cudaError_t launch_tc(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const int cs = (m.n + TC_NLOC - 1) / TC_NLOC;
    const int nloc = (m.n + cs - 1) / cs;
    const int tiles = (int)((a.N + TC_P - 1) / TC_P);
    if (tiles == 0) return cudaSuccess;
    auto kern = traj_tc_kernel<LOGIT, X3>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    if (cs > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tiles * cs), 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = TC_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, m, a, cs, nloc);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

bool traj_tc_supported(const DevModel& m) {
    if (m.kind != LOGISTIC && m.kind != LINEAR_GAUSS) return false;
    if (m.D < 1 || m.D > TC_DK || !m.Xbf || !m.Xbf_lo) return false;
    const int cs = (m.n + TC_NLOC - 1) / TC_NLOC;
    return m.n >= 1 && cs <= 8;
}

cudaError_t launch_traj_tc(const DevModel& m, const TrajArgs& a, bool x3, cudaStream_t s) {
    if (!traj_tc_supported(m)) return cudaErrorInvalidValue;
    const bool logit = m.kind == LOGISTIC;
    if (logit) return x3 ? launch_tc<true, true>(m, a, s) : launch_tc<true, false>(m, a, s);
    return x3 ? launch_tc<false, true>(m, a, s) : launch_tc<false, false>(m, a, s);
}

}  // namespace smc
