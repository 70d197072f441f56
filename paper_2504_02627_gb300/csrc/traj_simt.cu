// traj_simt.cu -- FP32 SIMT leapfrog trajectory kernels (Sec. 2.1, Algorithm 1)
// with the fused momentum draw (Sec. 2.1: p ~ N(0, I)), the endpoint energy
// error Delta H and the acceptance probability min(1, exp(-Delta H)), and the
// dispatch of every model and precision to its trajectory kernel.
//
// Kernel families here (the thread-per-particle kernels are in
// traj_thread.cu):
//  * traj_glm_kernel: one CTA per group of G particles for the GEMM-shaped
//    likelihoods (logistic and linear-Gaussian regression): the design matrix
//    X stays in shared memory for the whole trajectory, the 512 threads split
//    the observations (lanes of a half-warp share one broadcast row of X) and
//    the per-particle gradient X'r is reduced across slices through shared
//    memory once per leapfrog step.
#include <cstdio>
#include <math_constants.h>
#include "traj.cuh"

namespace smc {

// ============================================================ GLM kernel
// G particles per CTA, NT threads, PP particles per thread: thread ->
// (particle group pl = tid % (G / PP), slice sl = tid / (G / PP)); the thread
// carries particles pl, pl + G/PP, ... and slice sl owns observations
// i = sl, sl + SL, ... (SL = NT / (G / PP)).  One X row loaded from shared
// memory serves the PP particles of the thread.  The products run over the
// first DR <= DP dimensions only (DR = D when the dimension is known at
// compile time, so no padding FMAs).
constexpr int GLM_THREADS = 512;

template <int DP, int G, int NT = GLM_THREADS>
struct GlmSmem {
    static constexpr int NW = NT / 32;
    static size_t bytes(int n) {
        size_t npad = (size_t)((n + 3) & ~3);
        return sizeof(float) * ((size_t)n * DP + npad + 3 * DP * G + (size_t)NW * DP * G) +
               sizeof(double) * (2 * G + NW * G) + sizeof(int) * (G + 4);
    }
};

template <bool LOGIT>
__device__ __forceinline__ float glm_resid(float y, float eta, float inv_s2) {
    if (LOGIT) return y - __fdividef(1.0f, 1.0f + __expf(-eta));
    return (y - eta) * inv_s2;
}

template <bool LOGIT>
__device__ __forceinline__ float glm_loglik_term(float y, float eta, float inv_s) {
    if (LOGIT) {
        float sp = eta > 0.0f ? eta + log1pf(expf(-eta)) : log1pf(expf(eta));
        return y * eta - sp;
    }
    float z = (y - eta) * inv_s;
    return -0.5f * z * z;
}

template <int DP, int G, bool LOGIT, int PP = 1, int NT = GLM_THREADS, int DR = DP>
__global__ void __launch_bounds__(NT, 1) traj_glm_kernel(DevModel m, TrajArgs a) {
    constexpr int NW = NT / 32, PG = G / PP, SL = NT / PG;
    static_assert(G <= 32 && (32 % G) == 0, "G must divide 32");
    static_assert(PG * PP == G && DR <= DP, "PP must divide G; DR <= DP");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = m.n, D = m.D;
    const int npad = (n + 3) & ~3;
    float* Xs = reinterpret_cast<float*>(smem_raw);
    float* ys = Xs + (size_t)n * DP;
    float* th_s = ys + npad;
    float* p_s = th_s + DP * G;
    float* g_s = p_s + DP * G;
    float* red = g_s + DP * G;
    double* H0_s = reinterpret_cast<double*>(red + NW * DP * G);
    double* lp_s = H0_s + G;
    double* red64 = lp_s + G;
    int* S_s = reinterpret_cast<int*>(red64 + NW * G);
    int* smax_s = S_s + G;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int pl = tid % PG, sl = tid / PG;

    // ---- model data into shared memory (whole trajectory reuses it)
    {
        const float4* Xg = reinterpret_cast<const float4*>(m.X);
        float4* Xs4 = reinterpret_cast<float4*>(Xs);
        const int nv = n * (DP / 4);
        for (int i = tid; i < nv; i += NT) Xs4[i] = Xg[i];
        for (int i = tid; i < n; i += NT) ys[i] = m.y[i];
    }
    const float inv_tau2 = LOGIT ? (float)(1.0 / (m.h0 * m.h0)) : (float)(1.0 / (m.h1 * m.h1));
    const double inv_tau2_d = LOGIT ? 1.0 / (m.h0 * m.h0) : 1.0 / (m.h1 * m.h1);
    const float inv_s2 = LOGIT ? 0.0f : (float)(1.0 / (m.h0 * m.h0));
    const float inv_s = LOGIT ? 0.0f : (float)(1.0 / m.h0);

    // ---- particle state of this CTA
    const int64_t slot0 = (int64_t)blockIdx.x * G;
    __shared__ int64_t j_s[G], src_s[G];
    __shared__ float eps_s[G];
    __shared__ uint64_t seed_s[G];
    __shared__ uint32_t k_s[G], jl_s[G];
    if (tid < G) {
        const int64_t t = slot0 + tid;
        int64_t j = -1, src = -1;
        int S = 0;
        float ef = 0.0f;
        if (t < a.N) {
            j = a.perm ? a.perm[t] : t;
            src = a.src ? a.src[j] : j;
            S = a.eval_only ? 0 : a.steps[j];
            int r;
            double eps;
            uint64_t seed;
            uint32_t kk, jl;
            particle_run(a, j, r, eps, seed, kk, jl);
            ef = (float)eps;
            seed_s[tid] = seed;
            k_s[tid] = kk;
            jl_s[tid] = jl;
        }
        j_s[tid] = j;
        src_s[tid] = src;
        S_s[tid] = S;
        eps_s[tid] = ef;
    }
    __syncthreads();
    if (tid == 0) {
        int mx = 0;
        for (int i = 0; i < G; ++i) mx = max(mx, S_s[i]);
        *smax_s = mx;
    }
    for (int e = tid; e < DP * G; e += NT) {
        const int d = e / G, q = e % G;
        const int64_t src = src_s[q];
        float tv = 0.0f, gv = 0.0f, pv = 0.0f;
        if (src >= 0 && d < D) {
            tv = a.theta_in[(int64_t)d * a.ld + src];
            if (!a.eval_only) gv = a.grad_in[(int64_t)d * a.ld + src];
            if (a.p_in && !a.eval_only) pv = a.p_in[(int64_t)d * a.ld + j_s[q]];
        }
        th_s[d * G + q] = tv;
        g_s[d * G + q] = gv;
        p_s[d * G + q] = pv;
    }
    __syncthreads();
    if (!a.p_in && !a.eval_only) {
        // momentum p ~ N(0, I) from the (seed, i, j, k, MOM) Philox stream
        const int npairs = (D + 1) / 2;
        for (int e = tid; e < npairs * G; e += NT) {
            const int i = e / G, q = e % G;
            if (j_s[q] < 0) continue;
            double z0, z1;
            normal_pair(seed_s[q], (uint32_t)i, jl_s[q], k_s[q], TAG_MOM, z0, z1);
            p_s[(2 * i) * G + q] = (float)z0;
            if (2 * i + 1 < D) p_s[(2 * i + 1) * G + q] = (float)z1;
        }
        __syncthreads();
    }
    if (tid < G && !a.eval_only) {
        double kin = 0.0;
        for (int d = 0; d < D; ++d) {
            double v = p_s[d * G + tid];
            kin += v * v;
        }
        H0_s[tid] = j_s[tid] >= 0 ? 0.5 * kin - a.logpi_in[src_s[tid]] : 0.0;
    }
    __syncthreads();   // H0 reads p_s before the first half kick below rewrites it
    const int smax = *smax_s;

    // ---- first half kick and drift of step 1
    for (int e = tid; e < DP * G; e += NT) {
        const int d = e / G, q = e % G;
        if (d < D && S_s[q] >= 1) {
            const float ef = eps_s[q], he = 0.5f * ef;
            float pv = fmaf(he, g_s[e], p_s[e]);
            p_s[e] = pv;
            th_s[e] = fmaf(ef, pv, th_s[e]);
        }
    }
    __syncthreads();

    const int nsteps = a.eval_only ? 1 : smax;
    for (int s = 1; s <= nsteps; ++s) {
        // ---- gradient X'(y - sigmoid(X theta)) for the G particles (phase B)
        float th[PP][DR], acc[PP][DR];
#pragma unroll
        for (int k = 0; k < PP; ++k)
#pragma unroll
            for (int d = 0; d < DR; ++d) {
                th[k][d] = th_s[d * G + pl + k * PG];
                acc[k][d] = 0.0f;
            }
        for (int i = sl; i < n; i += SL) {
            const float4* xr = reinterpret_cast<const float4*>(Xs + (size_t)i * DP);
            float xf[DP];
#pragma unroll
            for (int q = 0; q < DP / 4; ++q) {
                const float4 v = xr[q];
                xf[4 * q] = v.x;
                xf[4 * q + 1] = v.y;
                xf[4 * q + 2] = v.z;
                xf[4 * q + 3] = v.w;
            }
            const float yi = ys[i];
            float r[PP];
#pragma unroll
            for (int k = 0; k < PP; ++k) {
                float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, e3 = 0.0f;
#pragma unroll
                for (int d = 0; d < DR; d += 4) {
                    e0 = fmaf(xf[d], th[k][d], e0);
                    if (d + 1 < DR) e1 = fmaf(xf[d + 1], th[k][d + 1], e1);
                    if (d + 2 < DR) e2 = fmaf(xf[d + 2], th[k][d + 2], e2);
                    if (d + 3 < DR) e3 = fmaf(xf[d + 3], th[k][d + 3], e3);
                }
                r[k] = glm_resid<LOGIT>(yi, (e0 + e1) + (e2 + e3), inv_s2);
            }
#pragma unroll
            for (int k = 0; k < PP; ++k)
#pragma unroll
                for (int d = 0; d < DR; ++d) acc[k][d] = fmaf(r[k], xf[d], acc[k][d]);
        }
#pragma unroll
        for (int o = PG; o < 32; o <<= 1) {
#pragma unroll
            for (int k = 0; k < PP; ++k)
#pragma unroll
                for (int d = 0; d < DR; ++d) acc[k][d] += __shfl_xor_sync(0xffffffffu, acc[k][d], o);
        }
        if (lane < PG) {
#pragma unroll
            for (int k = 0; k < PP; ++k)
#pragma unroll
                for (int d = 0; d < DR; ++d) red[(wid * DP + d) * G + pl + k * PG] = acc[k][d];
        }
        __syncthreads();
        // ---- reduce, closing half kick of step s, opening kick + drift of s+1 (phase C)
        for (int e = tid; e < DP * G; e += NT) {
            const int d = e / G, q = e % G;
            if (d >= D) continue;
            float gs = 0.0f;
#pragma unroll
            for (int w = 0; w < NW; ++w) gs += red[(w * DP + d) * G + q];
            gs -= th_s[e] * inv_tau2;
            if (a.eval_only) {
                g_s[e] = gs;
            } else if (s <= S_s[q]) {
                const float ef = eps_s[q], he = 0.5f * ef;
                g_s[e] = gs;
                float pv = fmaf(he, gs, p_s[e]);
                if (s + 1 <= S_s[q]) {
                    pv = fmaf(he, gs, pv);
                    th_s[e] = fmaf(ef, pv, th_s[e]);
                }
                p_s[e] = pv;
            }
        }
        __syncthreads();
    }

    // ---- endpoint log pi in FP64 accumulation (energy error, Eq. for alpha)
    {
        float th[PP][DR];
#pragma unroll
        for (int k = 0; k < PP; ++k)
#pragma unroll
            for (int d = 0; d < DR; ++d) th[k][d] = th_s[d * G + pl + k * PG];
        double ll[PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) ll[k] = 0.0;
        for (int i = sl; i < n; i += SL) {
            const float4* xr = reinterpret_cast<const float4*>(Xs + (size_t)i * DP);
            float xf[DP];
#pragma unroll
            for (int q = 0; q < DP / 4; ++q) {
                const float4 v = xr[q];
                xf[4 * q] = v.x;
                xf[4 * q + 1] = v.y;
                xf[4 * q + 2] = v.z;
                xf[4 * q + 3] = v.w;
            }
#pragma unroll
            for (int k = 0; k < PP; ++k) {
                float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, e3 = 0.0f;
#pragma unroll
                for (int d = 0; d < DR; d += 4) {
                    e0 = fmaf(xf[d], th[k][d], e0);
                    if (d + 1 < DR) e1 = fmaf(xf[d + 1], th[k][d + 1], e1);
                    if (d + 2 < DR) e2 = fmaf(xf[d + 2], th[k][d + 2], e2);
                    if (d + 3 < DR) e3 = fmaf(xf[d + 3], th[k][d + 3], e3);
                }
                ll[k] += (double)glm_loglik_term<LOGIT>(ys[i], (e0 + e1) + (e2 + e3), inv_s);
            }
        }
#pragma unroll
        for (int o = PG; o < 32; o <<= 1)
#pragma unroll
            for (int k = 0; k < PP; ++k) ll[k] += __shfl_xor_sync(0xffffffffu, ll[k], o);
        if (lane < PG)
#pragma unroll
            for (int k = 0; k < PP; ++k) red64[wid * G + pl + k * PG] = ll[k];
        __syncthreads();
        if (tid < G) {
            double s = 0.0;
            for (int w = 0; w < NW; ++w) s += red64[w * G + tid];
            double sq = 0.0;
            for (int d = 0; d < D; ++d) {
                double v = th_s[d * G + tid];
                sq += v * v;
            }
            lp_s[tid] = s - 0.5 * sq * inv_tau2_d + m.lconst;
        }
        __syncthreads();
    }

    // ---- outputs
    for (int e = tid; e < DP * G; e += NT) {
        const int d = e / G, q = e % G;
        const int64_t j = j_s[q];
        if (j < 0 || d >= D) continue;
        if (!a.eval_only) a.theta_out[(int64_t)d * a.ld + j] = th_s[e];
        a.grad_out[(int64_t)d * a.ld + j] = g_s[e];
        if (a.p_out && !a.eval_only) a.p_out[(int64_t)d * a.ld + j] = p_s[e];
    }
    if (tid < G && j_s[tid] >= 0) {
        const int64_t j = j_s[tid];
        const double lp1 = lp_s[tid];
        a.logpi_out[j] = lp1;
        if (!a.eval_only) {
            double kin = 0.0;
            for (int d = 0; d < D; ++d) {
                double v = p_s[d * G + tid];
                kin += v * v;
            }
            double dH = (0.5 * kin - lp1) - H0_s[tid];
            if (!isfinite(dH)) dH = CUDART_INF;
            if (a.dH) a.dH[j] = dH;
            if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
        }
    }
}

// ============================================================ dense Gaussian, D > 32
// 32 particles per CTA, 256 threads.  The precision P (transposed, so that a
// thread's four rows are contiguous) and mu stay in shared memory; theta, p and
// grad live in shared memory as [DP][32].  grad = -P (theta - mu) is a
// register-tiled product: thread t owns rows 4*(t/8)..+3 and particles
// 4*(t%8)..+3 (16 accumulators, two 16-byte shared loads per 16 FMAs).
constexpr int DENSE_G = 32;
constexpr int DENSE_THREADS = 256;

template <int DP>
struct DenseSmem {
    static size_t bytes() { return sizeof(float) * ((size_t)DP * DP + DP + 3 * DP * DENSE_G) + sizeof(double) * 2 * DENSE_G; }
};

template <int DP>
__global__ void __launch_bounds__(DENSE_THREADS, 1) traj_dense_kernel(DevModel m, TrajArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Pt = reinterpret_cast<float*>(smem_raw);        // [DP][DP], Pt[k][d] = P[d][k]
    float* mu = Pt + DP * DP;                               // [DP]
    float* th_s = mu + DP;                                  // [DP][32]
    float* p_s = th_s + DP * DENSE_G;
    float* g_s = p_s + DP * DENSE_G;
    double* H0_s = reinterpret_cast<double*>(g_s + DP * DENSE_G);
    double* lp_s = H0_s + DENSE_G;
    __shared__ int64_t j_s[DENSE_G], src_s[DENSE_G];
    __shared__ int S_s[DENSE_G];
    __shared__ float eps_s[DENSE_G];
    __shared__ uint64_t seed_s[DENSE_G];
    __shared__ uint32_t k_s[DENSE_G], jl_s[DENSE_G];
    __shared__ int smax_s;
    const int tid = threadIdx.x, D = m.D;
    for (int e = tid; e < DP * DP; e += DENSE_THREADS) {
        const int k = e / DP, d = e % DP;
        Pt[e] = (k < D && d < D) ? m.P[d * D + k] : 0.0f;
    }
    for (int e = tid; e < DP; e += DENSE_THREADS) mu[e] = e < D ? m.mu[e] : 0.0f;
    const int64_t slot0 = (int64_t)blockIdx.x * DENSE_G;
    if (tid < DENSE_G) {
        const int64_t t = slot0 + tid;
        int64_t j = -1, src = -1;
        int S = 0;
        float ef = 0.0f;
        if (t < a.N) {
            j = a.perm ? a.perm[t] : t;
            src = a.src ? a.src[j] : j;
            S = a.eval_only ? 0 : a.steps[j];
            int r;
            double eps;
            uint64_t seed;
            uint32_t kk, jl;
            particle_run(a, j, r, eps, seed, kk, jl);
            ef = (float)eps;
            seed_s[tid] = seed;
            k_s[tid] = kk;
            jl_s[tid] = jl;
        }
        j_s[tid] = j;
        src_s[tid] = src;
        S_s[tid] = S;
        eps_s[tid] = ef;
    }
    __syncthreads();
    if (tid == 0) {
        int mx = 0;
        for (int i = 0; i < DENSE_G; ++i) mx = max(mx, S_s[i]);
        smax_s = mx;
    }
    for (int e = tid; e < DP * DENSE_G; e += DENSE_THREADS) {
        const int d = e / DENSE_G, q = e % DENSE_G;
        const int64_t src = src_s[q];
        float tv = 0.0f, gv = 0.0f, pv = 0.0f;
        if (src >= 0 && d < D) {
            tv = a.theta_in[(int64_t)d * a.ld + src];
            if (!a.eval_only) gv = a.grad_in[(int64_t)d * a.ld + src];
            if (a.p_in && !a.eval_only) pv = a.p_in[(int64_t)d * a.ld + j_s[q]];
        }
        th_s[e] = tv;
        g_s[e] = gv;
        p_s[e] = pv;
    }
    __syncthreads();
    if (!a.p_in && !a.eval_only) {
        const int npairs = (D + 1) / 2;
        for (int e = tid; e < npairs * DENSE_G; e += DENSE_THREADS) {
            const int i = e / DENSE_G, q = e % DENSE_G;
            if (j_s[q] < 0) continue;
            double z0, z1;
            normal_pair(seed_s[q], (uint32_t)i, jl_s[q], k_s[q], TAG_MOM, z0, z1);
            p_s[(2 * i) * DENSE_G + q] = (float)z0;
            if (2 * i + 1 < D) p_s[(2 * i + 1) * DENSE_G + q] = (float)z1;
        }
        __syncthreads();
    }
    if (tid < DENSE_G && !a.eval_only) {
        double kin = 0.0;
        for (int d = 0; d < D; ++d) {
            const double v = p_s[d * DENSE_G + tid];
            kin += v * v;
        }
        H0_s[tid] = j_s[tid] >= 0 ? 0.5 * kin - a.logpi_in[src_s[tid]] : 0.0;
    }
    __syncthreads();   // H0 reads p_s before the first half kick rewrites it
    const int smax = smax_s;
    for (int e = tid; e < DP * DENSE_G; e += DENSE_THREADS) {
        const int d = e / DENSE_G, q = e % DENSE_G;
        if (d < D && S_s[q] >= 1) {
            const float ef = eps_s[q], he = 0.5f * ef;
            const float pv = fmaf(he, g_s[e], p_s[e]);
            p_s[e] = pv;
            th_s[e] = fmaf(ef, pv, th_s[e]);
        }
    }
    __syncthreads();
    const int nsteps = a.eval_only ? 1 : smax;
    for (int s = 1; s <= nsteps; ++s) {
        // gradient at the drifted positions into a staging copy (g_s keeps the
        // frozen gradient of particles whose trajectory has ended)
        __syncthreads();
        {
            const int db = tid >> 3, pb = tid & 7;
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] = 0.0f;
            if (4 * db < DP) {
                for (int k = 0; k < D; ++k) {
                    const float4 av4 = *reinterpret_cast<const float4*>(Pt + k * DP + 4 * db);
                    const float4 t4 = *reinterpret_cast<const float4*>(th_s + k * DENSE_G + 4 * pb);
                    const float mk = mu[k];
                    const float b0 = t4.x - mk, b1 = t4.y - mk, b2 = t4.z - mk, b3 = t4.w - mk;
                    const float av[4] = {av4.x, av4.y, av4.z, av4.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        acc[i][0] = fmaf(av[i], b0, acc[i][0]);
                        acc[i][1] = fmaf(av[i], b1, acc[i][1]);
                        acc[i][2] = fmaf(av[i], b2, acc[i][2]);
                        acc[i][3] = fmaf(av[i], b3, acc[i][3]);
                    }
                }
            }
            __syncthreads();   // every thread has read th_s before anyone moves it
            if (4 * db < DP) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int d = 4 * db + i;
                    if (d >= D) continue;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        const int q = 4 * pb + qq, e = d * DENSE_G + q;
                        const float gsv = -acc[i][qq];
                        if (a.eval_only) {
                            g_s[e] = gsv;
                        } else if (s <= S_s[q]) {
                            const float ef = eps_s[q], he = 0.5f * ef;
                            g_s[e] = gsv;
                            float pv = fmaf(he, gsv, p_s[e]);
                            if (s + 1 <= S_s[q]) {
                                pv = fmaf(he, gsv, pv);
                                th_s[e] = fmaf(ef, pv, th_s[e]);
                            }
                            p_s[e] = pv;
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    // end point: log pi = c - 1/2 (theta - mu)' P (theta - mu) = c + 1/2 (theta - mu)' grad,
    // FP64 accumulation of the FP32 gradient of the final position
    if (tid < DENSE_G) {
        double q2 = 0.0, kin = 0.0;
        for (int d = 0; d < D; ++d) {
            const double dl = (double)th_s[d * DENSE_G + tid] - (double)mu[d];
            q2 += dl * (double)g_s[d * DENSE_G + tid];
            const double v = p_s[d * DENSE_G + tid];
            kin += v * v;
        }
        lp_s[tid] = m.lconst + 0.5 * q2;
        if (j_s[tid] >= 0) {
            const int64_t j = j_s[tid];
            const double lp1 = lp_s[tid];
            a.logpi_out[j] = lp1;
            if (!a.eval_only) {
                double dH = (0.5 * kin - lp1) - H0_s[tid];
                if (!isfinite(dH)) dH = CUDART_INF;
                if (a.dH) a.dH[j] = dH;
                if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
            }
        }
    }
    for (int e = tid; e < DP * DENSE_G; e += DENSE_THREADS) {
        const int d = e / DENSE_G, q = e % DENSE_G;
        const int64_t j = j_s[q];
        if (j < 0 || d >= D) continue;
        if (!a.eval_only) a.theta_out[(int64_t)d * a.ld + j] = th_s[e];
        a.grad_out[(int64_t)d * a.ld + j] = g_s[e];
        if (a.p_out && !a.eval_only) a.p_out[(int64_t)d * a.ld + j] = p_s[e];
    }
}

// ============================================================ dispatch
namespace {

template <int DP, int G, bool LOGIT, int PP = 1, int NT = GLM_THREADS, int DR = DP>
cudaError_t launch_glm(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const size_t sm = GlmSmem<DP, G, NT>::bytes(m.n);
    auto kern = traj_glm_kernel<DP, G, LOGIT, PP, NT, DR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t grid = (a.N + G - 1) / G;
    if (grid == 0) return cudaSuccess;
    kern<<<(unsigned)grid, NT, sm, s>>>(m, a);
    return cudaGetLastError();
}

template <bool LOGIT>
cudaError_t dispatch_glm(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    switch (m.Dp) {
        case 4: return launch_glm<4, 16, LOGIT, 2, 384>(m, a, s);
        case 8: return launch_glm<8, 16, LOGIT, 2, 384>(m, a, s);
        case 16: return launch_glm<16, 16, LOGIT, 2, 384>(m, a, s);
        case 28:   // two particles per thread; the 25-dimensional regression without padding FMAs
            return m.D == 25 ? launch_glm<28, 16, LOGIT, 2, 384, 25>(m, a, s) : launch_glm<28, 16, LOGIT, 2, 384>(m, a, s);
        case 32: return launch_glm<32, 16, LOGIT>(m, a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int DP>
cudaError_t launch_dense(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const size_t sm = DenseSmem<DP>::bytes();
    auto kern = traj_dense_kernel<DP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t grid = (a.N + DENSE_G - 1) / DENSE_G;
    if (grid == 0) return cudaSuccess;
    kern<<<(unsigned)grid, DENSE_THREADS, sm, s>>>(m, a);
    return cudaGetLastError();
}

cudaError_t dispatch_dense(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    if (m.D <= 48) return launch_dense<48>(m, a, s);
    if (m.D <= 64) return launch_dense<64>(m, a, s);
    if (m.D <= 100) return launch_dense<100>(m, a, s);
    if (m.D <= 128) return launch_dense<128>(m, a, s);
    return cudaErrorInvalidValue;
}

bool glm_shape_ok(const DevModel& m) {
    if (m.Dp != 4 && m.Dp != 8 && m.Dp != 16 && m.Dp != 28 && m.Dp != 32) return false;
    return GlmSmem<32, 16>::bytes(m.n) <= 220 * 1024;
}

}  // namespace

bool traj_supported(const DevModel& m, int32_t precision) {
    if (precision == 1 || precision == 2) {
        if (m.kind == GAUSS_DENSE) return traj_gauss_mma_supported(m);
        if (precision == 1) return traj_glm_mma_supported(m, true) || traj_tc_supported(m);
        return traj_glm_mma_supported(m, false) || traj_tc_supported(m) || traj_stream_supported(m);
    }
    if (precision == 3) return traj_stream_supported(m);
    if (precision == 4) return traj_centred_supported(m);
    switch (m.kind) {
        case GAUSS_DENSE: return precision == 0 && m.D <= 128;
        case BANANA: return precision == 0 && m.D <= 64;
        case HIER_NORMAL: return precision == 0 && m.D <= 64;
        case LOGISTIC:
        case LINEAR_GAUSS: return precision == 0 && (glm_shape_ok(m) || traj_glm_stream_supported(m));
        default: return false;
    }
}

int32_t traj_tile_count(const DevModel& m, int32_t precision) {
    if (precision != 0 || !traj_supported(m, precision)) return 1;
    if (m.kind == GAUSS_DENSE && m.D > 32) return 1;
    return m.kind == GAUSS_DENSE || m.kind == BANANA || m.kind == HIER_NORMAL ? traj_thread_tiles(m) : 1;
}

cudaError_t launch_traj(const DevModel& m, const TrajArgs& a, int32_t precision, cudaStream_t s) {
    if (!traj_supported(m, precision)) return cudaErrorInvalidValue;
    if (a.N <= 0) return cudaSuccess;   // nothing to launch (a zero-size grid is an error)
    if ((precision == 1 || precision == 2) && m.kind == GAUSS_DENSE)
        return launch_traj_gauss_mma(m, a, precision == 1, s);
    if (precision == 1)
        return traj_glm_mma_supported(m, true) ? launch_traj_glm_mma(m, a, true, s) : launch_traj_tc(m, a, true, s);
    if (precision == 2) {
        if (traj_glm_mma_supported(m, false)) return launch_traj_glm_mma(m, a, false, s);
        return traj_tc_supported(m) ? launch_traj_tc(m, a, false, s) : launch_traj_stream(m, a, 1, s);
    }
    if (precision == 3) return launch_traj_stream(m, a, 2, s);
    if (precision == 4) return launch_traj_centred(m, a, s);
    switch (m.kind) {
        case GAUSS_DENSE: return m.D <= 32 ? launch_traj_thread(m, a, s) : dispatch_dense(m, a, s);
        case BANANA:
        case HIER_NORMAL: return launch_traj_thread(m, a, s);
        case LOGISTIC:
            return glm_shape_ok(m) ? dispatch_glm<true>(m, a, s) : launch_traj_glm_stream(m, a, s);
        case LINEAR_GAUSS:
            return glm_shape_ok(m) ? dispatch_glm<false>(m, a, s) : launch_traj_glm_stream(m, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace smc
