// traj_glm_mma.cu -- tensor-core leapfrog trajectories (Algorithm 1) for
// Bayesian logistic regression (Sec. 4) and linear-Gaussian regression of
// moderate size (X resident in shared memory, D <= 32), on warp-level BF16
// MMAs (m16n8k16, FP32 accumulation).
//
// Per leapfrog step the gradient of a tile of 16 particles is two products
// joined by an elementwise map,
//
//   eta [16 x obs]  = Theta [16 x 32] . X^T        (GEMM1)
//   r               = y - sigmoid(eta)  (or (y - eta) / sigma^2)
//   G   [16 x 32]  += r [16 x obs] . X [obs x 32]   (GEMM2)
//
// and both stay in registers: the FP32 accumulator fragment of GEMM1 for 16
// observations has exactly the thread/element distribution of the A operand
// of GEMM2, so the residual is computed where eta lands and fed to the next
// product without a round trip through shared or tensor memory.  This shape
// matters here: the benchmark's 4096 particles leave about 27 per SM, far
// fewer than the 128 rows of a tcgen05 tile, so an SM's share of the work is
// a long chain of small dependent products.  Issued per warp and
// synchronously, with 16 warps per CTA each on its own slice of the
// observations, the chain keeps the tensor pipe fed without TMEM traffic or
// cross-proxy fences between the two products.
//
// Precision: BF16 operands, FP32 accumulation.  In the x3 mode every operand
// is split a = hi + lo (both BF16) and hi*hi + lo*hi + hi*lo is accumulated
// (the lo*lo term is dropped); the plain mode uses the hi parts only.  The
// reduced-precision gradient only changes the integrator: the end-point
// log pi that enters the importance weight is an FP32 product with FP64
// accumulation, as in every trajectory kernel here.
//
// Shared memory of one CTA: X as BF16 hi (and lo) rows of 32 dims (64 bytes,
// 16-byte chunks XOR-swizzled by row so that the 8-row matrix loads of both
// products are free of bank conflicts), y, the particle state, and the
// per-warp partial gradients, summed in warp order once per step.
#include <cuda_bf16.h>
#include <math_constants.h>
#include "tc_ptx.cuh"
#include "traj.cuh"

namespace smc {
namespace {

constexpr int GM_P = 16;              // particles per CTA (the M of the MMA)
constexpr int GM_W = 16;              // warps per CTA, each on a slice of the observation chunks
constexpr int GM_T = 32 * GM_W;
constexpr int GM_DK = 32;             // padded dimension: two k-steps of GEMM1, four n-tiles of GEMM2
constexpr int GM_RS = 40;             // floats per particle row of the partial-gradient buffer
constexpr int GM_TS = 40;             // floats per particle row of theta, p, grad (padding zero)
constexpr int GM_CH = 16;             // observations per chunk (one k-step of GEMM2)
constexpr int GM_AS = 40;             // bf16 per row of the theta operand tile (80 bytes: an odd
                                      // number of 16-byte units, conflict-free 8x8 matrix loads)
static_assert(GM_W == GM_P, "the end point gives one warp to each particle");

// Dynamic shared memory (bytes): X hi [n16][64] | X lo [n16][64] (x3) |
// y [n16] f32 | theta, p, grad [16][40] f32 | partials [16 warps][16][40] f32 |
// theta operand hi, lo [16][40] bf16 | H0, log pi [16] f64.
struct GmLayout {
    int n16;
    size_t xh, xl, y, th, p, g, red, at, h0, lp, bytes;
    __host__ __device__ GmLayout(int n, bool x3) {
        n16 = (n + GM_CH - 1) / GM_CH * GM_CH;
        xh = 0;
        xl = xh + (size_t)n16 * 64;
        y = xl + (x3 ? (size_t)n16 * 64 : 0);
        th = y + (size_t)n16 * 4;
        p = th + GM_P * GM_TS * 4;
        g = p + GM_P * GM_TS * 4;
        red = g + GM_P * GM_TS * 4;
        at = red + (size_t)GM_W * GM_P * GM_RS * 4;
        h0 = at + 2 * (size_t)GM_P * GM_AS * 2;
        lp = h0 + GM_P * 8;
        bytes = lp + GM_P * 8;
    }
};

// byte offset of the 16-byte chunk c (dims 8c .. 8c+7) of X row r
__device__ __forceinline__ uint32_t gm_xoff(int r, int c) {
    return (uint32_t)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4));
}

template <bool LOGIT, bool X3>
__device__ __forceinline__ float gm_resid(float y, float eta, float inv_s2) {
    if (LOGIT) {
        // x3: 1 / (1 + 2^(-eta log2 e)) on the SFU (relative error ~2^-22);
        // plain BF16: (1 + tanh(eta / 2)) / 2 (absolute error ~2^-11, below the
        // BF16 rounding of the residual it feeds)
        const float sg = X3 ? tc::rcp_approx(1.0f + tc::ex2_approx(-1.4426950408889634f * eta))
                            : fmaf(0.5f, tc::tanh_approx(0.5f * eta), 0.5f);
        return y - sg;
    }
    return (y - eta) * inv_s2;
}

template <bool LOGIT, bool X3>
__global__ void __launch_bounds__(GM_T, 1) traj_glm_mma_kernel(DevModel m, TrajArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = m.n, D = m.D;
    const GmLayout L(n, X3);
    const int nch = L.n16 / GM_CH;
    float* y_s = reinterpret_cast<float*>(smem_raw + L.y);
    float* th_s = reinterpret_cast<float*>(smem_raw + L.th);
    float* p_s = reinterpret_cast<float*>(smem_raw + L.p);
    float* g_s = reinterpret_cast<float*>(smem_raw + L.g);
    float* red = reinterpret_cast<float*>(smem_raw + L.red);
    double* H0_s = reinterpret_cast<double*>(smem_raw + L.h0);
    double* lp_s = reinterpret_cast<double*>(smem_raw + L.lp);
    const uint32_t xh_base = tc::smem_u32(smem_raw + L.xh);
    const uint32_t xl_base = tc::smem_u32(smem_raw + L.xl);
    // theta as the A operand of GEMM1: BF16 hi and lo rows [16][GM_AS], written
    // by the threads that move theta, read by every warp with 8x8 matrix loads
    const uint32_t at_base = tc::smem_u32(smem_raw + L.at);
    constexpr uint32_t AT_LO = GM_P * GM_AS * 2;   // bytes from the hi tile to the lo tile
    auto put_at = [&](int q, int d, float v) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        __nv_bfloat16* t = reinterpret_cast<__nv_bfloat16*>(smem_raw + L.at) + q * GM_AS + d;
        t[0] = h;
        if (X3) t[GM_P * GM_AS] = __float2bfloat16_rn(v - __bfloat162float(h));
    };
    __shared__ int64_t j_s[GM_P], src_s[GM_P];
    __shared__ float eps_s[GM_P];
    __shared__ uint64_t seed_s[GM_P];
    __shared__ uint32_t k_s[GM_P], jl_s[GM_P];
    __shared__ int S_s[GM_P];
    __shared__ int smax_s;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gq = lane >> 2, tq = lane & 3;   // MMA fragment row group / column pair

    // ---- X (BF16 hi, lo): the pre-swizzled image copied asynchronously
    //      (waited on before the first product); y; rows past n are zero
    {
        const uint4* img = reinterpret_cast<const uint4*>(m.xmma_img);
        const int nv = L.n16 * 4;   // 16-byte units per block
        for (int e = tid; e < nv; e += GM_T) tc::cp_async16(smem_raw + L.xh + 16 * (size_t)e, img + e);
        if (X3)
            for (int e = tid; e < nv; e += GM_T) tc::cp_async16(smem_raw + L.xl + 16 * (size_t)e, img + nv + e);
        tc::cp_async_commit();
    }
    for (int i = tid; i < L.n16; i += GM_T) y_s[i] = i < n ? m.y[i] : 0.0f;
    const float inv_tau2 = LOGIT ? (float)(1.0 / (m.h0 * m.h0)) : (float)(1.0 / (m.h1 * m.h1));
    const double inv_tau2_d = LOGIT ? 1.0 / (m.h0 * m.h0) : 1.0 / (m.h1 * m.h1);
    const float inv_s2 = LOGIT ? 0.0f : (float)(1.0 / (m.h0 * m.h0));
    const float inv_s = LOGIT ? 0.0f : (float)(1.0 / m.h0);

    // ---- particle state of this CTA
    const int64_t slot0 = (int64_t)blockIdx.x * GM_P;
    if (tid < GM_P) {
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
        for (int q = 0; q < GM_P; ++q) mx = max(mx, S_s[q]);
        smax_s = mx;
    }
    for (int e = tid; e < GM_P * GM_TS; e += GM_T) {
        const int q = e / GM_TS, d = e % GM_TS;
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
    // the theta operand tile starts at zero (columns past D stay zero)
    for (int e = tid; e < GM_P * GM_AS; e += GM_T)   // 32-bit words: both tiles
        reinterpret_cast<uint32_t*>(smem_raw + L.at)[e] = 0u;
    __syncthreads();
    if (!a.p_in && !a.eval_only) {
        // momentum p ~ N(0, I) from the (seed, i, j, k, MOM) Philox stream
        const int npairs = (D + 1) / 2;
        for (int e = tid; e < npairs * GM_P; e += GM_T) {
            const int i = e / GM_P, q = e % GM_P;
            if (j_s[q] < 0) continue;
            double z0, z1;
            normal_pair(seed_s[q], (uint32_t)i, jl_s[q], k_s[q], TAG_MOM, z0, z1);
            p_s[q * GM_TS + 2 * i] = (float)z0;
            if (2 * i + 1 < D) p_s[q * GM_TS + 2 * i + 1] = (float)z1;
        }
        __syncthreads();
    }
    if (tid < GM_P && !a.eval_only) {
        double kin = 0.0;
        for (int d = 0; d < D; ++d) {
            const double v = p_s[tid * GM_TS + d];
            kin += v * v;
        }
        H0_s[tid] = j_s[tid] >= 0 ? 0.5 * kin - a.logpi_in[src_s[tid]] : 0.0;
    }
    __syncthreads();   // H0 reads p_s before the first half kick below rewrites it
    const int smax = smax_s;

    // ---- first half kick and drift of step 1
    for (int e = tid; e < GM_P * GM_TS; e += GM_T) {
        const int q = e / GM_TS, d = e % GM_TS;
        if (d < D && S_s[q] >= 1) {
            const float ef = eps_s[q], he = 0.5f * ef;
            const float pv = fmaf(he, g_s[e], p_s[e]);
            p_s[e] = pv;
            th_s[e] = fmaf(ef, pv, th_s[e]);
        }
        if (d < D) put_at(q, d, th_s[e]);
    }
    tc::cp_async_wait<0>();
    __syncthreads();

    // ldmatrix lane roles: matrix mi = lane / 8, row lane % 8 of it
    const int mi = lane >> 3, mr = lane & 7;
    const int nsteps = a.eval_only ? 1 : smax;
    for (int s = 1; s <= nsteps; ++s) {
        // ---- Theta as the A operand of GEMM1 (hi, lo) for the two k-steps:
        //      matrices (particles 8 (mi & 1) .., dims 16 ks + 8 (mi >> 1) ..)
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const uint32_t aoff = (uint32_t)(((8 * (mi & 1) + mr) * GM_AS + 16 * ks + 8 * (mi >> 1)) * 2);
            tc::ldsm4(ah[ks], at_base + aoff);
            if (X3) tc::ldsm4(al[ks], at_base + AT_LO + aoff);
        }
        float gacc[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int v = 0; v < 4; ++v) gacc[nt][v] = 0.0f;

        // GEMM1 of observations r0 .. r0 + 15 (two n-tiles of 8); in the x3
        // mode the correction products accumulate apart from hi*hi, which
        // halves the dependent chain of each accumulator
        auto gemm1 = [&](int r0, float (&eta)[2][4]) {
            float cor[2][4];
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int v = 0; v < 4; ++v) eta[j][v] = cor[j][v] = 0.0f;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                // matrices: (n-tile mi >> 1, dims 16 ks + 8 (mi & 1) .. + 7)
                const uint32_t off = gm_xoff(r0 + 8 * (mi >> 1) + mr, 2 * ks + (mi & 1));
                uint32_t bh[4], bl[4];
                tc::ldsm4(bh, xh_base + off);
                if (X3) tc::ldsm4(bl, xl_base + off);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    tc::mma_bf16_16816(eta[j], ah[ks], bh[2 * j], bh[2 * j + 1]);
                    if (X3) {
                        tc::mma_bf16_16816(cor[j], al[ks], bh[2 * j], bh[2 * j + 1]);
                        tc::mma_bf16_16816(cor[j], ah[ks], bl[2 * j], bl[2 * j + 1]);
                    }
                }
            }
            if (X3)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int v = 0; v < 4; ++v) eta[j][v] += cor[j][v];
        };

        // chunks c = wid, wid + 16, ...: GEMM1 of the next chunk is issued
        // before the residuals and GEMM2 of the current one
        float eta[2][4], eta_nx[2][4];
        if (wid < nch) gemm1(wid * GM_CH, eta);
        for (int c = wid; c < nch; c += GM_W) {
            const int r0 = c * GM_CH;
            const bool more = c + GM_W < nch;
            if (more) gemm1(r0 + GM_W * GM_CH, eta_nx);
            // residuals -> A operand of GEMM2 (rows g, g + 8; observations 2t, 2t + 1 (+ 8))
            uint32_t rh[4], rl[4];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float2 yv = *reinterpret_cast<const float2*>(y_s + r0 + 8 * j + 2 * tq);
                const float q0 = gm_resid<LOGIT, X3>(yv.x, eta[j][0], inv_s2);
                const float q1 = gm_resid<LOGIT, X3>(yv.y, eta[j][1], inv_s2);
                const float q2 = gm_resid<LOGIT, X3>(yv.x, eta[j][2], inv_s2);
                const float q3 = gm_resid<LOGIT, X3>(yv.y, eta[j][3], inv_s2);
                tc::split_bf16x2(q0, q1, rh[2 * j], rl[2 * j]);
                tc::split_bf16x2(q2, q3, rh[2 * j + 1], rl[2 * j + 1]);
            }
            // GEMM2: G += r . X over these 16 observations (four n-tiles of 8 dims)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // matrices (transposed): (dims 8 (2h + (mi >> 1)) .., observations 8 (mi & 1) ..)
                const uint32_t off = gm_xoff(r0 + 8 * (mi & 1) + mr, 2 * h + (mi >> 1));
                uint32_t bh[4], bl[4];
                tc::ldsm4_t(bh, xh_base + off);
                if (X3) tc::ldsm4_t(bl, xl_base + off);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int nt = 2 * h + u;
                    tc::mma_bf16_16816(gacc[nt], rh, bh[2 * u], bh[2 * u + 1]);
                    if (X3) {
                        tc::mma_bf16_16816(gacc[nt], rl, bh[2 * u], bh[2 * u + 1]);
                        tc::mma_bf16_16816(gacc[nt], rh, bl[2 * u], bl[2 * u + 1]);
                    }
                }
            }
            if (more)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int v = 0; v < 4; ++v) eta[j][v] = eta_nx[j][v];
        }
        // ---- this warp's partial gradients (rows g, g + 8; dims 8 nt + 2t, + 1)
        {
            float* rw = red + (size_t)wid * GM_P * GM_RS;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                *reinterpret_cast<float2*>(rw + gq * GM_RS + 8 * nt + 2 * tq) = make_float2(gacc[nt][0], gacc[nt][1]);
                *reinterpret_cast<float2*>(rw + (gq + 8) * GM_RS + 8 * nt + 2 * tq) =
                    make_float2(gacc[nt][2], gacc[nt][3]);
            }
        }
        __syncthreads();
        // ---- warp sums, prior term, closing half kick of step s, opening kick + drift of s + 1
        for (int e = tid; e < GM_P * GM_DK; e += GM_T) {
            const int q = e / GM_DK, d = e % GM_DK;
            if (d >= D) continue;
            const int ei = q * GM_TS + d;
            float gs = 0.0f;
#pragma unroll
            for (int w = 0; w < GM_W; ++w) gs += red[(w * GM_P + q) * GM_RS + d];
            gs -= th_s[ei] * inv_tau2;
            if (a.eval_only) {
                g_s[ei] = gs;
            } else if (s <= S_s[q]) {
                const float ef = eps_s[q], he = 0.5f * ef;
                g_s[ei] = gs;
                float pv = fmaf(he, gs, p_s[ei]);
                if (s + 1 <= S_s[q]) {
                    pv = fmaf(he, gs, pv);
                    th_s[ei] = fmaf(ef, pv, th_s[ei]);
                    put_at(q, d, th_s[ei]);
                }
                p_s[ei] = pv;
            }
        }
        __syncthreads();
    }

    // ---- end-point log pi: FP32 products with the FP32 X (each row read once
    //      per CTA, by one thread, for all 16 particles); a thread's few terms
    //      (ceil(n / 512) observations) summed in FP32, FP64 from there on
    {
        float llf[GM_P];
#pragma unroll
        for (int q = 0; q < GM_P; ++q) llf[q] = 0.0f;
        for (int i = tid; i < n; i += GM_T) {
            float x[GM_DK];
            const float4* xr = reinterpret_cast<const float4*>(m.X + (int64_t)i * m.Dp);
#pragma unroll
            for (int u = 0; u < GM_DK / 4; ++u) {
                const float4 v = 4 * u < m.Dp ? __ldg(xr + u) : make_float4(0.f, 0.f, 0.f, 0.f);
                x[4 * u] = v.x;
                x[4 * u + 1] = v.y;
                x[4 * u + 2] = v.z;
                x[4 * u + 3] = v.w;
            }
            const float yv = y_s[i];
#pragma unroll
            for (int q = 0; q < GM_P; ++q) {
                const float* thq = th_s + q * GM_TS;   // zero past D
                float e0 = 0.0f, e1 = 0.0f;
#pragma unroll
                for (int d = 0; d < GM_DK; d += 2) {
                    e0 = fmaf(x[d], thq[d], e0);
                    e1 = fmaf(x[d + 1], thq[d + 1], e1);
                }
                const float eta = e0 + e1;
                float term;
                if (LOGIT) {
                    const float sp = eta > 0.0f ? eta + log1pf(expf(-eta)) : log1pf(expf(eta));
                    term = yv * eta - sp;
                } else {
                    const float z = (yv - eta) * inv_s;
                    term = -0.5f * z * z;
                }
                llf[q] += term;
            }
        }
        // sum over the threads: lanes by a reduce-scatter butterfly (lane pair
        // 2 q, 2 q + 1 ends with particle q), warps through shared memory
        double* red64 = reinterpret_cast<double*>(red);   // [GM_W][GM_P]
        double ll[GM_P];
#pragma unroll
        for (int q = 0; q < GM_P; ++q) ll[q] = (double)llf[q];
        const double wsum = warp_sum16_scatter(ll, lane);
        if ((lane & 1) == 0) red64[wid * GM_P + (lane >> 1)] = wsum;
        __syncthreads();
        if (tid < GM_P) {
            double tot = 0.0;
            for (int w = 0; w < GM_W; ++w) tot += red64[w * GM_P + tid];
            double sq = 0.0;
            for (int d = 0; d < D; ++d) {
                const double v = th_s[tid * GM_TS + d];
                sq += v * v;
            }
            lp_s[tid] = tot - 0.5 * sq * inv_tau2_d + m.lconst;
        }
    }
    __syncthreads();

    // ---- outputs
    for (int e = tid; e < GM_P * GM_DK; e += GM_T) {
        const int q = e / GM_DK, d = e % GM_DK;
        const int64_t j = j_s[q];
        if (j < 0 || d >= D) continue;
        const int ei = q * GM_TS + d;
        if (!a.eval_only) a.theta_out[(int64_t)d * a.ld + j] = th_s[ei];
        a.grad_out[(int64_t)d * a.ld + j] = g_s[ei];
        if (a.p_out && !a.eval_only) a.p_out[(int64_t)d * a.ld + j] = p_s[ei];
    }
    if (tid < GM_P && j_s[tid] >= 0) {
        const int64_t j = j_s[tid];
        const double lp1 = lp_s[tid];
        a.logpi_out[j] = lp1;
        if (!a.eval_only) {
            double kin = 0.0;
            for (int d = 0; d < D; ++d) {
                const double v = p_s[tid * GM_TS + d];
                kin += v * v;
            }
            double dH = (0.5 * kin - lp1) - H0_s[tid];
            if (!isfinite(dH)) dH = CUDART_INF;
            if (a.dH) a.dH[j] = dH;
            if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
        }
    }
}

template <bool LOGIT, bool X3>
cudaError_t launch_gm(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const GmLayout L(m.n, X3);
    auto kern = traj_glm_mma_kernel<LOGIT, X3>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
    if (e != cudaSuccess) return e;
    const int64_t grid = (a.N + GM_P - 1) / GM_P;
    if (grid == 0) return cudaSuccess;
    kern<<<(unsigned)grid, GM_T, L.bytes, s>>>(m, a);
    return cudaGetLastError();
}

// The X image: unit c (dims 8c .. 8c + 7) of row r of the hi block at byte
// gm_xoff(r, c), the lo block after it
__global__ void k_glm_mma_image(const uint16_t* __restrict__ xh, const uint16_t* __restrict__ xl, int n, int n16,
                                int D, int Dp, uint16_t* __restrict__ img) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n16 * 4) return;
    const int r = e >> 2, c = e & 3;
    uint32_t hv[4] = {0u, 0u, 0u, 0u}, lv[4] = {0u, 0u, 0u, 0u};
    if (r < n) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int d = 8 * c + 2 * h;
            const uint32_t h0 = d < D ? xh[(int64_t)r * Dp + d] : 0u;
            const uint32_t h1 = d + 1 < D ? xh[(int64_t)r * Dp + d + 1] : 0u;
            const uint32_t l0 = d < D ? xl[(int64_t)r * Dp + d] : 0u;
            const uint32_t l1 = d + 1 < D ? xl[(int64_t)r * Dp + d + 1] : 0u;
            hv[h] = h0 | (h1 << 16);
            lv[h] = l0 | (l1 << 16);
        }
    }
    unsigned char* base = reinterpret_cast<unsigned char*>(img);
    const uint32_t off = gm_xoff(r, c);
    *reinterpret_cast<uint4*>(base + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<uint4*>(base + (size_t)n16 * 64 + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
}

}  // namespace

int64_t glm_mma_image_elems(int64_t n) { return 2 * ((n + GM_CH - 1) / GM_CH * GM_CH) * GM_DK; }

cudaError_t build_glm_mma_image(const uint16_t* xh, const uint16_t* xl, int64_t n, int D, int Dp, uint16_t* img,
                                cudaStream_t s) {
    if (!xh || !xl || !img || n < 1 || n > (1 << 24) || D < 1 || D > GM_DK) return cudaErrorInvalidValue;
    const int n16 = (int)((n + GM_CH - 1) / GM_CH * GM_CH);
    const int items = n16 * 4;
    k_glm_mma_image<<<(items + 255) / 256, 256, 0, s>>>(xh, xl, (int)n, n16, D, Dp, img);
    return cudaGetLastError();
}

bool traj_glm_mma_supported(const DevModel& m, bool x3) {
    if (m.kind != LOGISTIC && m.kind != LINEAR_GAUSS) return false;
    if (m.D < 1 || m.D > GM_DK || m.n < 1 || !m.xmma_img) return false;
    return GmLayout(m.n, x3).bytes <= 220 * 1024;
}

cudaError_t launch_traj_glm_mma(const DevModel& m, const TrajArgs& a, bool x3, cudaStream_t s) {
    if (!traj_glm_mma_supported(m, x3)) return cudaErrorInvalidValue;
    if (m.kind == LOGISTIC) return x3 ? launch_gm<true, true>(m, a, s) : launch_gm<true, false>(m, a, s);
    return x3 ? launch_gm<false, true>(m, a, s) : launch_gm<false, false>(m, a, s);
}

}  // namespace smc
