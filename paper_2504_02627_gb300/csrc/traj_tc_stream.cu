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
// issues the MMAs, GEMM1 two chunks ahead of GEMM2 (three eta and three R
// buffers in flight), so the tensor core works while residuals are formed;
// warps 0-7 form the residuals r = y - sigmoid(eta) (or (y - eta)/sigma^2)
// from TMEM and write them back to TMEM as BF16, where GEMM2 reads its A
// operand (warps 0-3 the even chunks, 4-7 the odd ones), and they hold the
// particle state: warp w owns TMEM lanes 32 (w % 4) .. + 31 (one particle per
// lane) and dimensions 64 (w / 4) .. + 63.
// TMEM columns: eta [0, 192), G [192, 192 + dk), R^T [320, 512).  Every wait on
// an mbarrier is bounded (then *dev_err is set and the kernel still runs to
// its end) in wall time (2 s of %globaltimer per wait); a waiting thread polls
// with try_wait, which suspends it in hardware between polls, and reads the
// clock once per 64 polls, so it takes few issue slots from the epilogue.
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
constexpr int XK_BYTES = 2 * SC * 128;        // X chunk, K-major over dims: 2 atoms of 64 obs rows
constexpr int S_NB = 3;                       // eta and R^T buffers in flight (both in TMEM)
constexpr uint32_t S_TMEM_COLS = 512;
constexpr uint32_t S_COL_ETA = 0;             // S_NB eta buffers of 64 FP32 columns
constexpr uint32_t S_COL_G = 192;             // gradient accumulator, dk <= 128 columns
constexpr uint32_t S_COL_R = 320;             // S_NB x np R^T parts of 32 columns (64 BF16 obs)
constexpr int S_SMEM_MAX = 232448;            // opt-in shared memory per CTA

struct SLayout {
    int dkr, stages, xt_bytes, stage_bytes;
    int off_th, off_stage, off_y, off_misc, off_bar, total;
};

// Byte layout of the dynamic shared memory (from a 1024-aligned base).
__host__ __device__ inline SLayout s_layout(int dk, int np, int stages) {
    SLayout L;
    L.dkr = dk;                                   // dk is a multiple of 16: whole 8-row swizzle groups
    L.stages = stages;
    L.xt_bytes = L.dkr * 128;
    L.stage_bytes = XK_BYTES + L.xt_bytes;        // multiple of 1024
    L.off_th = 0;                                 // [np][2 atoms]
    L.off_stage = L.off_th + np * 2 * TH_ATOM;    // [stages]
    L.off_y = L.off_stage + stages * L.stage_bytes;   // [stages][64] f32
    L.off_misc = L.off_y + stages * SC * 4;       // kin, sq, ll: [2][128] f64 each
    L.off_bar = L.off_misc + 6 * SP * 8;          // mbarriers, TMEM base, flags
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

// Residual on the SFU's base-2 exponential and reciprocal in their flush-to-
// zero forms (a few ulp; the value is then split into BF16 parts with 2^-16
// relative resolution); e^-eta overflowing to +inf gives residual y.
template <bool LOGIT>
__device__ __forceinline__ float residual(float y, float eta, float inv_s2) {
    if (LOGIT) return y - tc::rcp_approx(1.0f + tc::ex2_approx(-1.4426950408889634f * eta));
    return (y - eta) * inv_s2;
}

// (a, b) -> BF16 pair hi (round to nearest even) and the BF16 pair of the
// remainders (a - hi, b - hi): one conversion per pair for each part.
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
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
    uint64_t* eta_full = empty + 4;                                  // [S_NB] GEMM1 done
    uint64_t* eta_empty = eta_full + S_NB;                           // [S_NB] eta read by the epilogue
    uint64_t* r_full = eta_empty + S_NB;                             // [S_NB] R^T written
    uint64_t* r_empty = r_full + S_NB;                               // [S_NB] GEMM2 done with R^T
    uint64_t* g_full = r_empty + S_NB;                               // step's gradient complete
    uint64_t* th_full = g_full + 1;                                  // next step's Theta^T written
    uint64_t* fin = th_full + 1;                                     // every MMA issued has completed
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(fin + 1);
    int* smax_s = reinterpret_cast<int*>(tmem_s + 1);
    volatile int* abort_s = smax_s + 1;                              // a bounded wait gave up
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
        for (int i = 0; i < S_NB; ++i) {
            tc::mbar_init(&eta_full[i], 1);
            tc::mbar_init(&eta_empty[i], S_EPI_WARPS / 2);   // one group of four warps per chunk
            tc::mbar_init(&r_full[i], S_EPI_WARPS / 2);
            tc::mbar_init(&r_empty[i], 1);
        }
        tc::mbar_init(g_full, 1);
        tc::mbar_init(th_full, S_EPI_WARPS);
        tc::mbar_init(fin, 1);
        tc::fence_mbar_init();
        *smax_s = 0;
        *abort_s = 0;
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
            // ring position (stage, its phase bit) and chunk, advanced without divisions
            int st = 0, c = 0;
            uint32_t ph = 0;
            for (int64_t it = 0; it < total; ++it) {
                tc::mbar_wait_timed(&empty[st], ph ^ 1u, err, abort_s);
                tc::mbar_arrive_expect_tx(&full[st], bytes);
                unsigned char* dst = sm + L.off_stage + st * L.stage_bytes;
                tc::bulk_g2s(dst, m.xk_img + (int64_t)c * (XK_BYTES / 2), XK_BYTES, &full[st]);
                tc::bulk_g2s(dst + XK_BYTES, m.xt_img + (int64_t)c * (L.xt_bytes / 2), (uint32_t)L.xt_bytes,
                             &full[st]);
                tc::bulk_g2s(y_s + st * SC, m.y_img + (int64_t)c * SC, SC * 4, &full[st]);
                if (++c == nch) c = 0;
                if (++st == stages) {
                    st = 0;
                    ph ^= 1u;
                }
            }
            // every copy has landed before the stage memory is reused or the CTA exits:
            // the last `stages` fills are the most recent phase of each stage
            const int64_t first = total > stages ? total - stages : 0;
            for (int64_t it = first; it < total; ++it) {
                const int sst = (int)(it % stages);
                tc::mbar_wait_timed(&full[sst], (uint32_t)((it / stages) & 1), err, abort_s);
            }
        }
    } else if (wid == S_MMA_WARP) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            // GEMM2 of one chunk: A = R^T from TMEM buffer b, B = the chunk's X image
            struct Pend { int st, b, ci; uint32_t bph; };
            auto gemm2 = [&](const Pend& q2) {
                tc::mbar_wait_timed(&r_full[q2.b], q2.bph, err, abort_s);
                tc::fence_after_sync();
                const uint32_t xt = s_base + L.off_stage + q2.st * L.stage_bytes + XK_BYTES;
                for (int q = 0; q < NP; ++q)
                    for (int kk = 0; kk < SC / 16; ++kk) {
                        const uint32_t at = tmem + S_COL_R + (uint32_t)((q2.b * NP + q) * 32 + kk * 8);
                        const uint64_t bd = tc::smem_desc(xt + kk * 32, 16, 1024, tc::SWZ_128B);
                        tc::mma_bf16_ta(tmem + S_COL_G, at, bd, IDESC2, (q2.ci > 0 || q > 0 || kk > 0) ? 1u : 0u);
                    }
                tc::mma_commit(&r_empty[q2.b]);
                tc::mma_commit(&empty[q2.st]);
            };
            int st = 0, b = 0;            // ring stage and buffer of the next chunk
            uint32_t ph = 0, bph = 0;     // their phase bits
            Pend p0{}, p1{};              // the two chunks whose GEMM2 is pending (oldest first)
            for (int s = 1; s <= nsteps; ++s) {
                if (s >= 2) tc::mbar_wait_timed(th_full, (uint32_t)((s - 2) & 1), err, abort_s);
                tc::fence_after_sync();
                for (int c = 0; c < nch; ++c) {
                    tc::mbar_wait_timed(&full[st], ph, err, abort_s);
                    tc::mbar_wait_timed(&eta_empty[b], bph ^ 1u, err, abort_s);
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
                    // GEMM2 two chunks behind: the stage ring holds chunks c-2 .. c (+ prefetch)
                    if (c >= 2) gemm2(p0);
                    p0 = p1;
                    p1 = Pend{st, b, c, bph};
                    if (++st == stages) {
                        st = 0;
                        ph ^= 1u;
                    }
                    if (++b == S_NB) {
                        b = 0;
                        bph ^= 1u;
                    }
                }
                if (nch >= 2) gemm2(p0);
                gemm2(p1);
                tc::mma_commit(g_full);
            }
            tc::mma_commit(fin);   // lets the CTA drain its MMAs even after an aborted wait
        }
    } else {
        // ------------------------------------------------------------ residuals and state (warps 0-7)
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        const float hf = 0.5f * ef;
        // Warps 0-3 take the even chunks of a step and warps 4-7 the odd ones
        // (all 64 observations of the chunk for their 32 particles), so one
        // group's TMEM load and store latencies overlap the other's arithmetic.
        // Every warp advances the ring counters for every chunk.
        int st = 0, b = 0;
        uint32_t sph = 0, bph = 0;
        for (int s = 1; s <= nsteps; ++s) {
            for (int c = 0; c < nch; ++c) {
                if ((c & 1) == dh) {
                    // one lane waits, the warp follows (__syncwarp orders the rest)
                    if (lane == 0) tc::mbar_wait_timed(&eta_full[b], bph, err, abort_s);
                    __syncwarp();
                    tc::fence_after_sync();
                    // the stage's y was written by the bulk copy: acquire its barrier
                    // phase (still current: the stage is refilled only after this
                    // chunk's GEMM2, which waits for these residuals)
                    if (lane == 0) tc::mbar_wait_timed(&full[st], sph, err, abort_s);
                    if (lane == 0) tc::mbar_wait_timed(&r_empty[b], bph ^ 1u, err, abort_s);
                    __syncwarp();
                    tc::fence_after_sync();
                    const uint32_t rcol = tmem + lane_base + S_COL_R + (uint32_t)(b * NP * 32);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float eta[32];
                        tc::tmem_ld32(tmem + lane_base + S_COL_ETA + b * SC + 32 * h, eta);
                        if (h == 1) {
                            tc::fence_before_sync();
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(&eta_empty[b]);
                        }
                        const float4* yv = reinterpret_cast<const float4*>(y_s + st * SC + 32 * h);
                        uint32_t rh[16], rl[16];
#pragma unroll
                        for (int e = 0; e < 32; e += 4) {
                            const float4 y4 = yv[e / 4];     // the same four y for every lane
                            const float r0 = residual<LOGIT>(y4.x, eta[e], inv_s2);
                            const float r1 = residual<LOGIT>(y4.y, eta[e + 1], inv_s2);
                            const float r2 = residual<LOGIT>(y4.z, eta[e + 2], inv_s2);
                            const float r3 = residual<LOGIT>(y4.w, eta[e + 3], inv_s2);
                            split_pair(r0, r1, rh[e / 2], rl[e / 2]);
                            split_pair(r2, r3, rh[e / 2 + 1], rl[e / 2 + 1]);
                        }
                        tc::tmem_st16(rcol + 16 * h, rh);
                        if (NP == 2) tc::tmem_st16(rcol + 32 + 16 * h, rl);
                    }
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&r_full[b]);
                }
                if (++st == stages) {
                    st = 0;
                    sph ^= 1u;
                }
                if (++b == S_NB) {
                    b = 0;
                    bph ^= 1u;
                }
            }
            // the step's gradient: G - theta / tau^2, then the leapfrog update
            tc::mbar_wait_timed(g_full, (uint32_t)((s - 1) & 1), err, abort_s);
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
    // eta = X theta in FP32 from the FP32 data (register tile of 8
    // observations x 4 particles per thread, X chunks double-buffered in
    // shared memory by cp.async), FP64 accumulation of the log-likelihood.
    // The whole dynamic shared memory is free again: all MMAs completed
    // (g_full, and fin even if a wait gave up) and every bulk copy landed
    // (the producer's drain).
    if (tid == 0) {
        volatile int ignore_abort = 0;   // this drain wait runs even after an abort
        tc::mbar_wait_timed(fin, 0u, err, &ignore_abort, 4000000000ull);
    }
    __syncthreads();
    const int Dp = m.Dp, n = m.n;
    float* thT = reinterpret_cast<float*>(sm + L.off_th);      // [dk][128]
    float* xs = thT + dk * SP;                                  // [2][SC][Dp]
    double* llp = reinterpret_cast<double*>(xs + 2 * SC * Dp);  // [8][128]
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
    auto issue_x = [&](int c, int buf) {
        const int64_t row0 = (int64_t)c * SC;
        const int64_t left = (int64_t)n - row0;
        const int rows = left < SC ? (int)left : SC;
        const int nvec = rows * Dp / 4;
        float* dst = xs + buf * SC * Dp;
        const float* srcx = m.X + row0 * Dp;
        for (int v = tid; v < nvec; v += S_THREADS) tc::cp_async16(dst + 4 * v, srcx + 4 * v);
        tc::cp_async_commit();
    };
    issue_x(0, 0);
    {
        const int pg = tid & 31, og = tid >> 5;     // warps 0-7 compute, 8-9 only copy
        double ll[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) issue_x(c + 1, (c + 1) & 1);
            else tc::cp_async_commit();             // keeps one group per iteration
            tc::cp_async_wait<1>();                 // chunk c has landed (this thread's copies)
            __syncthreads();                        // ... and everyone else's
            if (og < 8) {
                const float* xc = xs + (c & 1) * SC * Dp + og * 8 * Dp;
                float acc[8][4];
#pragma unroll
                for (int o = 0; o < 8; ++o)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[o][q] = 0.0f;
#pragma unroll 4
                for (int d = 0; d < D; ++d) {
                    const float4 t4 = *reinterpret_cast<const float4*>(thT + d * SP + 4 * pg);
#pragma unroll
                    for (int o = 0; o < 8; ++o) {
                        const float x = xc[o * Dp + d];
                        acc[o][0] = fmaf(x, t4.x, acc[o][0]);
                        acc[o][1] = fmaf(x, t4.y, acc[o][1]);
                        acc[o][2] = fmaf(x, t4.z, acc[o][2]);
                        acc[o][3] = fmaf(x, t4.w, acc[o][3]);
                    }
                }
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    const int64_t i = (int64_t)c * SC + og * 8 + o;
                    if (i < n) {
                        const float yv = __ldg(m.y + i);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float eta = acc[o][q];
                            float term;
                            if (LOGIT) {
                                const float sp = eta > 0.0f ? eta + log1pf(expf(-eta)) : log1pf(expf(eta));
                                term = yv * eta - sp;
                            } else {
                                const float z = (yv - eta) * inv_s;
                                term = -0.5f * z * z;
                            }
                            ll[q] += (double)term;
                        }
                    }
                }
            }
            __syncthreads();                        // buffer (c & 1) is refilled at iteration c + 1
        }
        if (og < 8)
#pragma unroll
            for (int q = 0; q < 4; ++q) llp[og * SP + 4 * pg + q] = ll[q];
        __syncthreads();
        if (tid < SP) {
            double tot = 0.0;
            for (int w = 0; w < 8; ++w) tot += llp[w * SP + tid];   // fixed order
            ll_s[tid] = tot;
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
            const double lp1 = ll_s[prow] - 0.5 * sq * inv_tau2_d + m.lconst;
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
    // three stages are in use at once (GEMM2 runs two chunks behind GEMM1); a
    // fourth lets the copy of the next chunk start early
    int stages = 4;
    while (stages > 3 && s_layout(m.dk, NP, stages).total > S_SMEM_MAX) --stages;
    const SLayout L = s_layout(m.dk, NP, stages);
    if (L.total > S_SMEM_MAX) return cudaErrorInvalidValue;
    // end-point staging (theta^T, two FP32 X chunks, partial sums) reuses [off_th, off_y)
    if ((int64_t)m.dk * SP * 4 + 2LL * SC * m.Dp * 4 + 8LL * SP * 8 > L.off_y) return cudaErrorInvalidValue;
    const int bytes = L.total;
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
