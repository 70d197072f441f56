// traj_centred.cu -- tensor-core (tcgen05) leapfrog trajectories for Bayesian
// logistic and linear-Gaussian regression in the centred precision form.
//
// Centring.  Before each move, every run gets a reference point theta_ref
// (the mean of its particles) and the per-observation reference quantities
// eta_ref = X theta_ref, s = sigmoid(eta_ref) and the reference gradient
// g_ref = X'(y - s) are evaluated once, with the FP32 data and FP64
// accumulation.  During the trajectory only the deviations are products on
// the tensor cores, in BF16 with FP32 accumulation:
//
//   GEMM1  d_eta^T [128 x 128 obs] = (theta - theta_ref)^T [128 x dk] . X_c^T
//   GEMM2  G^T     [128 x dk]     += d_r^T [128 x 128 obs] . X_c
//
// with d_r = s - sigmoid(eta_ref + d_eta) (logistic) or -d_eta / sigma^2
// (linear), and the gradient is g_ref + G - theta / tau^2.  Where particles
// sit near each other -- the posterior, after the first iterations -- the
// deviations are small, so one BF16 product per GEMM carries fewer rounding
// errors in absolute terms than a hi + lo split of the full theta and
// residual would.  The gradient is a fixed, deterministic function of theta
// within a move (theta_ref changes only between moves, and the kernel
// re-evaluates the gradient at the start point with the move's own
// reference rather than reusing the cached one), so each trajectory is a
// volume-preserving, reversible composition of shears; the end-point energy
// that enters the importance weight is recomputed with the FP32 data and
// FP64 accumulation, as in every other kernel.
//
// Layout.  One CTA holds 128 particles (MMA M = 128).  X streams through a
// ring of up to four stages (as many as fit in shared memory next to the
// deviations and the partial gradients) of 128-observation tiles:
// [atom][128 obs rows][128 B], an
// atom being 64 dimensions in the 128-byte swizzle.  GEMM1 reads a tile as its
// K-major B operand (rows = observations); GEMM2 reads the same bytes as an
// MN-major B operand (N = dimensions, K = observations: leading byte offset =
// the atom stride, stride byte offset = eight rows), so each observation is
// staged once per step for both products.  TMEM columns: G [0, 128), two eta
// buffers [128, 384), two d_r^T buffers (BF16 pairs) [384, 512); GEMM2 takes
// its A operand from TMEM.
//
// Roles (608 threads): warp 16 lane 0 issues the bulk copies; warp 17 lane 0
// issues GEMM1 and warp 18 lane 0 GEMM2, each from fully unrolled loops, so
// neither product waits behind the other's dependencies; warps 0-15 form the
// residuals from TMEM (warps 0-7 the even-numbered tiles of the pass
// sequence, 8-15 the odd ones, each group of four half of a tile's
// observations) and update the particle state, which lives in theta_out /
// p_out during the move.  A residual thread reads eta in the 16-lane shape
// (two observations of two particles per access) and writes the packed BF16
// residuals in the matching 16x128b shape, which is GEMM2's K order; it forms
// its two 16-lane groups one after the other (one group's eta live at a time),
// so one shared-memory load of an observation pair's reference values serves
// two particles.  The sigmoid's exponential is the SFU's base-2
// exponential; one SFU reciprocal of the product (1 + 2^x0)(1 + 2^x1) serves
// a pair of observations, and the pair's FMAs and adds run as packed FP32x2
// instructions.
//
// Clusters.  A tile's observations may be split over a cluster of k CTAs
// (k = 1, 2, 4 or 8, fixed by the tile count and the SM count, so that the
// long trajectories of a move, which sorting by step count gathers in the
// first tiles, spread over several SMs).  Every CTA of the cluster holds the
// same 128 particles and accumulates the partial gradient of its share of
// the observation tiles; each pass the partials are published in shared
// memory, and the CTA that owns an 8-dimension unit of the state sums the k
// partials of that unit in rank order (the same sum in every CTA), updates
// theta and p for the unit, and writes the unit's BF16 deviations into the
// GEMM1 operand of every CTA of the cluster through distributed shared
// memory.  The split changes only the FP32 summation order of the gradient.
// Every mbarrier wait is bounded in wall time (2 s), after which *dev_err is
// set and the kernel runs to its end without further waiting.
#include <cuda_bf16.h>
#include <math_constants.h>
#include "tc_ptx.cuh"
#include "traj.cuh"

namespace smc {
namespace {

constexpr int CP = 128;                     // particles per CTA
constexpr int CC = CENTRED_CHUNK;           // observations per tile
constexpr int C_EPI_WARPS = 16;
constexpr int C_PRODUCER_WARP = 16, C_MMA1_WARP = 17, C_MMA2_WARP = 18;
constexpr int C_THREADS = 32 * 19;
constexpr int C_NS_MAX = 4;                 // X tile stages (4 when shared memory allows, else 3 or 2)
constexpr int C_ATOM = CC * 128;            // one 64-dimension atom of a tile: 128 rows x 128 B
constexpr int C_DATOM = CP * 128;           // one 64-dimension atom of the deviation operand
constexpr uint32_t C_TMEM_COLS = 512;
constexpr uint32_t C_COL_G = 0, C_COL_ETA = 128, C_COL_R = 384;
constexpr int C_SMEM_MAX = 232448;
constexpr float C_X_MAX = 60.0f;           // clamp of the exponent: two factors 1 + 2^x multiply without overflow

struct CLayout {
    int atoms, tile_bytes, ref_bytes, stage_bytes, stages, xbufs;
    int off_d, off_stage, off_gx, off_emisc, off_cref, off_bar, total;
};

// Byte layout of the dynamic shared memory (from a 1024-aligned base) with
// `stages` X tile stages.  The end-point pass reuses [0, off_cref), the
// pipeline's memory, for theta^T, two FP32 X chunks, the partial sums and
// its kinetic / prior / likelihood parts, so off_cref covers both uses.
__host__ __device__ inline CLayout c_layout_n(int dk, int Dp, int n_ref, int n_run, int stages, int xbufs) {
    CLayout L;
    L.xbufs = xbufs;
    L.atoms = (dk + 63) / 64;
    L.tile_bytes = L.atoms * C_ATOM;
    L.ref_bytes = n_ref * CC * 8;                         // (c, s) pairs per run, a multiple of 1024
    L.stage_bytes = L.tile_bytes + L.ref_bytes;
    L.stages = stages;
    L.off_d = 0;
    L.off_stage = L.atoms * C_DATOM;
    L.off_gx = L.off_stage + stages * L.stage_bytes;     // [dk][128] f32 partial gradient of this CTA
    const int pipe = L.off_gx + dk * CP * 4;
    // the end point reuses the pipeline's memory: theta^T, one or two FP32
    // X chunks of CC observations and per-warp parts, then its kin, sq:
    // [4][128] f64 and ll: [128] f64 (the prologue keeps its kinetic parts in
    // the first stage, idle until the copies start)
    const int endp = dk * CP * 4 + xbufs * CC * Dp * 4 + C_EPI_WARPS * CP * 8;
    L.off_emisc = (endp + 1023) & ~1023;
    const int endx = L.off_emisc + 9 * CP * 8;
    L.off_cref = ((pipe > endx ? pipe : endx) + 1023) & ~1023;
    L.off_bar = L.off_cref + 2 * n_run * dk * 4;          // reference points, reference gradients [runs][dk]
    L.total = L.off_bar + 256 + 1024;                     // + alignment slack of the base
    // more than half of the SM's shared memory, so that a second CTA, which
    // would wait for the 512 TMEM columns, is never co-scheduled
    if (L.total < 118 * 1024) L.total = 118 * 1024;
    return L;
}
// The most X stages that fit (4, 3 or 2) with a double-buffered end point,
// else two stages with a single end-point buffer.
__host__ __device__ inline CLayout c_layout(int dk, int Dp, int n_ref, int n_run) {
    CLayout L = c_layout_n(dk, Dp, n_ref, n_run, C_NS_MAX, 2);
    for (int st = C_NS_MAX - 1; st >= 2 && L.total > C_SMEM_MAX; --st) L = c_layout_n(dk, Dp, n_ref, n_run, st, 2);
    if (L.total > C_SMEM_MAX) L = c_layout_n(dk, Dp, n_ref, n_run, 2, 1);
    return L;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Named hardware barrier of `count` threads (ids 1.. are free: 0 is __syncthreads).
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <bool LOGIT>
__global__ void __launch_bounds__(C_THREADS, 1) traj_centred_kernel(DevModel m, TrajArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-aligned base by pointer arithmetic on the shared array, so that
    // accesses through it stay shared-space loads and stores
    unsigned char* sm = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const CLayout L = c_layout(m.dk, m.Dp, LOGIT ? 1 : 0, a.c_runs);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int D = m.D, dk = m.dk, nch_all = m.n_tiles128;
    const int64_t ld = a.ld;
    // cluster split of the observation tiles: this CTA takes [c_lo, c_hi)
    const int kc = (int)a.c_split, rank = (int)tc::cluster_rank();
    const int64_t tile = blockIdx.x / kc;
    // the tile's run and first slot (run-uniform tiles), else the slots of perm in order
    int trun = 0;
    int64_t slot0 = tile * CP;
    if (a.c_tiles) {
        const int2 tt = a.c_tiles[tile];
        trun = tt.x;
        slot0 = tt.y;
    }
    const int c_lo = (int)((int64_t)rank * nch_all / kc), c_hi = (int)((int64_t)(rank + 1) * nch_all / kc);
    const int nch = c_hi - c_lo;
    // ownership of the state for the update: 8-dimension units, a contiguous share per rank
    const int nunit = dk / 8, u_lo = rank * nunit / kc, u_hi = (rank + 1) * nunit / kc;
    const int NS = L.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.off_bar);   // [NS] stage filled
    uint64_t* empty = full + C_NS_MAX;                               // [NS] stage consumed by both GEMMs
    uint64_t* eta_full = empty + C_NS_MAX;                           // [2] GEMM1 done
    uint64_t* eta_empty = eta_full + 2;                              // [2] eta read by the epilogue
    uint64_t* r_full = eta_empty + 2;                                // [2] d_r^T written
    uint64_t* r_empty = r_full + 2;                                  // [2] GEMM2 done with d_r^T
    uint64_t* g_full = r_empty + 2;                                  // pass's gradient complete
    uint64_t* th_full = g_full + 1;                                  // next pass's deviation operand written
    uint64_t* fin1 = th_full + 1;                                    // every GEMM1 issued has completed
    uint64_t* fin2 = fin1 + 1;                                       // every GEMM2 issued has completed
    uint64_t* gx_full = fin2 + 1;                                    // every CTA's partial gradient published
    uint64_t* gx_free = gx_full + 1;                                 // every CTA done reading this CTA's partial
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(gx_free + 1);
    int* smax_s = reinterpret_cast<int*>(tmem_s + 1);
    volatile int* abort_s = smax_s + 1;
    double* kin0_s = reinterpret_cast<double*>(sm + L.off_stage);    // prologue: [4][128] |p_0|^2 parts
    double* kin_s = reinterpret_cast<double*>(sm + L.off_emisc);     // end point: [4][128] |p|^2 parts
    double* sq_s = kin_s + 4 * CP;                                   // [4][128] |theta|^2 parts
    double* ll_s = sq_s + 4 * CP;                                    // [128] log-likelihood
    const uint32_t s_base = tc::smem_u32(sm);
    float* gx = reinterpret_cast<float*>(sm + L.off_gx);             // [dk][128] this CTA's partial gradient
    const uint32_t gx_base = s_base + (uint32_t)L.off_gx, dev_base = s_base + (uint32_t)L.off_d;
    int* err = a.dev_err;

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&eta_full[i], 1);
            tc::mbar_init(&eta_empty[i], 8);   // the two groups of four warps of the buffer
            tc::mbar_init(&r_full[i], 8);
            tc::mbar_init(&r_empty[i], 1);
        }
        tc::mbar_init(g_full, 1);
        tc::mbar_init(th_full, C_EPI_WARPS * kc);   // every epilogue warp of the cluster
        tc::mbar_init(fin1, 1);
        tc::mbar_init(fin2, 1);
        tc::mbar_init(gx_full, C_EPI_WARPS * kc);
        tc::mbar_init(gx_free, C_EPI_WARPS * kc);
        tc::fence_mbar_init();
        *smax_s = 0;
        *abort_s = 0;
    }
    if (wid == 0) {
        tc::tmem_alloc(tmem_s, C_TMEM_COLS);
        tc::tmem_relinquish();
    }
    // the runs' reference points and reference gradients, read every pass
    float* cref_s = reinterpret_cast<float*>(sm + L.off_cref);       // [runs][dk]
    float* gref_s = cref_s + a.c_runs * dk;                          // [runs][dk]
    for (int i = tid; i < a.c_runs * dk; i += C_THREADS) {
        cref_s[i] = a.c_centre[i];
        gref_s[i] = a.c_gref[i];
    }
    __syncthreads();

    // ---------------------------------------------------------------- particle state (warps 0-15)
    // warp w: TMEM lanes 32 (w % 4) .. + 31 (one particle per lane); group
    // q = w / 4 owns dimensions 32 q .. 32 q + 31 of those particles and, in
    // the tile loop, half (q % 2) of the observations of the tiles that use
    // buffer q / 2.  theta and p live in the slot-ordered buffers c_sth /
    // c_sp during the move (index: the slot), else in theta_out / p_out
    // (index: the particle).
    const bool epi = wid < C_EPI_WARPS;
    const int quarter = wid & 3, q = (wid >> 2) & 3;
    const int prow = 32 * quarter + lane;
    const int ds = 32 * q;                             // first state dimension of this thread
    const int bq = q >> 1, half = q & 1;
    const float inv_tau2 = LOGIT ? (float)(1.0 / (m.h0 * m.h0)) : (float)(1.0 / (m.h1 * m.h1));
    const double inv_tau2_d = LOGIT ? 1.0 / (m.h0 * m.h0) : 1.0 / (m.h1 * m.h1);
    const float inv_s2 = LOGIT ? 0.0f : (float)(1.0 / (m.h0 * m.h0));
    const float inv_s = LOGIT ? 0.0f : (float)(1.0 / m.h0);
    const bool evalm = a.eval_only != 0;
    const bool slotst = a.c_sth != nullptr && a.c_sp != nullptr && !evalm;
    float* const thb = slotst ? a.c_sth : a.theta_out;
    float* const pb = slotst ? a.c_sp : a.p_out;
    const int64_t sld = slotst ? a.c_sld : ld;           // stride of thb / pb
    int64_t j = -1, src = -1;
    int S = 0, run = 0;
    float ef = 0.0f;
    float th[32];
    {
        const int64_t t = slot0 + prow;
        double kin = 0.0;
        int64_t jt = -1;
        if (a.c_tiles) jt = a.c_perm[t];                     // -1 in a pad slot
        else if (t < a.N) jt = a.perm ? a.perm[t] : t;
        if (epi && jt >= 0) {
            j = jt;
            src = a.src ? a.src[j] : j;
            S = evalm ? 0 : a.steps[j];
            double eps;
            uint64_t seed;
            uint32_t kk, jl;
            particle_run(a, j, run, eps, seed, kk, jl);
            ef = (float)eps;
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
                const int d = ds + i;
                float tv[2] = {0.0f, 0.0f}, pv[2] = {0.0f, 0.0f};
                if (d < D) {
                    tv[0] = a.theta_in[(int64_t)d * ld + src];
                    if (d + 1 < D) tv[1] = a.theta_in[(int64_t)(d + 1) * ld + src];
                    if (!evalm) {
                        // momentum (given, or Philox + Box-Muller); the first half
                        // kick waits for the gradient of pass 0
                        if (a.p_in) {
                            pv[0] = a.p_in[(int64_t)d * ld + j];
                            if (d + 1 < D) pv[1] = a.p_in[(int64_t)(d + 1) * ld + j];
                        } else {
                            double z0, z1;
                            normal_pair(seed, (uint32_t)(d >> 1), jl, kk, TAG_MOM, z0, z1);
                            pv[0] = (float)z0;
                            pv[1] = d + 1 < D ? (float)z1 : 0.0f;
                        }
                        const bool own = (d >> 3) >= u_lo && (d >> 3) < u_hi;
#pragma unroll
                        for (int e = 0; e < 2; ++e)
                            if (d + e < D) {
                                kin += (double)pv[e] * (double)pv[e];
                                if (own) {
                                    pb[(int64_t)(d + e) * sld + (slotst ? t : j)] = pv[e];
                                    thb[(int64_t)(d + e) * sld + (slotst ? t : j)] = tv[e];
                                }
                            }
                    }
                }
                th[i] = tv[0];
                th[i + 1] = tv[1];
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) th[i] = 0.0f;
        }
        if (epi) kin0_s[q * CP + prow] = kin;
    }
    const float* cref = cref_s + run * dk;                // this particle's run reference point
    const int64_t si = slotst ? slot0 + prow : j;         // index of this thread's state in thb / pb
    // deviation operand: unit u (8 dimensions) of this thread's 32 dimensions
    // of its particle row, BF16, swizzled
    auto write_unit = [&](int u, const float* tv) {
        unsigned char* row = sm + L.off_d + (q >> 1) * C_DATOM + prow * 128;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int d = ds + 8 * u + e;
            v[e] = (j >= 0 && d < D) ? tv[e] - cref[d] : 0.0f;
        }
        const uint4 w = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                   pack_bf16(v[6], v[7]));
        const int unit = 4 * (q & 1) + u;
        *reinterpret_cast<uint4*>(row + ((unit ^ (prow & 7)) << 4)) = w;
    };
    auto write_dev = [&](const float (&tv)[32]) {
        if (ds >= dk) return;
#pragma unroll
        for (int u = 0; u < 4; ++u) write_unit(u, tv + 8 * u);
    };
    if (epi) write_dev(th);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (epi && S > 0) atomicMax(smax_s, S);
    tc::cluster_sync();   // barriers of every CTA of the cluster initialised before any remote arrive
    double H0 = 0.0;
    if (epi && q == 0 && j >= 0 && !evalm)
        H0 = 0.5 * (kin0_s[prow] + kin0_s[CP + prow] + kin0_s[2 * CP + prow] + kin0_s[3 * CP + prow]) -
             a.logpi_in[src];
    __syncthreads();
    const uint32_t tmem = *tmem_s;
    const int smax = *smax_s;
    const int npass = evalm ? 1 : smax + 1;   // pass 0: gradient at the start point

    const int ksteps1 = dk / 16;
    const int64_t total = (int64_t)npass * nch;

    if (wid == C_PRODUCER_WARP) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)(L.tile_bytes + L.ref_bytes);
            int st = 0, c = c_lo;
            uint32_t ph = 0;
            for (int64_t it = 0; it < total; ++it) {
                tc::mbar_wait_timed(&empty[st], ph ^ 1u, err, abort_s);
                tc::mbar_arrive_expect_tx(&full[st], bytes);
                unsigned char* dst = sm + L.off_stage + st * L.stage_bytes;
                tc::bulk_g2s(dst, m.xc_img + (int64_t)c * (L.tile_bytes / 2), (uint32_t)L.tile_bytes, &full[st]);
                if (L.ref_bytes > 0)
                    tc::bulk_g2s(dst + L.tile_bytes, a.c_refs + ((int64_t)c * a.c_runs + trun) * CC, (uint32_t)L.ref_bytes,
                                 &full[st]);
                if (++c == c_hi) c = c_lo;
                if (++st == NS) {
                    st = 0;
                    ph ^= 1u;
                }
            }
            // every copy has landed before the stage memory is reused or the CTA exits
            const int64_t first = total > NS ? total - NS : 0;
            for (int64_t it = first; it < total; ++it)
                tc::mbar_wait_timed(&full[(int)(it % NS)], (uint32_t)((it / NS) & 1), err, abort_s);
        }
    } else if (wid == C_MMA1_WARP) {
        // ------------------------------------------------------------ GEMM1: d_eta = dev . X_c^T
        if (lane == 0) {
            const uint32_t IDESC1 = tc::idesc_bf16_f32(CP, CC);
            int st = 0, b = 0;
            uint32_t ph = 0, bph = 0;
            for (int s = 0; s < npass; ++s) {
                if (s >= 1) tc::mbar_wait_cluster_timed(th_full, (uint32_t)((s - 1) & 1), err, abort_s);
                for (int c = c_lo; c < c_hi; ++c) {
                    tc::mbar_wait_timed(&full[st], ph, err, abort_s);
                    tc::mbar_wait_timed(&eta_empty[b], bph ^ 1u, err, abort_s);
                    tc::fence_after_sync();
                    const uint32_t xt = s_base + L.off_stage + st * L.stage_bytes;
                    const uint32_t dcol = tmem + C_COL_ETA + (uint32_t)(b * CC);
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        if (kk < ksteps1) {
                            const int atom = kk >> 2, ko = (kk & 3) * 32;
                            const uint64_t ad = tc::smem_desc(s_base + L.off_d + atom * C_DATOM + ko, 16, 1024,
                                                              tc::SWZ_128B);
                            const uint64_t bd = tc::smem_desc(xt + atom * C_ATOM + ko, 16, 1024, tc::SWZ_128B);
                            tc::mma_bf16(dcol, ad, bd, IDESC1, kk > 0 ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(&eta_full[b]);
                    if (++st == NS) {
                        st = 0;
                        ph ^= 1u;
                    }
                    if (++b == 2) {
                        b = 0;
                        bph ^= 1u;
                    }
                }
            }
            tc::mma_commit(fin1);
        }
    } else if (wid == C_MMA2_WARP) {
        // ------------------------------------------------------------ GEMM2: G += d_r^T . X_c
        if (lane == 0) {
            const uint32_t IDESC2 = tc::idesc_bf16_f32(CP, (uint32_t)dk) | (1u << 16);   // B MN-major
            int st = 0, b = 0;
            uint32_t ph = 0, bph = 0;
            for (int s = 0; s < npass; ++s) {
                for (int c = c_lo; c < c_hi; ++c) {
                    tc::mbar_wait_timed(&full[st], ph, err, abort_s);
                    tc::mbar_wait_timed(&r_full[b], bph, err, abort_s);
                    tc::fence_after_sync();
                    const uint32_t xt = s_base + L.off_stage + st * L.stage_bytes;
                    const uint32_t acol = tmem + C_COL_R + (uint32_t)(b * (CC / 2));
#pragma unroll
                    for (int kk = 0; kk < CC / 16; ++kk) {
                        const uint64_t bd = tc::smem_desc(xt + kk * 2048, C_ATOM, 1024, tc::SWZ_128B);
                        tc::mma_bf16_ta(tmem + C_COL_G, acol + (uint32_t)(kk * 8), bd, IDESC2,
                                        (c > c_lo || kk > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(&r_empty[b]);
                    tc::mma_commit(&empty[st]);
                    if (c == c_hi - 1) tc::mma_commit(g_full);
                    if (++st == NS) {
                        st = 0;
                        ph ^= 1u;
                    }
                    if (++b == 2) {
                        b = 0;
                        bph ^= 1u;
                    }
                }
            }
            tc::mma_commit(fin2);
        }
    } else {
        // ------------------------------------------------------------ residuals and state (warps 0-15)
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        const float hf = 0.5f * ef;
        const float kneg = -1.4426950408889634f;
        const float* gref = gref_s + run * dk;
        // a residual thread's observation pairs: 8 mm + 2 tig (+1)
        const int tig = lane & 3;
        int st = 0;
        uint32_t sph = 0, bph = 0;
        int64_t it = 0;
        for (int s = 0; s < npass; ++s) {
            for (int c = c_lo; c < c_hi; ++c, ++it) {
                if ((int)(it & 1) == bq) {
                    // one thread of the buffer's eight warps waits for the tile;
                    // the others sleep on a hardware barrier instead of polling
                    if (lane == 0 && (wid & 7) == 0) {
                        tc::mbar_wait_timed(&eta_full[bq], bph, err, abort_s);
                        tc::mbar_wait_timed(&full[st], sph, err, abort_s);
                    }
                    named_sync(1u + (uint32_t)bq, 256u);
                    tc::fence_after_sync();
                    const uint32_t ecol = tmem + lane_base + C_COL_ETA + (uint32_t)(bq * CC + 64 * half);
                    const uint32_t rcol = tmem + lane_base + C_COL_R + (uint32_t)(bq * (CC / 2) + 32 * half);
                    const unsigned char* refs0 =
                        sm + L.off_stage + st * L.stage_bytes + L.tile_bytes + half * (64 * 8);
                    // One SFU reciprocal serves both observations of a pair:
                    // 1 / q0 = q1 / (q0 q1), 1 / q1 = q0 / (q0 q1), with the
                    // exponents clamped so that q0 q1 < 2^121 (a sigmoid below
                    // 2^-60 is then taken as 2^-60, i.e. zero here).  cs holds
                    // the pair's (c0, c1, s0, s1); the exponents, 1 + 2^x and
                    // the residuals are packed pair operations (each lane
                    // rounded as its scalar form), the sum taken as (q1, q0)
                    // so that it multiplies -1 / (q0 q1) into (r0, r1) as is.
                    auto res_pair = [&](uint32_t e0, uint32_t e1, const float4& cs) -> uint32_t {
                        const float v0f = __uint_as_float(e0), v1f = __uint_as_float(e1);
                        float r0, r1;
                        if (LOGIT) {
                            float x0, x1;
                            tc::f32x2_unpack(tc::f32x2_fma(tc::f32x2_pack(kneg, kneg), tc::f32x2_pack(v0f, v1f),
                                                           tc::f32x2_pack(cs.x, cs.y)),
                                             x0, x1);
                            x0 = fminf(x0, C_X_MAX);
                            x1 = fminf(x1, C_X_MAX);
                            const uint64_t q10 = tc::f32x2_add(
                                tc::f32x2_pack(tc::ex2_approx(x1), tc::ex2_approx(x0)), tc::f32x2_pack(1.0f, 1.0f));
                            float q1, q0;
                            tc::f32x2_unpack(q10, q1, q0);
                            const float rp = tc::rcp_approx(q0 * q1);
                            tc::f32x2_unpack(tc::f32x2_fma(q10, tc::f32x2_pack(-rp, -rp), tc::f32x2_pack(cs.z, cs.w)),
                                             r0, r1);
                        } else {
                            r0 = -inv_s2 * v0f;
                            r1 = -inv_s2 * v1f;
                        }
                        return pack_bf16(r0, r1);
                    };
                    // this thread forms the residuals of the quarter's lanes
                    // g4, g4 + 8 (first group) and g4 + 16, g4 + 24 (second)
                    // for the observation pairs 8 mm + 2 tig (+1), mm = 0..7,
                    // of the half: one (c0, c1, s0, s1) load serves two
                    // observations of two particles.  Each observation pair's packed residuals
                    // overwrite already consumed registers: v[2 mm] (lane g4 or
                    // g4 + 16) and v[2 mm + 1] (lane + 8), the order of the
                    // 16x128b store.
                    // every particle of the tile belongs to the tile's run,
                    // whose (c, s) pairs are the stage's only ones
                    const float4* f = reinterpret_cast<const float4*>(refs0);
                    auto form = [&](uint32_t (&v)[32]) {
#pragma unroll
                        for (int mm = 0; mm < 8; ++mm) {
                            const float4 cs = LOGIT ? f[4 * mm + tig] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                            const uint32_t a0 = res_pair(v[4 * mm], v[4 * mm + 1], cs);
                            const uint32_t a1 = res_pair(v[4 * mm + 2], v[4 * mm + 3], cs);
                            v[2 * mm] = a0;
                            v[2 * mm + 1] = a1;
                        }
                    };
                    // The two groups go one after the other, so that only one
                    // group's eta is live at a time (no register spills); the
                    // second group's load overlaps the first group's store,
                    // and the eta buffer is released once both are read.
                    uint32_t va[32], vb[32];
                    tc::tmem_ld16x256_x8_nowait(ecol, va);
                    tc::tmem_wait_ld();
                    form(va);
                    // the buffer's previous residuals have been read by GEMM2
                    if (lane == 0) tc::mbar_wait_timed(&r_empty[bq], bph ^ 1u, err, abort_s);
                    __syncwarp();
                    tc::fence_after_sync();
                    tc::tmem_st16x128_x8_nowait(rcol, va);
                    tc::tmem_ld16x256_x8_nowait(ecol + (16u << 16), vb);
                    tc::tmem_wait_ld();
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&eta_empty[bq]);
                    form(vb);
                    tc::tmem_st16x128_x8_nowait(rcol + (16u << 16), vb);
                    tc::tmem_wait_st();
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&r_full[bq]);
                    bph ^= 1u;   // the next use of buffer bq is its next phase
                }
                if (++st == NS) {
                    st = 0;
                    sph ^= 1u;
                }
            }
            // the pass's gradient g_ref + (sum of the cluster's partial G) -
            // theta / tau^2, then the leapfrog update of the units this CTA owns
            // one thread waits for the pass's gradient (and for every CTA to be
            // done with the previous pass's partials); the other epilogue
            // warps sleep on a hardware barrier instead of polling
            if (tid == 0) {
                tc::mbar_wait_timed(g_full, (uint32_t)(s & 1), err, abort_s);
                if (kc > 1 && s >= 1) tc::mbar_wait_cluster_timed(gx_free, (uint32_t)((s - 1) & 1), err, abort_s);
            }
            named_sync(3u, 32u * C_EPI_WARPS);
            tc::fence_after_sync();
            if (kc > 1) {
                // publish this CTA's partial gradient (dims ds .. ds + 31 below
                // dk: with dk = 112 the last group holds only 16 rows of gx);
                // a CTA alone reads its own units from TMEM instead
                if (ds < dk) {
                    uint32_t gv[32];
                    tc::tmem_ld32_nowait(tmem + lane_base + C_COL_G + ds, gv);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        if (ds + e < dk) gx[(ds + e) * CP + prow] = __uint_as_float(gv[e]);
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0)
                    for (int r = 0; r < kc; ++r)
                        tc::mbar_arrive_cluster(tc::map_to_rank(tc::smem_u32(gx_full), (uint32_t)r));
                if (tid == 0) tc::mbar_wait_cluster_timed(gx_full, (uint32_t)(s & 1), err, abort_s);
                named_sync(3u, 32u * C_EPI_WARPS);
            }
            const bool live = j >= 0 && (evalm || s <= S);
            const bool more = s + 1 < npass;
            // the update of the units this CTA owns, spread over all sixteen
            // warps: group q takes units q, q + 4, q + 8, q + 12 of its particle
#pragma unroll
            for (int uu = 0; uu < 4; ++uu) {
                const int unit = q + 4 * uu;
                if (unit >= nunit || unit < u_lo || unit >= u_hi) continue;
                // every load of the unit is issued before its first store (the
                // state arrays may alias as far as the compiler knows)
                float gs[8], tcur[8], pcur[8];
                if (kc == 1) {
                    // the unit's eight gradient columns of this thread's
                    // particle (its warp's TMEM lane quarter)
                    uint32_t gv[8];
                    tc::tmem_ld8_nowait(tmem + lane_base + C_COL_G + (uint32_t)(8 * unit), gv);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 8; ++e) gs[e] = __uint_as_float(gv[e]);
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        // the cluster's partials of this dimension, summed in rank order
                        const uint32_t ga = gx_base + (uint32_t)(((8 * unit + e) * CP + prow) * 4);
                        gs[e] = tc::ld_cluster_f32(tc::map_to_rank(ga, 0u));
                    }
                    // each rank's eight values are all requested before the
                    // first is added, so a rank costs one round trip
                    for (int r = 1; r < kc; ++r) {
                        float v[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            v[e] = tc::ld_cluster_f32(
                                tc::map_to_rank(gx_base + (uint32_t)(((8 * unit + e) * CP + prow) * 4), (uint32_t)r));
#pragma unroll
                        for (int e = 0; e < 8; ++e) gs[e] += v[e];
                    }
                }
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int d = 8 * unit + e;
                    tcur[e] = 0.0f;
                    pcur[e] = 0.0f;
                    if (live && d < D) {
                        tcur[e] = evalm ? a.theta_in[(int64_t)d * ld + src] : thb[(int64_t)d * sld + si];
                        if (!evalm) pcur[e] = pb[(int64_t)d * sld + si];
                    }
                }
                float tv[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int d = 8 * unit + e;
                    float tnew = 0.0f;
                    if (live && d < D) {
                        float t0 = tcur[e];
                        const float g = gref[d] + gs[e] - t0 * inv_tau2;
                        if (evalm || s == S) a.grad_out[(int64_t)d * ld + j] = g;
                        if (!evalm) {
                            float pv = pcur[e];
                            if (s >= 1) pv = fmaf(hf, g, pv);
                            if (s < S) {
                                pv = fmaf(hf, g, pv);
                                t0 = fmaf(ef, pv, t0);
                                thb[(int64_t)d * sld + si] = t0;
                            }
                            pb[(int64_t)d * sld + si] = pv;
                        }
                        tnew = t0;
                    }
                    tv[e] = tnew;
                }
                if (more) {
                    // the unit's 16 bytes of the deviation row, into the GEMM1
                    // operand of every CTA of the cluster
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int d = 8 * unit + e;
                        v[e] = (j >= 0 && d < D) ? tv[e] - cref[d] : 0.0f;
                    }
                    const uint4 w = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                               pack_bf16(v[6], v[7]));
                    const uint32_t uoff =
                        (uint32_t)((unit >> 3) * C_DATOM + prow * 128 + (((unit & 7) ^ (prow & 7)) << 4));
                    if (kc == 1) {
                        *reinterpret_cast<uint4*>(sm + L.off_d + uoff) = w;
                    } else {
                        for (int r = 0; r < kc; ++r) tc::st_cluster_u4(tc::map_to_rank(dev_base + uoff, (uint32_t)r), w);
                    }
                }
            }
            // the deviations reach the other CTAs' tensor cores, and this CTA
            // is done with the cluster's partials
            if (kc == 1) tc::fence_proxy_async_smem();
            else tc::fence_proxy_async_cluster();
            __syncwarp();
            if (lane == 0)
                for (int r = 0; r < kc; ++r) {
                    if (more) tc::mbar_arrive_cluster(tc::map_to_rank(tc::smem_u32(th_full), (uint32_t)r));
                    if (kc > 1) tc::mbar_arrive_cluster(tc::map_to_rank(tc::smem_u32(gx_free), (uint32_t)r));
                }
        }
    }

    // ---------------------------------------------------------------- end point energy
    // eta = X theta in FP32 from the FP32 data (register tile of 4
    // observations x 4 particles per thread, X chunks double-buffered in
    // shared memory by cp.async), a thread's four terms of a particle summed in
    // FP32, then FP64 accumulation of the log-likelihood.
    if (tid == 0) {
        volatile int ignore_abort = 0;   // these drain waits run even after an abort
        tc::mbar_wait_timed(fin1, 0u, err, &ignore_abort, 4000000000ull);
        tc::mbar_wait_timed(fin2, 0u, err, &ignore_abort, 4000000000ull);
    }
    __syncthreads();
    tc::cluster_sync();   // every CTA of the cluster has written its units of the final state
    const int Dp = m.Dp, n = m.n;
    // this CTA's share of the CC-observation chunks of the end point (the
    // same split as its X tiles)
    const int e_lo = c_lo, e_hi = c_hi;
    const int XB = L.xbufs;
    float* thT = reinterpret_cast<float*>(sm);                  // [dk][128]
    float* xs = thT + dk * CP;                                  // [XB][CC][Dp]
    double* llp = reinterpret_cast<double*>(xs + XB * CC * Dp);   // [16][128]
    if (epi) {
        double sq = 0.0, kin = 0.0;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            const int d = ds + e;
            float tvv = 0.0f;
            if (j >= 0 && d < D) {
                tvv = evalm ? a.theta_in[(int64_t)d * ld + src] : thb[(int64_t)d * sld + si];
                if (!evalm) {
                    const float pvf = pb[(int64_t)d * sld + si];
                    const double pv = pvf;
                    kin += pv * pv;
                    // the final state from the slot-ordered buffers to the
                    // particle's outputs, by the CTA that owns the unit
                    if (slotst && (d >> 3) >= u_lo && (d >> 3) < u_hi) {
                        a.theta_out[(int64_t)d * ld + j] = tvv;
                        a.p_out[(int64_t)d * ld + j] = pvf;
                    }
                }
            }
            if (d < dk) thT[d * CP + prow] = tvv;
            sq += (double)tvv * (double)tvv;
        }
        sq_s[q * CP + prow] = sq;
        kin_s[q * CP + prow] = kin;
    }
    auto issue_x = [&](int c, int buf) {
        const int64_t row0 = (int64_t)c * CC;
        const int64_t left = (int64_t)n - row0;
        const int rows = left < CC ? (int)left : CC;
        const int nvec = rows * Dp / 4;
        float* dst = xs + buf * CC * Dp;
        const float* srcx = m.X + row0 * Dp;
        for (int v = tid; v < nvec; v += C_THREADS) tc::cp_async16(dst + 4 * v, srcx + 4 * v);
        tc::cp_async_commit();
    };
    if (e_lo < e_hi) issue_x(e_lo, 0);
    {
        // warps 0-15 compute 8 observations each for 4 particles per lane
        // (a register tile of 8 x 4: every theta^T load serves 8
        // observations), warps 16-18 only copy
        const int pg = lane, og = wid;
        double ll[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = e_lo; c < e_hi; ++c) {
            const int buf = (c - e_lo) % XB;
            if (XB == 2) {
                if (c + 1 < e_hi) issue_x(c + 1, buf ^ 1);
                else tc::cp_async_commit();
                tc::cp_async_wait<1>();
            } else {
                tc::cp_async_wait<0>();
            }
            __syncthreads();
            if (og < C_EPI_WARPS) {
                const float* xc = xs + buf * CC * Dp + og * 8 * Dp;
                float acc[8][4];
#pragma unroll
                for (int o = 0; o < 8; ++o)
#pragma unroll
                    for (int k = 0; k < 4; ++k) acc[o][k] = 0.0f;
                // four dimensions per iteration: X rows as float4 (Dp is a
                // multiple of 4 and zero-padded; theta^T rows past D are zero)
                const float* tcol = thT + 4 * pg;
                for (int d = 0; d < Dp; d += 4) {
                    float4 xv[8];
#pragma unroll
                    for (int o = 0; o < 8; ++o) xv[o] = *reinterpret_cast<const float4*>(xc + o * Dp + d);
#pragma unroll
                    for (int dd = 0; dd < 4; ++dd) {
                        const float4 t4 = *reinterpret_cast<const float4*>(tcol + (d + dd) * CP);
#pragma unroll
                        for (int o = 0; o < 8; ++o) {
                            const float x = dd == 0 ? xv[o].x : dd == 1 ? xv[o].y : dd == 2 ? xv[o].z : xv[o].w;
                            acc[o][0] = fmaf(x, t4.x, acc[o][0]);
                            acc[o][1] = fmaf(x, t4.y, acc[o][1]);
                            acc[o][2] = fmaf(x, t4.z, acc[o][2]);
                            acc[o][3] = fmaf(x, t4.w, acc[o][3]);
                        }
                    }
                }
                float part[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    const int64_t i = (int64_t)c * CC + og * 8 + o;
                    if (i < n) {
                        const float yv = __ldg(m.y + i);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float eta = acc[o][k];
                            float term;
                            if (LOGIT) {
                                const float sp = eta > 0.0f ? eta + log1pf(expf(-eta)) : log1pf(expf(eta));
                                term = yv * eta - sp;
                            } else {
                                const float z = (yv - eta) * inv_s;
                                term = -0.5f * z * z;
                            }
                            part[k] += term;
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) ll[k] += (double)part[k];
            }
            __syncthreads();
            if (XB == 1 && c + 1 < e_hi) issue_x(c + 1, 0);
        }
        if (og < C_EPI_WARPS)
#pragma unroll
            for (int k = 0; k < 4; ++k) llp[og * CP + 4 * pg + k] = ll[k];
        __syncthreads();
        if (tid < CP) {
            double tot = 0.0;
            for (int w = 0; w < C_EPI_WARPS; ++w) tot += llp[w * CP + tid];   // fixed order
            ll_s[tid] = tot;
        }
    }
    __syncthreads();
    tc::cluster_sync();   // every CTA's log-likelihood part is in its shared memory
    if (rank == 0 && epi && q == 0 && j >= 0) {
        // the cluster's parts, summed in rank order
        const uint32_t la = tc::smem_u32(ll_s + prow);
        double llsum = tc::ld_cluster_f64(tc::map_to_rank(la, 0u));
        for (int r = 1; r < kc; ++r) llsum += tc::ld_cluster_f64(tc::map_to_rank(la, (uint32_t)r));
        const double sq = sq_s[prow] + sq_s[CP + prow] + sq_s[2 * CP + prow] + sq_s[3 * CP + prow];
        const double lp1 = llsum - 0.5 * sq * inv_tau2_d + m.lconst;
        a.logpi_out[j] = lp1;
        if (!evalm) {
            const double kin = kin_s[prow] + kin_s[CP + prow] + kin_s[2 * CP + prow] + kin_s[3 * CP + prow];
            double dH = (0.5 * kin - lp1) - H0;
            if (!isfinite(dH)) dH = CUDART_INF;
            if (a.dH) a.dH[j] = dH;
            if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
        }
    }
    tc::fence_before_sync();
    tc::cluster_sync();   // no CTA leaves while another may still read its shared memory
    tc::fence_after_sync();
    if (wid == 0) tc::tmem_dealloc(tmem, C_TMEM_COLS);
}

// ---------------------------------------------------------------- reference point and quantities
// Run r of the launch: particles [off, off + n) (the whole launch when the
// launch has no run table).
__device__ __forceinline__ void run_range(const TrajArgs& a, int r, int64_t& off, int64_t& cnt) {
    if (a.runs) {
        off = a.runs[r].off;
        cnt = a.runs[r].n;
    } else {
        off = 0;
        cnt = a.N;
    }
}

// theta_ref[r][d] = mean over the run's particles (after resampling: through
// src) of theta[d]; zero for the padding dimensions D <= d < dk.
__global__ void __launch_bounds__(256) k_centre_mean(TrajArgs a, int D, int dk) {
    __shared__ double red[256];
    const int r = blockIdx.x, d = blockIdx.y;
    int64_t off, cnt;
    run_range(a, r, off, cnt);
    double sum = 0.0;
    if (d < D)
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int64_t jj = off + i;
            const int64_t sj = a.src ? a.src[jj] : jj;
            sum += (double)a.theta_in[(int64_t)d * a.ld + sj];
        }
    red[threadIdx.x] = sum;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.c_centre[(int64_t)r * dk + d] = (d < D && cnt > 0) ? (float)(red[0] / (double)cnt) : 0.0f;
}

// Per 128-observation tile: eta_ref = X theta_ref (FP32 data, FP64 sums), the
// tile's (c, s) pairs c = -log2(e) eta_ref, s = sigmoid(eta_ref) for the
// logistic model, and the tile's part of g_ref = X'(y - s) (logistic, with the
// FP32 s the kernel subtracts from) or X'(y - eta_ref) / sigma^2 (linear).
template <bool LOGIT>
__global__ void __launch_bounds__(128) k_centre_obs(DevModel m, TrajArgs a) {
    __shared__ double rr[CC];
    const int c = blockIdx.x, t = threadIdx.x;
    const int64_t i = (int64_t)c * CC + t;
    const int D = m.D, dk = m.dk, Dp = m.Dp, R = a.c_runs;
    for (int r = 0; r < R; ++r) {
        const float* cr = a.c_centre + (int64_t)r * dk;
        double res = 0.0;
        float2 cs = make_float2(0.0f, 0.5f);
        if (i < m.n) {
            double eta = 0.0;
            for (int d = 0; d < D; ++d) eta += (double)m.X[i * Dp + d] * (double)cr[d];
            if (LOGIT) {
                const float s = (float)(1.0 / (1.0 + exp(-eta)));
                cs = make_float2((float)(-1.4426950408889634 * eta), s);
                res = (double)m.y[i] - (double)s;
            } else {
                res = ((double)m.y[i] - eta) / (m.h0 * m.h0);
            }
        }
        if (LOGIT) {
            // an observation pair's values as (c0, c1, s0, s1): the
            // epilogue's packed FMAs take each pair from adjacent registers
            float* fr = reinterpret_cast<float*>(a.c_refs + ((int64_t)c * R + r) * CC);
            fr[4 * (t >> 1) + (t & 1)] = cs.x;
            fr[4 * (t >> 1) + 2 + (t & 1)] = cs.y;
        }
        rr[t] = res;
        __syncthreads();
        if (t < dk) {
            double g = 0.0;
            if (t < D) {
                const int rows = (int)((int64_t)m.n - (int64_t)c * CC < CC ? (int64_t)m.n - (int64_t)c * CC : CC);
                for (int o = 0; o < rows; ++o) g += (double)m.X[((int64_t)c * CC + o) * Dp + t] * rr[o];
            }
            a.c_part[((int64_t)c * R + r) * dk + t] = g;
        }
        __syncthreads();
    }
}

// Run-uniform tiles (several runs): a stable partition of the launch's
// particles, in the order of perm, by run.  Counts per 1024-slot block, their
// exclusive scan over the blocks for every run (from the run's first slot),
// then each particle's slot: its block's base + the counts of its run in the
// earlier warps of the block + its rank among the warp's lanes of that run.
__global__ void __launch_bounds__(1024) k_part_count(TrajArgs a) {
    __shared__ int cnt[CENTRED_MAX_RUNS];
    const int R = a.c_runs;
    if ((int)threadIdx.x < R) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    if (t < a.N) {
        const int64_t j = a.perm ? a.perm[t] : t;
        atomicAdd(&cnt[a.run_of ? a.run_of[j] : 0], 1);
    }
    __syncthreads();
    if ((int)threadIdx.x < R) a.c_pcnt[(int64_t)blockIdx.x * R + threadIdx.x] = cnt[threadIdx.x];
}
__global__ void __launch_bounds__(32 * CENTRED_MAX_RUNS) k_part_scan(TrajArgs a, int64_t nblk) {
    const int R = a.c_runs, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= R) return;
    int32_t* base = a.c_pcnt + nblk * R;
    int carry = a.c_padoff[w];
    for (int64_t b0 = 0; b0 < nblk; b0 += 32) {
        const int64_t b = b0 + lane;
        const int v = b < nblk ? a.c_pcnt[b * R + w] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (b < nblk) base[b * R + w] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
}
__global__ void __launch_bounds__(1024) k_part_scatter(TrajArgs a, int64_t nblk) {
    __shared__ int wc[32][CENTRED_MAX_RUNS];   // per warp: particles of each run
    const int R = a.c_runs, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    int64_t j = -1;
    int r = -1;
    if (t < a.N) {
        j = a.perm ? a.perm[t] : t;
        r = a.run_of ? a.run_of[j] : 0;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, r);
    const int lower = __popc(peers & ((1u << lane) - 1u));
    if (lane < R) wc[w][lane] = 0;
    __syncwarp();
    if (r >= 0 && lower == 0) wc[w][r] = __popc(peers);
    __syncthreads();
    if (r >= 0) {
        int pos = a.c_pcnt[nblk * R + (int64_t)blockIdx.x * R + r] + lower;
        for (int v = 0; v < w; ++v) pos += wc[v][r];
        a.c_perm[pos] = (int32_t)j;
    }
}

// g_ref[r][d] = sum over tiles of the partial sums, in tile order.
__global__ void __launch_bounds__(128) k_centre_grad(TrajArgs a, int dk, int nch) {
    const int r = blockIdx.x, d = threadIdx.x, R = a.c_runs;
    if (d >= dk) return;
    double g = 0.0;
    for (int c = 0; c < nch; ++c) g += a.c_part[((int64_t)c * R + r) * dk + d];
    a.c_gref[(int64_t)r * dk + d] = (float)g;
}

// CTAs per particle tile: the largest k in {1, 2, 4, 8} with at most two CTAs
// per SM over the launch and at least one observation tile per CTA.  It
// depends only on the particle count, the data and the device, so a result
// never depends on a timing.
int centred_split(const DevModel& m, int64_t tiles) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
    }
    int k = 8;
    while (k > 1 && (tiles * k > 2 * (int64_t)sms || k > m.n_tiles128)) k >>= 1;
    return k;
}

template <bool LOGIT>
cudaError_t launch_centred(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const int R = a.c_runs;
    if (R < 1 || R > CENTRED_MAX_RUNS || !a.c_centre || !a.c_gref || !a.c_part || (LOGIT && !a.c_refs))
        return cudaErrorInvalidValue;
    // several runs need the run-uniform tile layout (a handle's); a tile's
    // stage then carries the reference pairs of its own run only
    if (R > 1 && (!a.c_tiles || !a.c_perm || !a.c_padoff || !a.c_pcnt || a.c_ntiles < 1))
        return cudaErrorInvalidValue;
    const CLayout L = c_layout(m.dk, m.Dp, LOGIT ? 1 : 0, R);
    if (L.total > C_SMEM_MAX) return cudaErrorInvalidValue;
    if (a.c_tiles) {
        const int64_t nblk = (a.N + 1023) / 1024;
        k_part_count<<<(unsigned)nblk, 1024, 0, s>>>(a);
        k_part_scan<<<1, 32 * R, 0, s>>>(a, nblk);
        k_part_scatter<<<(unsigned)nblk, 1024, 0, s>>>(a, nblk);
    }
    k_centre_mean<<<dim3((unsigned)R, (unsigned)m.dk), 256, 0, s>>>(a, m.D, m.dk);
    k_centre_obs<LOGIT><<<(unsigned)m.n_tiles128, 128, 0, s>>>(m, a);
    k_centre_grad<<<(unsigned)R, 128, 0, s>>>(a, m.dk, m.n_tiles128);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t tiles = a.c_tiles ? a.c_ntiles : (a.N + CP - 1) / CP;
    TrajArgs a2 = a;
    a2.c_split = centred_split(m, tiles);
    auto kern = traj_centred_kernel<LOGIT>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tiles * a2.c_split), 1, 1);
    cfg.blockDim = dim3(C_THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)L.total;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a2.c_split;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, m, a2);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

bool traj_centred_supported(const DevModel& m) {
    return (m.kind == LOGISTIC || m.kind == LINEAR_GAUSS) && m.D >= 1 && m.D <= 128 && m.xc_img &&
           m.n_tiles128 >= 1 && m.n_chunks >= 1;
}

int64_t centred_refs_elems(const DevModel& m, int n_runs) { return (int64_t)m.n_tiles128 * n_runs * CC; }
int64_t centred_part_elems(const DevModel& m, int n_runs) { return (int64_t)m.n_tiles128 * n_runs * m.dk; }

cudaError_t launch_traj_centred(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    if (!traj_centred_supported(m)) return cudaErrorInvalidValue;
    if (!a.eval_only && !a.p_out) return cudaErrorInvalidValue;   // the momenta live in p_out
    if (a.N <= 0) return cudaSuccess;
    return m.kind == LOGISTIC ? launch_centred<true>(m, a, s) : launch_centred<false>(m, a, s);
}

}  // namespace smc
