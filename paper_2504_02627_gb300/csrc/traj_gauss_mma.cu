// traj_gauss_mma.cu -- tensor-core leapfrog trajectories (Algorithm 1) for the
// correlated Gaussian target N(mu, P^-1) (Sec. 4), dimension D <= 128, on
// warp-level BF16 MMAs (m16n8k16, FP32 accumulation).
//
// Per leapfrog step the gradient of a tile of 16 particles is one dense
// product, G [16 x D] = -(Theta - mu)^T [16 x D] . P^T [D x D] (P symmetric).
// Each warp owns 16 output dimensions (two n-tiles) and keeps, in registers,
// the B fragments of its rows of P (BF16 hi and, in the x3 mode, lo = P - hi)
// for every k-step, and the particle state (theta, p, grad) of its output
// dimensions in the accumulator layout of the product: the leapfrog update
// runs on the accumulator registers, and the only per-step exchange between
// warps is the A operand (theta - mu as BF16 hi and lo), written to a
// double-buffered shared-memory tile and read with 8x8 matrix loads, so one
// CTA barrier per step.  In the x3 mode hi*hi + lo*hi + hi*lo is accumulated.
// The end-point log pi that enters the importance weight,
// c - 1/2 (theta - mu)' P (theta - mu), uses the FP32 P (copied to shared
// memory asynchronously while the steps run) with FP64 accumulation, so the
// reduced-precision gradient changes only the integrator.
#include <cuda_bf16.h>
#include <math_constants.h>
#include "tc_ptx.cuh"
#include "traj.cuh"

namespace smc {
namespace {

constexpr int GG_P = 16;   // particles per CTA (the M of the MMA)
constexpr int AT_LD = 20;  // row stride of the end point's (theta - mu) rows: conflict-free stores

// Dynamic shared memory (bytes), DK = D rounded up to 16:
//   A operand: two buffers of (hi, lo) [16][DK + 8] bf16; at the end point
//     the same bytes hold (theta - mu) [DK][20] f32 |
//   P [D][D + 1] f32 (end point) | kinetic partials [2][8][16] f64 |
//   end-point partial sums [32 KS][4] f64
struct GgLayout {
    int dk, ldp;
    size_t a, pf, kin, part, bytes;
    __host__ __device__ GgLayout(int D) {
        dk = (D + 15) & ~15;
        ldp = dk + 8;          // odd number of 16-byte units per row: conflict-free 8-row matrix loads
        a = 0;
        pf = a + 4 * (size_t)GG_P * ldp * 2;
        kin = pf + (size_t)D * (D + 1) * 4;
        kin = (kin + 15) & ~(size_t)15;
        part = kin + 2 * 8 * GG_P * 8;
        bytes = part + (size_t)2 * dk * 4 * 8;   // 32 KS = 2 DK threads
    }
};

// 4-byte asynchronous global -> shared copy
__device__ __forceinline__ void gg_cp_async4(uint32_t dst_smem, const float* src_gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst_smem), "l"(src_gmem) : "memory");
}

// FP64 sum over the four lanes of a quad (lanes 4 gq .. 4 gq + 3); every lane
// of the quad gets the same bits
__device__ __forceinline__ double gg_quad_sum(double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

// sum of the squares of a thread's four momentum elements of particle half h
__device__ __forceinline__ float gg_sq4(const float (&pp)[2][4], int h) {
    const float a = fmaf(pp[0][2 * h], pp[0][2 * h], pp[0][2 * h + 1] * pp[0][2 * h + 1]);
    const float b = fmaf(pp[1][2 * h], pp[1][2 * h], pp[1][2 * h + 1] * pp[1][2 * h + 1]);
    return a + b;
}

// KS = DK / 16 k-steps and warps.  Thread (warp w, lane 4 gq + tq) holds the
// state elements (u, 2 h + v), u, h, v in {0, 1}: particle gq + 8 h of the
// CTA, dimension 16 w + 8 u + 2 tq + v -- the m16n8 accumulator layout of
// n-tile 2 w + u.
template <int KS, bool X3>
__global__ void __launch_bounds__(32 * KS, 2) traj_gauss_mma_kernel(DevModel m, TrajArgs a) {
    constexpr int NTH = 32 * KS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int D = m.D;
    const GgLayout L(D);
    const int LDP = L.ldp;
    float* pf_s = reinterpret_cast<float*>(smem_raw + L.pf);
    float* at_s = reinterpret_cast<float*>(smem_raw + L.a);
    double* kin_s = reinterpret_cast<double*>(smem_raw + L.kin);
    double* part_s = reinterpret_cast<double*>(smem_raw + L.part);
    const uint32_t a_base = tc::smem_u32(smem_raw + L.a);
    const uint32_t a_mat = (uint32_t)(GG_P * LDP * 2);   // one [16][DK + 8] bf16 matrix
    __shared__ int64_t j_s[GG_P], src_s[GG_P];
    __shared__ float eps_s[GG_P];
    __shared__ uint64_t seed_s[GG_P];
    __shared__ uint32_t k_s[GG_P], jl_s[GG_P];
    __shared__ int S_s[GG_P];
    __shared__ double lp_s[GG_P];

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gq = lane >> 2, tq = lane & 3;

    // ---- FP32 P for the end point, row stride D + 1 (conflict-free row
    //      walks); waited on before the end point
    for (int e = tid; e < D * D; e += NTH) {
        const int r = e / D, c = e - r * D;
        gg_cp_async4(tc::smem_u32(pf_s + r * (D + 1) + c), m.P + e);
    }
    tc::cp_async_commit();

    // ---- B fragments: P rows 16 wid + 8 u + gq, columns 16 ks + 8 hk + 2 tq, + 1
    uint32_t bh[KS][2][2], bl[KS][2][2];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int hk = 0; hk < 2; ++hk) {
                const int n = 16 * wid + 8 * u + gq, k = 16 * ks + 8 * hk + 2 * tq;
                const float v0 = (n < D && k < D) ? __ldg(m.P + (int64_t)n * D + k) : 0.0f;
                const float v1 = (n < D && k + 1 < D) ? __ldg(m.P + (int64_t)n * D + k + 1) : 0.0f;
                tc::split_bf16x2(v0, v1, bh[ks][u][hk], bl[ks][u][hk]);
            }

    // ---- particle scalars of this CTA
    const int64_t slot0 = (int64_t)blockIdx.x * GG_P;
    if (tid < GG_P) {
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
    int smax = 0;
#pragma unroll
    for (int q = 0; q < GG_P; ++q) smax = max(smax, S_s[q]);

    // ---- state of this thread's elements, straight from global memory
    float th[2][4], pp[2][4], gr[2][4], mu[2][2], ef[2], he[2];
    int S[2];
    int64_t jq[2], sq[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = gq + 8 * h;
        jq[h] = j_s[q];
        sq[h] = src_s[q];
        S[h] = S_s[q];
        ef[h] = eps_s[q];
        he[h] = 0.5f * ef[h];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int d = 16 * wid + 8 * u + 2 * tq + v;
            mu[u][v] = d < D ? m.mu[d] : 0.0f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = 2 * h + v;
                float tv = 0.0f, gv = 0.0f, pv = 0.0f;
                if (sq[h] >= 0 && d < D) {
                    tv = a.theta_in[(int64_t)d * a.ld + sq[h]];
                    if (!a.eval_only) gv = a.grad_in[(int64_t)d * a.ld + sq[h]];
                    if (a.p_in && !a.eval_only) pv = a.p_in[(int64_t)d * a.ld + jq[h]];
                }
                th[u][e] = tv;
                gr[u][e] = gv;
                pp[u][e] = pv;
            }
        }
    if (!a.p_in && !a.eval_only) {
        // momentum p ~ N(0, I) from the (seed, i, j, k, MOM) Philox stream: this
        // thread's dimensions 2 i, 2 i + 1 are one pair, i = 8 wid + 4 u + tq
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = gq + 8 * h, i = 8 * wid + 4 * u + tq;
                if (jq[h] >= 0 && 2 * i < D) {
                    float z0, z1;
                    normal_pair_f32(seed_s[q], (uint32_t)i, jl_s[q], k_s[q], TAG_MOM, z0, z1);
                    pp[u][2 * h] = z0;
                    pp[u][2 * h + 1] = 2 * i + 1 < D ? z1 : 0.0f;
                }
            }
    }
    // kinetic energy of the starting momenta, per (warp, particle): a thread's
    // four squares summed in FP32, FP64 from the quad sum on
    if (!a.eval_only) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double k = gg_quad_sum((double)gg_sq4(pp, h));
            if (tq == 0) kin_s[wid * GG_P + gq + 8 * h] = k;
        }
    }

    // A operand element pairs of this thread into buffer `buf`
    auto put_a = [&](int buf) {
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t hi, lo;
                tc::split_bf16x2(th[u][2 * h] - mu[u][0], th[u][2 * h + 1] - mu[u][1], hi, lo);
                const uint32_t off = (uint32_t)(((gq + 8 * h) * LDP + 16 * wid + 8 * u + 2 * tq) * 2);
                unsigned char* base = smem_raw + L.a + (size_t)2 * buf * a_mat;
                *reinterpret_cast<uint32_t*>(base + off) = hi;
                if (X3) *reinterpret_cast<uint32_t*>(base + a_mat + off) = lo;
            }
    };

    // ---- first half kick and drift of step 1 (dimensions past D stay 0)
    if (!a.eval_only) {
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int h = e >> 1;
                if (S[h] >= 1) {
                    const float pv = fmaf(he[h], gr[u][e], pp[u][e]);
                    pp[u][e] = pv;
                    th[u][e] = fmaf(ef[h], pv, th[u][e]);
                }
            }
    }
    put_a(0);
    __syncthreads();

    const int mi = lane >> 3, mr = lane & 7;
    // this lane's 8x8 matrix row of the A tile: matrices (particles 8 (mi & 1) ..,
    // k 8 (mi >> 1) ..) of each k-step
    const uint32_t a_lane = a_base + (uint32_t)(((8 * (mi & 1) + mr) * LDP + 8 * (mi >> 1)) * 2);
    const int nsteps = a.eval_only ? 1 : smax;
    for (int s = 1; s <= nsteps; ++s) {
        const int buf = (s - 1) & 1;
        const uint32_t ahb = a_lane + (uint32_t)(2 * buf) * a_mat;
        // ---- G = -(Theta - mu)^T P for this warp's 16 output dimensions
        // two accumulators per n-tile halve the dependent MMA chain: hi*hi in
        // acc and the two correction products in cor (x3), or even and odd
        // k-steps (plain BF16)
        float acc[2][4], cor[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[u][e] = cor[u][e] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            uint32_t ah[4], al[4];
            tc::ldsm4(ah, ahb + 32 * ks);
            if (X3) tc::ldsm4(al, ahb + a_mat + 32 * ks);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (X3) {
                    tc::mma_bf16_16816(acc[u], ah, bh[ks][u][0], bh[ks][u][1]);
                    tc::mma_bf16_16816(cor[u], al, bh[ks][u][0], bh[ks][u][1]);
                    tc::mma_bf16_16816(cor[u], ah, bl[ks][u][0], bl[ks][u][1]);
                } else {
                    tc::mma_bf16_16816((ks & 1) ? cor[u] : acc[u], ah, bh[ks][u][0], bh[ks][u][1]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int e = 0; e < 4; ++e) gr[u][e] = -(acc[u][e] + cor[u][e]);
        // ---- closing half kick of step s; opening kick + drift of step s + 1
        //      and its A operand into the other buffer (its readers, step
        //      s - 1, finished at the previous barrier)
        if (!a.eval_only) {
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int h = e >> 1;
                    if (s <= S[h]) {
                        float pv = fmaf(he[h], gr[u][e], pp[u][e]);
                        if (s + 1 <= S[h]) {
                            pv = fmaf(he[h], gr[u][e], pv);
                            th[u][e] = fmaf(ef[h], pv, th[u][e]);
                        }
                        pp[u][e] = pv;
                    }
                }
            if (s < nsteps) put_a(buf ^ 1);
        }
        __syncthreads();
    }

    // ---- end point.  (theta - mu) transposed [DK][AT_LD] f32 over the A tiles
    //      (free after the last barrier); kinetic energy of the final momenta
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int d = 16 * wid + 8 * u + 2 * tq + (e & 1), q = gq + 8 * (e >> 1);
            at_s[d * AT_LD + q] = th[u][e] - mu[u][e & 1];
        }
    if (!a.eval_only) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double k = gg_quad_sum((double)gg_sq4(pp, h));
            if (tq == 0) kin_s[(8 + wid) * GG_P + gq + 8 * h] = k;
        }
    }
    tc::cp_async_wait<0>();
    __syncthreads();
    // (theta - mu)' P (theta - mu): thread t takes particles 4 (t & 3) .. + 3 and
    // rows t / 4, t / 4 + NTH / 4, ... (at most two, as 8 KS >= D / 2); each
    // row product in FP32, a thread's terms summed in FP32, FP64 from there on
    {
        const int g4 = tid & 3;
        float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int r = tid >> 2; r < D; r += NTH / 4) {
            const float* prow = pf_s + r * (D + 1);
            float row[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int c = 0; c < D; ++c) {
                const float pv = prow[c];
                const float4 av = *reinterpret_cast<const float4*>(at_s + c * AT_LD + 4 * g4);
                row[0] = fmaf(pv, av.x, row[0]);
                row[1] = fmaf(pv, av.y, row[1]);
                row[2] = fmaf(pv, av.z, row[2]);
                row[3] = fmaf(pv, av.w, row[3]);
            }
            const float4 ar = *reinterpret_cast<const float4*>(at_s + r * AT_LD + 4 * g4);
            s4[0] = fmaf(ar.x, row[0], s4[0]);
            s4[1] = fmaf(ar.y, row[1], s4[1]);
            s4[2] = fmaf(ar.z, row[2], s4[2]);
            s4[3] = fmaf(ar.w, row[3], s4[3]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) part_s[tid * 4 + i] = (double)s4[i];
    }
    __syncthreads();
    // per particle q: the NTH / 4 partial sums of threads (q >> 2) + 4 r, in
    // four interleaved chains (items 4 q .. 4 q + 3, one quad of lanes) joined
    // by a quad sum; 4 GG_P = 64 items, so whole warps take part
    for (int e = tid; e < 4 * GG_P; e += NTH) {
        const int q = e >> 2, c = e & 3;
        double qf = 0.0;
        for (int r = c; r < NTH / 4; r += 4) qf += part_s[((q >> 2) + 4 * r) * 4 + (q & 3)];
        qf = gg_quad_sum(qf);
        if (c == 0) lp_s[q] = qf;
    }
    __syncthreads();
    if (tid < GG_P) {
        const int q = tid;
        const int64_t j = j_s[q];
        if (j >= 0) {
            const double lp1 = m.lconst - 0.5 * lp_s[q];
            a.logpi_out[j] = lp1;
            if (!a.eval_only) {
                double kin0 = 0.0, kin1 = 0.0;
                for (int w = 0; w < KS; ++w) {
                    kin0 += kin_s[w * GG_P + q];
                    kin1 += kin_s[(8 + w) * GG_P + q];
                }
                const double H0 = 0.5 * kin0 - a.logpi_in[src_s[q]];
                double dH = (0.5 * kin1 - lp1) - H0;
                if (!isfinite(dH)) dH = CUDART_INF;
                if (a.dH) a.dH[j] = dH;
                if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
            }
        }
    }

    // ---- outputs, straight from the registers (8 consecutive particle slots
    //      of one dimension per 32-byte sector)
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int d = 16 * wid + 8 * u + 2 * tq + (e & 1);
            const int64_t j = jq[e >> 1];
            if (j < 0 || d >= D) continue;
            if (!a.eval_only) a.theta_out[(int64_t)d * a.ld + j] = th[u][e];
            a.grad_out[(int64_t)d * a.ld + j] = gr[u][e];
            if (a.p_out && !a.eval_only) a.p_out[(int64_t)d * a.ld + j] = pp[u][e];
        }
}

template <int KS, bool X3>
cudaError_t launch_gg(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const GgLayout L(m.D);
    auto kern = traj_gauss_mma_kernel<KS, X3>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
    if (e != cudaSuccess) return e;
    const int64_t grid = (a.N + GG_P - 1) / GG_P;
    if (grid == 0) return cudaSuccess;
    kern<<<(unsigned)grid, 32 * KS, L.bytes, s>>>(m, a);
    return cudaGetLastError();
}

template <bool X3>
cudaError_t dispatch_gg(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    switch ((m.D + 15) / 16) {
        case 1: return launch_gg<1, X3>(m, a, s);
        case 2: return launch_gg<2, X3>(m, a, s);
        case 3: return launch_gg<3, X3>(m, a, s);
        case 4: return launch_gg<4, X3>(m, a, s);
        case 5: return launch_gg<5, X3>(m, a, s);
        case 6: return launch_gg<6, X3>(m, a, s);
        case 7: return launch_gg<7, X3>(m, a, s);
        case 8: return launch_gg<8, X3>(m, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool traj_gauss_mma_supported(const DevModel& m) {
    return m.kind == GAUSS_DENSE && m.D >= 1 && m.D <= 128 && m.P && m.mu && GgLayout(m.D).bytes <= 220 * 1024;
}

cudaError_t launch_traj_gauss_mma(const DevModel& m, const TrajArgs& a, bool x3, cudaStream_t s) {
    if (!traj_gauss_mma_supported(m)) return cudaErrorInvalidValue;
    return x3 ? dispatch_gg<true>(m, a, s) : dispatch_gg<false>(m, a, s);
}

}  // namespace smc
