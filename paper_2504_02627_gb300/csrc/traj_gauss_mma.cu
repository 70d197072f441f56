// traj_gauss_mma.cu -- tensor-core leapfrog trajectories (Algorithm 1) for the
// correlated Gaussian target N(mu, P^-1) (Sec. 4), dimension D <= 128, on
// warp-level BF16 MMAs (m16n8k16, FP32 accumulation).
//
// Per leapfrog step the gradient of a tile of 16 particles is one dense
// product, G [16 x D] = -(Theta - mu)^T [16 x D] . P^T [D x D] (P symmetric):
// the A operand is built in registers from the particles' positions, the B
// operand is P, staged once per CTA in shared memory as BF16 rows (hi and, in
// the x3 mode, lo = P - hi), and each warp owns two n-tiles (16 output
// dimensions).  In the x3 mode both operands are split and hi*hi + lo*hi +
// hi*lo is accumulated.  The end-point log pi that enters the importance
// weight, c - 1/2 (theta - mu)' P (theta - mu), is computed with the FP32 P
// and FP64 accumulation, so the reduced-precision gradient changes only the
// integrator.
#include <cuda_bf16.h>
#include <math_constants.h>
#include "tc_ptx.cuh"
#include "traj.cuh"

namespace smc {
namespace {

constexpr int GG_P = 16;   // particles per CTA (the M of the MMA)

// Dynamic shared memory, for DK = D rounded up to 16 (bytes):
//   P hi [DK][DK + 8] bf16 | P lo (x3) | theta, p, grad [16][DK + 8] f32 |
//   mu [DK] f32 | H0, log pi [16] f64 | end-point terms [16][DK] f64
struct GgLayout {
    int dk, ldp, ds;
    size_t ph, pl, th, p, g, mu, h0, lp, part, bytes;
    __host__ __device__ GgLayout(int D, bool x3) {
        dk = (D + 15) & ~15;
        ldp = dk + 8;          // odd number of 16-byte units per row: conflict-free 8-row matrix loads
        ds = dk + 8;           // state rows: the 8-byte operand loads of a half-warp hit distinct banks
        ph = 0;
        pl = ph + (size_t)dk * ldp * 2;
        th = pl + (x3 ? (size_t)dk * ldp * 2 : 0);
        p = th + (size_t)GG_P * ds * 4;
        g = p + (size_t)GG_P * ds * 4;
        mu = g + (size_t)GG_P * ds * 4;
        h0 = mu + (size_t)dk * 4;
        h0 = (h0 + 7) & ~(size_t)7;
        lp = h0 + GG_P * 8;
        part = lp + GG_P * 8;
        bytes = part + (size_t)GG_P * dk * 8;
    }
};

__device__ __forceinline__ void gg_ldsm4(uint32_t (&v)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(addr));
}

__device__ __forceinline__ void gg_mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void gg_split(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// KS = DK / 16 k-steps and warps (each warp two n-tiles of 8 output dimensions).
template <int KS, bool X3>
__global__ void __launch_bounds__(32 * KS, 1) traj_gauss_mma_kernel(DevModel m, TrajArgs a) {
    constexpr int NTH = 32 * KS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int D = m.D;
    const GgLayout L(D, X3);
    const int DK = L.dk, LDP = L.ldp, DS = L.ds;
    float* th_s = reinterpret_cast<float*>(smem_raw + L.th);
    float* p_s = reinterpret_cast<float*>(smem_raw + L.p);
    float* g_s = reinterpret_cast<float*>(smem_raw + L.g);
    float* mu_s = reinterpret_cast<float*>(smem_raw + L.mu);
    double* H0_s = reinterpret_cast<double*>(smem_raw + L.h0);
    double* lp_s = reinterpret_cast<double*>(smem_raw + L.lp);
    const uint32_t ph_base = tc::smem_u32(smem_raw + L.ph);
    const uint32_t pl_base = tc::smem_u32(smem_raw + L.pl);
    __shared__ int64_t j_s[GG_P], src_s[GG_P];
    __shared__ float eps_s[GG_P];
    __shared__ uint64_t seed_s[GG_P];
    __shared__ uint32_t k_s[GG_P], jl_s[GG_P];
    __shared__ int S_s[GG_P];
    __shared__ int smax_s;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gq = lane >> 2, tq = lane & 3;

    // ---- P as BF16 rows (hi, lo), zero past D; mu
    for (int e = tid; e < DK * (DK / 2); e += NTH) {
        const int r = e / (DK / 2), c = 2 * (e % (DK / 2));
        const float v0 = (r < D && c < D) ? m.P[(int64_t)r * D + c] : 0.0f;
        const float v1 = (r < D && c + 1 < D) ? m.P[(int64_t)r * D + c + 1] : 0.0f;
        uint32_t hi, lo;
        gg_split(v0, v1, hi, lo);
        *reinterpret_cast<uint32_t*>(smem_raw + L.ph + ((size_t)r * LDP + c) * 2) = hi;
        if (X3) *reinterpret_cast<uint32_t*>(smem_raw + L.pl + ((size_t)r * LDP + c) * 2) = lo;
    }
    for (int e = tid; e < DK; e += NTH) mu_s[e] = e < D ? m.mu[e] : 0.0f;

    // ---- particle state of this CTA
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
    if (tid == 0) {
        int mx = 0;
        for (int q = 0; q < GG_P; ++q) mx = max(mx, S_s[q]);
        smax_s = mx;
    }
    for (int e = tid; e < GG_P * DS; e += NTH) {
        const int q = e / DS, d = e % DS;
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
        // momentum p ~ N(0, I) from the (seed, i, j, k, MOM) Philox stream
        const int npairs = (D + 1) / 2;
        for (int e = tid; e < npairs * GG_P; e += NTH) {
            const int i = e / GG_P, q = e % GG_P;
            if (j_s[q] < 0) continue;
            double z0, z1;
            normal_pair(seed_s[q], (uint32_t)i, jl_s[q], k_s[q], TAG_MOM, z0, z1);
            p_s[q * DS + 2 * i] = (float)z0;
            if (2 * i + 1 < D) p_s[q * DS + 2 * i + 1] = (float)z1;
        }
        __syncthreads();
    }
    if (tid < GG_P && !a.eval_only) {
        double kin = 0.0;
        for (int d = 0; d < D; ++d) {
            const double v = p_s[tid * DS + d];
            kin += v * v;
        }
        H0_s[tid] = j_s[tid] >= 0 ? 0.5 * kin - a.logpi_in[src_s[tid]] : 0.0;
    }
    __syncthreads();   // H0 reads p_s before the first half kick below rewrites it
    const int smax = smax_s;

    // ---- first half kick and drift of step 1
    for (int e = tid; e < GG_P * DS; e += NTH) {
        const int q = e / DS, d = e % DS;
        if (d < D && S_s[q] >= 1) {
            const float ef = eps_s[q], he = 0.5f * ef;
            const float pv = fmaf(he, g_s[e], p_s[e]);
            p_s[e] = pv;
            th_s[e] = fmaf(ef, pv, th_s[e]);
        }
    }
    __syncthreads();

    const int mi = lane >> 3, mr = lane & 7;
    const int nt0 = 2 * wid;                       // this warp's n-tiles: output dimensions 16 wid .. + 15
    const int nsteps = a.eval_only ? 1 : smax;
    for (int s = 1; s <= nsteps; ++s) {
        // ---- G = -(Theta - mu)^T P for this warp's 16 output dimensions
        float acc[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            uint32_t ah[4], al[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int q = gq + 8 * (v & 1);
                const int d = 16 * ks + 2 * tq + 8 * (v >> 1);
                const float2 tv = *reinterpret_cast<const float2*>(th_s + q * DS + d);
                const float2 mv = *reinterpret_cast<const float2*>(mu_s + d);
                gg_split(tv.x - mv.x, tv.y - mv.y, ah[v], al[v]);
            }
            // matrices: (n-tile nt0 + (mi >> 1): P rows = output dims, k half mi & 1)
            const uint32_t off = (uint32_t)(((8 * (nt0 + (mi >> 1)) + mr) * LDP + 16 * ks + 8 * (mi & 1)) * 2);
            uint32_t bh[4], bl[4];
            gg_ldsm4(bh, ph_base + off);
            if (X3) gg_ldsm4(bl, pl_base + off);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                gg_mma(acc[u], ah, bh[2 * u], bh[2 * u + 1]);
                if (X3) {
                    gg_mma(acc[u], al, bh[2 * u], bh[2 * u + 1]);
                    gg_mma(acc[u], ah, bl[2 * u], bl[2 * u + 1]);
                }
            }
        }
        // ---- gradient rows g, g + 8; output dimensions 8 (nt0 + u) + 2t, + 1
        //      (the previous step's readers of g_s finished at its last barrier)
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int d = 8 * (nt0 + u) + 2 * tq;
            *reinterpret_cast<float2*>(g_s + gq * DS + d) = make_float2(-acc[u][0], -acc[u][1]);
            *reinterpret_cast<float2*>(g_s + (gq + 8) * DS + d) = make_float2(-acc[u][2], -acc[u][3]);
        }
        __syncthreads();
        // ---- closing half kick of step s, opening kick + drift of step s + 1
        if (!a.eval_only) {
            for (int e = tid; e < GG_P * DS; e += NTH) {
                const int q = e / DS, d = e % DS;
                if (d < D && s <= S_s[q]) {
                    const float ef = eps_s[q], he = 0.5f * ef, gv = g_s[e];
                    float pv = fmaf(he, gv, p_s[e]);
                    if (s + 1 <= S_s[q]) {
                        pv = fmaf(he, gv, pv);
                        th_s[e] = fmaf(ef, pv, th_s[e]);
                    }
                    p_s[e] = pv;
                }
            }
        }
        __syncthreads();
    }

    // ---- end-point log pi = c - 1/2 (theta - mu)' P (theta - mu): FP32 P from
    //      L2, one (particle, row) term per thread into a [16][DK] FP64 array,
    //      summed per particle in row order (deterministic)
    {
        double* part = reinterpret_cast<double*>(smem_raw + L.part);
        for (int e = tid; e < GG_P * D; e += NTH) {
            const int q = e / D, r = e % D;
            const float* prow = m.P + (int64_t)r * D;
            const float* tq_ = th_s + q * DS;
            float row = 0.0f;
            for (int c = 0; c < D; ++c) row = fmaf(__ldg(prow + c), tq_[c] - mu_s[c], row);
            part[q * DK + r] = (double)((tq_[r] - mu_s[r]) * row);
        }
        __syncthreads();
        if (tid < GG_P) {
            double qf = 0.0;
            for (int r = 0; r < D; ++r) qf += part[tid * DK + r];
            lp_s[tid] = m.lconst - 0.5 * qf;
        }
        __syncthreads();
    }

    // ---- outputs
    for (int e = tid; e < GG_P * DS; e += NTH) {
        const int q = e / DS, d = e % DS;
        const int64_t j = j_s[q];
        if (j < 0 || d >= D) continue;
        if (!a.eval_only) a.theta_out[(int64_t)d * a.ld + j] = th_s[e];
        a.grad_out[(int64_t)d * a.ld + j] = g_s[e];
        if (a.p_out && !a.eval_only) a.p_out[(int64_t)d * a.ld + j] = p_s[e];
    }
    if (tid < GG_P && j_s[tid] >= 0) {
        const int64_t j = j_s[tid];
        const double lp1 = lp_s[tid];
        a.logpi_out[j] = lp1;
        if (!a.eval_only) {
            double kin = 0.0;
            for (int d = 0; d < D; ++d) {
                const double v = p_s[tid * DS + d];
                kin += v * v;
            }
            double dH = (0.5 * kin - lp1) - H0_s[tid];
            if (!isfinite(dH)) dH = CUDART_INF;
            if (a.dH) a.dH[j] = dH;
            if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
        }
    }
}

template <int KS, bool X3>
cudaError_t launch_gg(const DevModel& m, const TrajArgs& a, cudaStream_t s) {
    const GgLayout L(m.D, X3);
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
    return m.kind == GAUSS_DENSE && m.D >= 1 && m.D <= 128 && m.P && m.mu && GgLayout(m.D, true).bytes <= 220 * 1024;
}

cudaError_t launch_traj_gauss_mma(const DevModel& m, const TrajArgs& a, bool x3, cudaStream_t s) {
    if (!traj_gauss_mma_supported(m)) return cudaErrorInvalidValue;
    return x3 ? dispatch_gg<true>(m, a, s) : dispatch_gg<false>(m, a, s);
}

}  // namespace smc
