// flow.cu -- the learned preconditioner on the GPU: an affine-coupling flow
// theta = T(z) (L coupling layers; layer l keeps half A_l and maps
// b -> b exp(s(a)) + t(a) on half B_l, (s_raw, t) = W3 tanh(W2 tanh(W1 a +
// b1) + b2) + b3, s = 2 tanh(s_raw)), HMC in the latent space with
// log pi_z(z) = log pi(T(z)) + log|det dT/dz| (Algorithm 1 applied to pi_z),
// and its training by the weighted negative log-likelihood of the particles.
//
// All conditioner products are batched over the 32 particles of a CTA: the
// activations [rows x 32] stay in shared memory and the weights stream from
// L2 as 16-byte rows of padded work copies (a transposed copy serves the
// backward products), each thread accumulating a 4 x 4 tile.  FP32 with the
// trajectory end-point energy accumulated in FP64.  The BF16 forms run the
// same products on m16n8k16 warp MMAs (BF16 operands, FP32 accumulation):
// the trajectories' conditioner and transposed products from pre-arranged
// weight fragments, and in training also the weight gradients, which are
// products over the CTA's 32 particles.
#include <cuda_bf16.h>
#include <math_constants.h>
#include "flow.cuh"
#include "tc_ptx.cuh"

namespace smc {
namespace {
constexpr int FG = 32;           // particles per CTA
constexpr int FT = 256;          // threads per CTA
}  // namespace

// activations [rows x 32] of: z, p, grad_z, x, cotangent, grad_x, the L
// layer inputs, h1, h2, the conditioner output, a scratch row block; FP64
// log-determinant partials
size_t flow_smem_bytes(int D, int H, int L, int O4) {
    return sizeof(float) * (size_t)FG * (6 * D + L * D + 3 * H + O4) + sizeof(double) * 9 * FG;
}
// ... plus the BF16 operand buffer of the MMA form: [32][K + 8] for K <= 128
static size_t flow_pm_bytes() { return sizeof(uint16_t) * (size_t)FG * (128 + 8); }

namespace {

// -------------------------------------------------------------- work copies
__global__ void k_flow_refresh(DevFlow f, bool bump, FlowGate gate) {
    const int64_t total = (int64_t)f.L * f.layer_work;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (bump && i == 0 && gate.open()) *f.adam_t += 1;
    if (i >= total) return;
    const int l = (int)(i / f.layer_work);
    const int64_t e = i % f.layer_work;
    const int H = f.H, Dh = f.Dh, Dh4 = f.Dh4, O4 = f.O4, D = f.D;
    const FlowLayerOff o = flow_layer_off(H, Dh, Dh4, O4);
    const int64_t lsz = (int64_t)H * Dh + H + (int64_t)H * H + H + (int64_t)D * H + D;
    const float* P = f.params + l * lsz;
    const float *W1 = P, *b1 = W1 + (int64_t)H * Dh, *W2 = b1 + H, *b2 = W2 + (int64_t)H * H, *W3 = b2 + H,
                *b3 = W3 + (int64_t)D * H;
    // padded output row r' of the conditioner -> canonical row (or -1)
    auto canon = [&](int rp) -> int { return rp < Dh ? rp : (rp >= Dh4 && rp < Dh4 + Dh ? Dh + (rp - Dh4) : -1); };
    float v = 0.0f;
    if (e < o.W1) {                                   // W1t [Dh][H]
        const int k = (int)(e / H), h = (int)(e % H);
        v = W1[(int64_t)h * Dh + k];
    } else if (e < o.b1) {                            // W1 [H][Dh4]
        const int64_t q = e - o.W1;
        const int h = (int)(q / Dh4), k = (int)(q % Dh4);
        v = k < Dh ? W1[(int64_t)h * Dh + k] : 0.0f;
    } else if (e < o.W2t) {
        v = b1[e - o.b1];
    } else if (e < o.W2) {                            // W2t [H][H]
        const int64_t q = e - o.W2t;
        const int k = (int)(q / H), h = (int)(q % H);
        v = W2[(int64_t)h * H + k];
    } else if (e < o.b2) {
        v = W2[e - o.W2];
    } else if (e < o.W3t) {
        v = b2[e - o.b2];
    } else if (e < o.W3) {                            // W3t [H][O4]
        const int64_t q = e - o.W3t;
        const int h = (int)(q / O4), rp = (int)(q % O4);
        const int r = canon(rp);
        v = r >= 0 ? W3[(int64_t)r * H + h] : 0.0f;
    } else if (e < o.b3) {                            // W3 [O4][H]
        const int64_t q = e - o.W3;
        const int rp = (int)(q / H), h = (int)(q % H);
        const int r = canon(rp);
        v = r >= 0 ? W3[(int64_t)r * H + h] : 0.0f;
    } else {                                          // b3 [O4]
        const int r = canon((int)(e - o.b3));
        v = r >= 0 ? b3[r] : 0.0f;
    }
    f.work[i] = v;
}

// BF16 operand fragments of the six conditioner matrices (layout in flow.cuh).
// Element (r, c) of each logical matrix, zero outside the valid block.
__global__ void k_flow_frag(DevFlow f) {
    const int64_t total = (int64_t)f.L * f.layer_frag;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int l = (int)(i / f.layer_frag);
    const int64_t e = i % f.layer_frag;
    const int H = f.H, Dh = f.Dh, Dh4 = f.Dh4;
    const FlowFragOff fo = flow_frag_off(H, f.kp1, f.o4p);
    const int64_t lsz = (int64_t)H * Dh + H + (int64_t)H * H + H + (int64_t)f.D * H + f.D;
    const float* P = f.params + l * lsz;
    const float *W1 = P, *W2 = W1 + (int64_t)H * Dh + H, *W3 = W2 + (int64_t)H * H + H;
    auto canon = [&](int rp) -> int { return rp < Dh ? rp : (rp >= Dh4 && rp < Dh4 + Dh ? Dh + (rp - Dh4) : -1); };
    int which, ks_n;
    int64_t base;
    if (e < fo.W2) { which = 0; base = fo.W1; ks_n = f.kp1 / 16; }
    else if (e < fo.W3) { which = 1; base = fo.W2; ks_n = H / 16; }
    else if (e < fo.W1t) { which = 2; base = fo.W3; ks_n = H / 16; }
    else if (e < fo.W2t) { which = 3; base = fo.W1t; ks_n = H / 16; }
    else if (e < fo.W3t) { which = 4; base = fo.W2t; ks_n = H / 16; }
    else { which = 5; base = fo.W3t; ks_n = f.o4p / 16; }
    const int64_t local = e - base;
    const int lane = (int)(local & 31);
    const int64_t tile = local >> 5;
    const int mt = (int)(tile / ks_n), ks = (int)(tile % ks_n);
    auto A = [&](int r, int c) -> float {
        switch (which) {
            case 0: return c < Dh ? W1[(int64_t)r * Dh + c] : 0.0f;                  // W1 [h][k]
            case 1: return W2[(int64_t)r * H + c];                                     // W2 [h][k]
            case 2: { const int cr = canon(r); return cr >= 0 ? W3[(int64_t)cr * H + c] : 0.0f; }   // W3 [rp][h]
            case 3: return r < Dh ? W1[(int64_t)c * Dh + r] : 0.0f;                  // W1t [k][h]
            case 4: return W2[(int64_t)c * H + r];                                     // W2t [k][h]
            default: { const int cr = canon(c); return cr >= 0 ? W3[(int64_t)cr * H + r] : 0.0f; }  // W3t [h][rp]
        }
    };
    const int g = lane >> 2, t = lane & 3;
    const int r0 = 16 * mt + g, r1 = r0 + 8, c0 = 16 * ks + 2 * t, c1 = c0 + 8;
    auto pk = [](float x, float y) -> uint32_t {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
        return *reinterpret_cast<const uint32_t*>(&h);
    };
    f.frag[i] = make_uint4(pk(A(r0, c0), A(r0, c0 + 1)), pk(A(r1, c0), A(r1, c0 + 1)), pk(A(r0, c1), A(r0, c1 + 1)),
                           pk(A(r1, c1), A(r1, c1 + 1)));
}

// -------------------------------------------------------------- building blocks
// Y[n][p] = act(sum_k At[k][n] X[k][p] + bias[n]) for n < Nout (multiple of 4,
// at most 128), the CTA's 32 particles p; At rows are 16-byte aligned.
template <bool TANH, bool BIAS>
__device__ __forceinline__ void cta_mm(const float* __restrict__ At, int K, int Nout, const float* X, float* Y,
                                       const float* __restrict__ bias) {
    const int t = threadIdx.x, nb = t >> 3, pb = t & 7;
    if (4 * nb < Nout) {
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = 0.0f;
        const float* ap = At + 4 * nb;
        for (int k = 0; k < K; ++k) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(ap + (int64_t)k * Nout));
            const float4 x = *reinterpret_cast<const float4*>(X + k * FG + 4 * pb);
            const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i][0] = fmaf(av[i], x.x, acc[i][0]);
                acc[i][1] = fmaf(av[i], x.y, acc[i][1]);
                acc[i][2] = fmaf(av[i], x.z, acc[i][2]);
                acc[i][3] = fmaf(av[i], x.w, acc[i][3]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float bb = BIAS ? __ldg(bias + 4 * nb + i) : 0.0f;
            float4 y;
            y.x = acc[i][0] + bb;
            y.y = acc[i][1] + bb;
            y.z = acc[i][2] + bb;
            y.w = acc[i][3] + bb;
            if (TANH) {
                y.x = tanhf(y.x);
                y.y = tanhf(y.y);
                y.z = tanhf(y.z);
                y.w = tanhf(y.w);
            }
            *reinterpret_cast<float4*>(Y + (4 * nb + i) * FG + 4 * pb) = y;
        }
    }
}

// FP32 rows X [R x 32] -> BF16 particle-major B [32][ldb] (k contiguous),
// zero for R <= k < Kpad: the B operand of the next MMA.  A thread converts
// eight consecutive k of one particle (lanes = particles: the row reads are
// conflict-free, and the 16-byte stores at a row stride of ldb = K + 8 fall
// in distinct bank groups).
__device__ __noinline__ void to_pm(const float* X, int R, int Kpad, __nv_bfloat16* B, int ldb) {
    for (int e = threadIdx.x; e < FG * (Kpad / 8); e += FT) {
        const int q = e & (FG - 1), k0 = 8 * (e / FG);
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int k = k0 + 2 * h;
            const float v0 = k < R ? X[k * FG + q] : 0.0f, v1 = k + 1 < R ? X[(k + 1) * FG + q] : 0.0f;
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v0, v1);
            w[h] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        *reinterpret_cast<uint4*>(B + q * ldb + k0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Y[r][p] = act(sum_k A[r][k] B[k][p] + bias[r]) for rows r < Mvalid and the
// CTA's 32 particles, on m16n8k16 BF16 MMAs with FP32 accumulation.  A: MT x KS
// tiles of fragments (L2), B: BF16 particle-major [32][ldb] in shared memory
// (ldb = K + 8: the eight 16-byte rows of a matrix load fall in distinct bank
// groups).  A warp takes one m-tile and all four n-tiles when there are eight
// or more m-tiles, else one m-tile and two n-tiles.
template <bool TANH, bool BIAS>
__device__ __noinline__ void cta_mma(const uint4* __restrict__ Af, int MT, int KS, const __nv_bfloat16* B, int ldb,
                                        float* Y, const float* __restrict__ bias, int Mvalid) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int mi = lane >> 3, mr = lane & 7;
    const bool full = MT >= FT / 32;
    const int items = full ? MT : 2 * MT;
    const uint32_t bbase = tc::smem_u32(B);
    for (int it = wid; it < items; it += FT / 32) {
        const int mt = full ? it : it >> 1;
        const int nt0 = full ? 0 : 2 * (it & 1);
        const int nh = full ? 2 : 1;          // n-tile pairs of this item
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
        // every A fragment of this m-tile in flight at once (KS <= 8): the
        // loads come from L2 and the products behind them are short
        uint4 afr[8];
#pragma unroll
        for (int ks = 0; ks < 8; ++ks)
            if (ks < KS) afr[ks] = __ldg(Af + ((int64_t)mt * KS + ks) * 32 + lane);
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
            if (ks >= KS) break;
            const uint32_t av[4] = {afr[ks].x, afr[ks].y, afr[ks].z, afr[ks].w};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h < nh) {
                    // matrices (n-tile nt0 + 2h + (mi >> 1), k half mi & 1)
                    const int prow = 8 * (nt0 + 2 * h + (mi >> 1)) + mr;
                    const int kcol = 16 * ks + 8 * (mi & 1);
                    uint32_t b[4];
                    tc::ldsm4(b, bbase + (uint32_t)(prow * ldb + kcol) * 2u);
                    tc::mma_bf16_16816(acc[2 * h], av, b[0], b[1]);
                    tc::mma_bf16_16816(acc[2 * h + 1], av, b[2], b[3]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (u < 2 * nh) {
                const int pc = 8 * (nt0 + u) + 2 * t;
                const int r0 = 16 * mt + g, r1 = r0 + 8;
                float v0 = acc[u][0], v1 = acc[u][1], v2 = acc[u][2], v3 = acc[u][3];
                if (BIAS) {
                    const float b0 = r0 < Mvalid ? __ldg(bias + r0) : 0.0f, b1 = r1 < Mvalid ? __ldg(bias + r1) : 0.0f;
                    v0 += b0;
                    v1 += b0;
                    v2 += b1;
                    v3 += b1;
                }
                if (TANH) {
                    v0 = tanhf(v0);
                    v1 = tanhf(v1);
                    v2 = tanhf(v2);
                    v3 = tanhf(v3);
                }
                if (r0 < Mvalid) *reinterpret_cast<float2*>(Y + r0 * FG + pc) = make_float2(v0, v1);
                if (r1 < Mvalid) *reinterpret_cast<float2*>(Y + r1 * FG + pc) = make_float2(v2, v3);
            }
        }
    }
}

struct FlowSmem {
    float *z, *p, *gz, *x, *c, *gx, *zl, *h1, *h2, *o, *ch;
    double *ldp, *ld;    // [8][32] partials, [32]
    __nv_bfloat16* pm;   // BF16 form: the B operand of the next product, [32][<= 136]
};

__device__ __forceinline__ FlowSmem flow_smem(unsigned char* base, int D, int H, int L, int O4) {
    FlowSmem s;
    float* f = reinterpret_cast<float*>(base);
    s.z = f;
    s.p = s.z + D * FG;
    s.gz = s.p + D * FG;
    s.x = s.gz + D * FG;
    s.c = s.x + D * FG;
    s.gx = s.c + D * FG;
    s.zl = s.gx + D * FG;
    s.h1 = s.zl + L * D * FG;
    s.h2 = s.h1 + H * FG;
    s.o = s.h2 + H * FG;
    s.ch = s.o + O4 * FG;
    s.ldp = reinterpret_cast<double*>(s.ch + H * FG);
    s.ld = s.ldp + 8 * FG;
    return s;
}

// Conditioner of layer l at rows [aoff, aoff + Dh) of `in`: h1, h2, o.
// MMA: the three products on BF16 warp MMAs (operands rounded to BF16, FP32
// accumulation, bias and tanh in FP32).
template <bool MMA = false>
__device__ __forceinline__ void conditioner(const DevFlow& f, int l, const float* in, FlowSmem& s) {
    const FlowLayerOff o = flow_layer_off(f.H, f.Dh, f.Dh4, f.O4);
    const float* w = f.work + (int64_t)l * f.layer_work;
    const int aoff = (l & 1) ? f.Dh : 0;
    if (MMA) {
        const uint4* fr = f.frag + (int64_t)l * f.layer_frag;
        const FlowFragOff fo = flow_frag_off(f.H, f.kp1, f.o4p);
        const int H = f.H;
        to_pm(in + aoff * FG, f.Dh, f.kp1, s.pm, f.kp1 + 8);
        __syncthreads();
        cta_mma<true, true>(fr + fo.W1, H / 16, f.kp1 / 16, s.pm, f.kp1 + 8, s.h1, w + o.b1, H);
        __syncthreads();
        to_pm(s.h1, H, H, s.pm, H + 8);
        __syncthreads();
        cta_mma<true, true>(fr + fo.W2, H / 16, H / 16, s.pm, H + 8, s.h2, w + o.b2, H);
        __syncthreads();
        to_pm(s.h2, H, H, s.pm, H + 8);
        __syncthreads();
        cta_mma<false, true>(fr + fo.W3, f.o4p / 16, H / 16, s.pm, H + 8, s.o, w + o.b3, f.O4);
        __syncthreads();
        return;
    }
    cta_mm<true, true>(w + o.W1t, f.Dh, f.H, in + aoff * FG, s.h1, w + o.b1);
    __syncthreads();
    cta_mm<true, true>(w + o.W2t, f.H, f.H, s.h1, s.h2, w + o.b2);
    __syncthreads();
    cta_mm<false, true>(w + o.W3t, f.H, f.O4, s.h2, s.o, w + o.b3);
    __syncthreads();
}

// Per-particle sum of v over the rows a thread visits, combined in a fixed
// order: thread t handles particle t % 32 and rows t / 32, t / 32 + 8, ...
__device__ __forceinline__ void ld_accumulate(FlowSmem& s, double v, bool add_to_ld) {
    const int t = threadIdx.x;
    s.ldp[(t >> 5) * FG + (t & 31)] = v;
    __syncthreads();
    if (t < FG) {
        double acc = 0.0;
        for (int g = 0; g < 8; ++g) acc += s.ldp[g * FG + t];
        s.ld[t] = add_to_ld ? s.ld[t] + acc : acc;
    }
    __syncthreads();
}

// x <- T(x), recording the input of every layer in zl; s.ld = log|det dT/dz|.
template <bool MMA = false>
__device__ void flow_forward(const DevFlow& f, FlowSmem& s, float* x) {
    const int t = threadIdx.x, D = f.D;
    if (t < FG) s.ld[t] = 0.0;
    for (int l = 0; l < f.L; ++l) {
        for (int e = t; e < D * FG; e += FT) s.zl[l * D * FG + e] = x[e];
        __syncthreads();
        conditioner<MMA>(f, l, x, s);
        const int boff = (l & 1) ? 0 : f.Dh;
        double part = 0.0;
        for (int k = t >> 5; k < f.Dh; k += 8) {
            const int q = t & 31;
            const float sv = 2.0f * tanhf(s.o[k * FG + q]);
            const float tv = s.o[(f.Dh4 + k) * FG + q];
            x[(boff + k) * FG + q] = fmaf(x[(boff + k) * FG + q], expf(sv), tv);
            part += (double)sv;
        }
        ld_accumulate(s, part, true);
    }
}

// x <- T^-1(x), recording the output of every inverse layer (= the input of
// forward layer l) in zl; s.ld = log|det dT^-1/dx| = -sum s.
template <bool MMA = false>
__device__ void flow_inverse(const DevFlow& f, FlowSmem& s, float* x) {
    const int t = threadIdx.x, D = f.D;
    if (t < FG) s.ld[t] = 0.0;
    __syncthreads();
    for (int l = f.L - 1; l >= 0; --l) {
        conditioner<MMA>(f, l, x, s);
        const int boff = (l & 1) ? 0 : f.Dh;
        double part = 0.0;
        for (int k = t >> 5; k < f.Dh; k += 8) {
            const int q = t & 31;
            const float sv = 2.0f * tanhf(s.o[k * FG + q]);
            const float tv = s.o[(f.Dh4 + k) * FG + q];
            x[(boff + k) * FG + q] = (x[(boff + k) * FG + q] - tv) * expf(-sv);
            part -= (double)sv;
        }
        ld_accumulate(s, part, true);
        for (int e = t; e < D * FG; e += FT) s.zl[l * D * FG + e] = x[e];
        __syncthreads();
    }
}

// c <- J_T(z)^T c + grad_z log|det dT/dz| using the recorded layer inputs.
template <bool MMA = false>
__device__ void flow_backward(const DevFlow& f, FlowSmem& s, float* c) {
    const int t = threadIdx.x, D = f.D;
    const FlowLayerOff off = flow_layer_off(f.H, f.Dh, f.Dh4, f.O4);
    for (int l = f.L - 1; l >= 0; --l) {
        const float* in = s.zl + l * D * FG;
        const float* w = f.work + (int64_t)l * f.layer_work;
        conditioner<MMA>(f, l, in, s);
        const int boff = (l & 1) ? 0 : f.Dh, aoff = (l & 1) ? f.Dh : 0;
        for (int e = t; e < f.Dh4 * FG; e += FT) {
            const int k = e / FG, q = e % FG;
            float cs_raw = 0.0f, ct = 0.0f;
            if (k < f.Dh) {
                const float th = tanhf(s.o[k * FG + q]);
                const float es = expf(2.0f * th);
                const float cbp = c[(boff + k) * FG + q];
                const float cs = fmaf(cbp * in[(boff + k) * FG + q], es, 1.0f);   // + d logdet / ds
                cs_raw = cs * 2.0f * (1.0f - th * th);
                ct = cbp;
                c[(boff + k) * FG + q] = cbp * es;
            }
            s.o[k * FG + q] = cs_raw;
            s.o[(f.Dh4 + k) * FG + q] = ct;
        }
        __syncthreads();
        if (MMA) {
            // the transposed products: W3^T og, W2^T d2, W1^T d1 (BF16 operands)
            const uint4* fr = f.frag + (int64_t)l * f.layer_frag;
            const FlowFragOff fo = flow_frag_off(f.H, f.kp1, f.o4p);
            const int H = f.H;
            to_pm(s.o, f.O4, f.o4p, s.pm, f.o4p + 8);
            __syncthreads();
            cta_mma<false, false>(fr + fo.W3t, H / 16, f.o4p / 16, s.pm, f.o4p + 8, s.ch, nullptr, H);
            __syncthreads();
            for (int e = t; e < H * FG; e += FT) s.h2[e] = s.ch[e] * (1.0f - s.h2[e] * s.h2[e]);
            __syncthreads();
            to_pm(s.h2, H, H, s.pm, H + 8);
            __syncthreads();
            cta_mma<false, false>(fr + fo.W2t, H / 16, H / 16, s.pm, H + 8, s.ch, nullptr, H);
            __syncthreads();
            for (int e = t; e < H * FG; e += FT) s.h1[e] = s.ch[e] * (1.0f - s.h1[e] * s.h1[e]);
            __syncthreads();
            to_pm(s.h1, H, H, s.pm, H + 8);
            __syncthreads();
            cta_mma<false, false>(fr + fo.W1t, f.kp1 / 16, H / 16, s.pm, H + 8, s.ch, nullptr, f.Dh4);
            __syncthreads();
        } else {
            cta_mm<false, false>(w + off.W3, f.O4, f.H, s.o, s.ch, nullptr);
            __syncthreads();
            for (int e = t; e < f.H * FG; e += FT) s.h2[e] = s.ch[e] * (1.0f - s.h2[e] * s.h2[e]);
            __syncthreads();
            cta_mm<false, false>(w + off.W2, f.H, f.H, s.h2, s.ch, nullptr);
            __syncthreads();
            for (int e = t; e < f.H * FG; e += FT) s.h1[e] = s.ch[e] * (1.0f - s.h1[e] * s.h1[e]);
            __syncthreads();
            cta_mm<false, false>(w + off.W1, f.H, f.Dh4, s.h1, s.ch, nullptr);
            __syncthreads();
        }
        for (int e = t; e < f.Dh * FG; e += FT) c[aoff * FG + e] += s.ch[e];
        __syncthreads();
    }
}

// grad log pi at x (dense Gaussian: -P (x - mu); banana pairs: closed form),
// into g.  For the Gaussian, P and mu are first staged in `scratch` (the
// conditioner's activation buffers, idle between a forward pass and the
// backward pass) when they fit (`fits`), else read from L2.
template <int TARGET>
__device__ void target_grad(const DevModel& m, const float* x, float* g, float* scratch, bool fits) {
    const int t = threadIdx.x, D = m.D;
    if constexpr (TARGET == 0) {
        const float* Pm = m.P;
        const float* mu = m.mu;
        if (fits) {
            for (int e = t; e < D * D; e += FT) scratch[e] = __ldg(m.P + e);
            for (int e = t; e < D; e += FT) scratch[D * D + e] = __ldg(m.mu + e);
            __syncthreads();
            Pm = scratch;
            mu = scratch + D * D;
        }
        const int db = t >> 3, pb = t & 7;
        if (4 * db < D) {
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] = 0.0f;
            for (int k = 0; k < D; ++k) {
                const float mk = mu[k];
                const float4 x4 = *reinterpret_cast<const float4*>(x + k * FG + 4 * pb);
                const float b0 = x4.x - mk, b1 = x4.y - mk, b2 = x4.z - mk, b3 = x4.w - mk;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int d = 4 * db + i;
                    const float a = d < D ? Pm[(int64_t)d * D + k] : 0.0f;
                    acc[i][0] = fmaf(a, b0, acc[i][0]);
                    acc[i][1] = fmaf(a, b1, acc[i][1]);
                    acc[i][2] = fmaf(a, b2, acc[i][2]);
                    acc[i][3] = fmaf(a, b3, acc[i][3]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int d = 4 * db + i;
                if (d < D)
                    *reinterpret_cast<float4*>(g + d * FG + 4 * pb) =
                        make_float4(-acc[i][0], -acc[i][1], -acc[i][2], -acc[i][3]);
            }
        }
    } else {
        const float a = (float)m.h0, b = (float)m.h1, inva = (float)(1.0 / m.h0);
        for (int e = t; e < (D / 2) * FG; e += FT) {
            const int i = e / FG, q = e % FG;
            const float xo = x[(2 * i) * FG + q], xe = x[(2 * i + 1) * FG + q];
            const float u = xe - b * (xo * xo - a);
            g[(2 * i) * FG + q] = -xo * inva + 2.0f * b * u * xo;
            g[(2 * i + 1) * FG + q] = -u;
        }
    }
}

// log pi at x in FP64 for particle q (the FP32 gradient g at x is reused for
// the dense Gaussian: log pi = c + 1/2 (x - mu)' g).
template <int TARGET>
__device__ double target_logpi(const DevModel& m, const float* x, const float* g, int q) {
    double s = 0.0;
    if constexpr (TARGET == 0) {
        for (int d = 0; d < m.D; ++d) s += ((double)x[d * FG + q] - (double)m.mu[d]) * (double)g[d * FG + q];
        return m.lconst + 0.5 * s;
    } else {
        for (int i = 0; i + 1 < m.D; i += 2) {
            const double xo = x[i * FG + q], xe = x[(i + 1) * FG + q];
            const double u = xe - m.h1 * (xo * xo - m.h0);
            s += -0.5 * xo * xo / m.h0 - 0.5 * u * u;
        }
        return s + m.lconst;
    }
}

// -------------------------------------------------------------- trajectories
template <int TARGET, bool MMA>
__global__ void __launch_bounds__(FT, 1) traj_flow_kernel(DevModel m, DevFlow f, TrajArgs a, float* z0out,
                                                          float* z1out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FlowSmem s = flow_smem(smem_raw, f.D, f.H, f.L, f.O4);
    s.pm = reinterpret_cast<__nv_bfloat16*>(s.ld + FG);   // past the FP64 block: flow_smem_bytes from the base
    // h1, h2, o and ch are contiguous: (3 H + O4) x 32 floats of scratch for P and mu
    const bool pfits = m.kind == GAUSS_DENSE && m.D * m.D + m.D <= (3 * f.H + f.O4) * FG;
    __shared__ int64_t j_s[FG], src_s[FG];
    __shared__ int S_s[FG];
    __shared__ float eps_s[FG];
    __shared__ uint64_t seed_s[FG];
    __shared__ uint32_t k_s[FG], jl_s[FG];
    __shared__ double H0_s[FG], lp_s[FG];
    __shared__ int smax_s;
    const int t = threadIdx.x, D = f.D;
    const int64_t slot0 = (int64_t)blockIdx.x * FG;
    if (t < FG) {
        const int64_t sl = slot0 + t;
        int64_t j = -1, src = -1;
        int S = 0;
        float ef = 0.0f;
        if (sl < a.N) {
            j = a.perm ? a.perm[sl] : sl;
            src = a.src ? a.src[j] : j;
            S = a.eval_only ? 0 : a.steps[j];
            int r;
            double eps;
            uint64_t seed;
            uint32_t kk, jl;
            particle_run(a, j, r, eps, seed, kk, jl);
            ef = (float)eps;
            seed_s[t] = seed;
            k_s[t] = kk;
            jl_s[t] = jl;
        }
        j_s[t] = j;
        src_s[t] = src;
        S_s[t] = S;
        eps_s[t] = ef;
    }
    __syncthreads();
    if (t == 0) {
        int mx = 0;
        for (int i = 0; i < FG; ++i) mx = max(mx, S_s[i]);
        smax_s = mx;
    }
    for (int e = t; e < D * FG; e += FT) {
        const int d = e / FG, q = e % FG;
        const int64_t src = src_s[q];
        s.x[e] = src >= 0 ? a.theta_in[(int64_t)d * a.ld + src] : 0.0f;
        s.c[e] = (src >= 0 && !a.eval_only) ? a.grad_in[(int64_t)d * a.ld + src] : 0.0f;
        s.p[e] = (src >= 0 && a.p_in && !a.eval_only) ? a.p_in[(int64_t)d * a.ld + j_s[q]] : 0.0f;
    }
    __syncthreads();
    if (a.eval_only) {
        // theta-space target evaluation (initial weights): no transport involved
        target_grad<TARGET>(m, s.x, s.gx, s.h1, pfits);
        __syncthreads();
        if (t < FG && j_s[t] >= 0) a.logpi_out[j_s[t]] = target_logpi<TARGET>(m, s.x, s.gx, t);
        for (int e = t; e < D * FG; e += FT) {
            const int d = e / FG, q = e % FG;
            if (j_s[q] >= 0) a.grad_out[(int64_t)d * a.ld + j_s[q]] = s.gx[e];
        }
        return;
    }
    const int smax = smax_s;
    // latent start z0 = T^-1(theta), its log pi_z and gradient
    flow_inverse<MMA>(f, s, s.x);                // s.x = z0, s.ld = log|det dT^-1|
    for (int e = t; e < D * FG; e += FT) s.z[e] = s.x[e];
    if (t < FG) lp_s[t] = (src_s[t] >= 0 ? a.logpi_in[src_s[t]] : 0.0) - s.ld[t];   // log pi_z(z0)
    __syncthreads();
    flow_backward<MMA>(f, s, s.c);               // s.c = grad_z log pi_z(z0)
    for (int e = t; e < D * FG; e += FT) s.gz[e] = s.c[e];
    if (!a.p_in) {
        const int npairs = (D + 1) / 2;
        for (int e = t; e < npairs * FG; e += FT) {
            const int i = e / FG, q = e % FG;
            if (j_s[q] < 0) continue;
            double z0, z1;
            normal_pair(seed_s[q], (uint32_t)i, jl_s[q], k_s[q], TAG_MOM, z0, z1);
            s.p[(2 * i) * FG + q] = (float)z0;
            if (2 * i + 1 < D) s.p[(2 * i + 1) * FG + q] = (float)z1;
        }
    }
    __syncthreads();
    if (t < FG) {
        double kin = 0.0;
        for (int d = 0; d < D; ++d) kin += (double)s.p[d * FG + t] * (double)s.p[d * FG + t];
        H0_s[t] = 0.5 * kin - lp_s[t];
    }
    if (z0out)
        for (int e = t; e < D * FG; e += FT) {
            const int d = e / FG, q = e % FG;
            if (j_s[q] >= 0) z0out[(int64_t)d * a.ld + j_s[q]] = s.z[e];
        }
    __syncthreads();
    // first half kick and drift
    for (int e = t; e < D * FG; e += FT) {
        const int q = e % FG;
        if (S_s[q] >= 1) {
            const float he = 0.5f * eps_s[q];
            const float pv = fmaf(he, s.gz[e], s.p[e]);
            s.p[e] = pv;
            s.z[e] = fmaf(eps_s[q], pv, s.z[e]);
        }
    }
    __syncthreads();
    for (int st = 1; st <= smax; ++st) {
        for (int e = t; e < D * FG; e += FT) s.x[e] = s.z[e];
        __syncthreads();
        flow_forward<MMA>(f, s, s.x);            // s.x = T(z), s.ld = log|det dT/dz|
        target_grad<TARGET>(m, s.x, s.gx, s.h1, pfits);       // grad_x log pi
        __syncthreads();
        for (int e = t; e < D * FG; e += FT) s.c[e] = s.gx[e];
        __syncthreads();
        flow_backward<MMA>(f, s, s.c);           // grad_z log pi_z
        for (int e = t; e < D * FG; e += FT) {
            const int q = e % FG;
            if (st <= S_s[q]) {
                const float he = 0.5f * eps_s[q];
                const float g = s.c[e];
                s.gz[e] = g;
                float pv = fmaf(he, g, s.p[e]);
                if (st + 1 <= S_s[q]) {
                    pv = fmaf(he, g, pv);
                    s.z[e] = fmaf(eps_s[q], pv, s.z[e]);
                }
                s.p[e] = pv;
            }
        }
        __syncthreads();
    }
    if (smax == 0) {   // nothing moved: restore theta and its gradient
        for (int e = t; e < D * FG; e += FT) {
            const int d = e / FG, q = e % FG;
            const int64_t src = src_s[q];
            s.x[e] = src >= 0 ? a.theta_in[(int64_t)d * a.ld + src] : 0.0f;
            s.gx[e] = src >= 0 ? a.grad_in[(int64_t)d * a.ld + src] : 0.0f;
        }
        if (t < FG) s.ld[t] = lp_s[t] - (src_s[t] >= 0 ? a.logpi_in[src_s[t]] : 0.0);
        __syncthreads();
    }
    // end point: theta' = T(z'), exact energy in FP64
    if (t < FG && j_s[t] >= 0) {
        const int64_t j = j_s[t];
        const double lpx = target_logpi<TARGET>(m, s.x, s.gx, t);
        const double lpz = lpx + s.ld[t];
        double kin = 0.0;
        for (int d = 0; d < D; ++d) kin += (double)s.p[d * FG + t] * (double)s.p[d * FG + t];
        double dH = (0.5 * kin - lpz) - H0_s[t];
        if (!isfinite(dH)) dH = CUDART_INF;
        a.logpi_out[j] = lpx;
        if (a.dH) a.dH[j] = dH;
        if (a.alpha) a.alpha[j] = dH <= 0.0 ? 1.0 : exp(-dH);
    }
    for (int e = t; e < D * FG; e += FT) {
        const int d = e / FG, q = e % FG;
        const int64_t j = j_s[q];
        if (j < 0) continue;
        a.theta_out[(int64_t)d * a.ld + j] = s.x[e];
        a.grad_out[(int64_t)d * a.ld + j] = s.gx[e];
        if (a.p_out) a.p_out[(int64_t)d * a.ld + j] = s.p[e];
        if (z1out) z1out[(int64_t)d * a.ld + j] = s.z[e];
    }
}

// -------------------------------------------------------------- training
// Per CTA of 32 particles: inverse pass, back-propagation of
// loss = sum_j W_j (1/2 |z_j|^2 + sum_l sum_k s_lk) through the inverse
// layers, and this CTA's share of every parameter gradient (canonical layout)
// into partials[blockIdx.x].
__device__ __forceinline__ float rot_dot(const float* A, const float* B, int lane) {
    // sum_p A[p] B[p] over the 32 particles, started at p = lane so that the
    // threads of a warp hit 32 different banks
    float acc = 0.0f;
#pragma unroll 8
    for (int u = 0; u < FG; ++u) {
        const int q = (u + lane) & 31;
        acc = fmaf(A[q], B[q], acc);
    }
    return acc;
}

// out[r] = sum over the CTA's 32 particles of X[row(r)][p] for r < R (the
// bias gradients): a warp per row, its lanes over the particles (one
// conflict-free load each), summed by shuffles in a fixed order.  CMAP: row
// r < Dh is X's row r, the others X's row Dh4 + (r - Dh) (the padded
// conditioner output).
template <bool CMAP>
__device__ __forceinline__ void row_sums(const float* X, int R, float* out, int Dh, int Dh4) {
    const int lane = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < R; r += FT / 32) {
        const int rp = CMAP ? (r < Dh ? r : Dh4 + (r - Dh)) : r;
        float v = X[rp * FG + lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) out[r] = v;
    }
}

__global__ void __launch_bounds__(FT, 1) k_flow_train(DevFlow f, const float* theta, int64_t ld,
                                                      const int32_t* src, const double* W, FlowGate gate, int64_t N,
                                                      float* partials) {
    if (!gate.open()) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FlowSmem s = flow_smem(smem_raw, f.D, f.H, f.L, f.O4);
    __shared__ float w_s[FG];
    const int t = threadIdx.x, lane = t & 31, D = f.D, H = f.H, Dh = f.Dh, Dh4 = f.Dh4;
    const int64_t slot0 = (int64_t)blockIdx.x * FG;
    if (t < FG) {
        const int64_t j = slot0 + t;
        float wv = 0.0f;
        if (j < N) {
            wv = (gate.rs && gate.rs->resample) ? (float)(1.0 / (double)gate.rp->n) : (float)W[j];
        }
        w_s[t] = wv;
    }
    __syncthreads();
    // a particle of zero weight adds nothing; its position may be non-finite
    // (the end of a divergent trajectory), so it enters as zeros
    for (int e = t; e < D * FG; e += FT) {
        const int d = e / FG, q = e % FG;
        const int64_t j = slot0 + q;
        s.x[e] = (j < N && w_s[q] != 0.0f) ? theta[(int64_t)d * ld + (src ? src[j] : j)] : 0.0f;
    }
    __syncthreads();
    // inverse pass; zl[l] = input of inverse layer l
    for (int l = f.L - 1; l >= 0; --l) {
        for (int e = t; e < D * FG; e += FT) s.zl[l * D * FG + e] = s.x[e];
        __syncthreads();
        conditioner(f, l, s.x, s);
        const int boff = (l & 1) ? 0 : Dh;
        for (int e = t; e < Dh * FG; e += FT) {
            const int k = e / FG, q = e % FG;
            const float sv = 2.0f * tanhf(s.o[k * FG + q]);
            const float tv = s.o[(Dh4 + k) * FG + q];
            s.x[(boff + k) * FG + q] = (s.x[(boff + k) * FG + q] - tv) * expf(-sv);
        }
        __syncthreads();
    }
    for (int e = t; e < D * FG; e += FT) s.c[e] = w_s[e % FG] * s.x[e];   // d(1/2 |z|^2) weighted
    __syncthreads();
    const int64_t lsz = (int64_t)H * Dh + H + (int64_t)H * H + H + (int64_t)D * H + D;
    const FlowLayerOff off = flow_layer_off(H, Dh, Dh4, f.O4);
    float* part = partials + (int64_t)blockIdx.x * f.n_params;
    for (int l = 0; l < f.L; ++l) {
        const float* in = s.zl + l * D * FG;
        const float* w = f.work + (int64_t)l * f.layer_work;
        float* gl = part + l * lsz;
        float *gW1 = gl, *gb1 = gW1 + (int64_t)H * Dh, *gW2 = gb1 + H, *gb2 = gW2 + (int64_t)H * H, *gW3 = gb2 + H,
              *gb3 = gW3 + (int64_t)D * H;
        conditioner(f, l, in, s);
        const int boff = (l & 1) ? 0 : Dh, aoff = (l & 1) ? Dh : 0;
        for (int e = t; e < Dh4 * FG; e += FT) {
            const int k = e / FG, q = e % FG;
            float cs_raw = 0.0f, ct = 0.0f;
            if (k < Dh) {
                const float th = tanhf(s.o[k * FG + q]);
                const float ems = expf(-2.0f * th);
                const float b = (in[(boff + k) * FG + q] - s.o[(Dh4 + k) * FG + q]) * ems;
                const float cb = s.c[(boff + k) * FG + q];
                const float cs = fmaf(-cb, b, w_s[q]);            // + W_j from sum s
                cs_raw = cs * 2.0f * (1.0f - th * th);
                ct = -cb * ems;
                s.c[(boff + k) * FG + q] = cb * ems;
            }
            s.o[k * FG + q] = cs_raw;
            s.o[(Dh4 + k) * FG + q] = ct;
        }
        __syncthreads();
        // dW3, db3 (canonical rows r: s rows 0..Dh-1, t rows Dh..D-1)
        for (int e = t; e < D * H; e += FT) {
            const int r = e / H, h = e % H;
            const int rp = r < Dh ? r : Dh4 + (r - Dh);
            gW3[(int64_t)r * H + h] = rot_dot(s.o + rp * FG, s.h2 + h * FG, lane);
        }
        row_sums<true>(s.o, D, gb3, Dh, Dh4);
        cta_mm<false, false>(w + off.W3, f.O4, H, s.o, s.ch, nullptr);
        __syncthreads();
        for (int e = t; e < H * FG; e += FT) s.ch[e] *= 1.0f - s.h2[e] * s.h2[e];   // c_h2
        __syncthreads();
        for (int e = t; e < H * H; e += FT) {
            const int r = e / H, h = e % H;
            gW2[(int64_t)r * H + h] = rot_dot(s.ch + r * FG, s.h1 + h * FG, lane);
        }
        row_sums<false>(s.ch, H, gb2, Dh, Dh4);
        cta_mm<false, false>(w + off.W2, H, H, s.ch, s.h2, nullptr);   // h2 no longer needed
        __syncthreads();
        for (int e = t; e < H * FG; e += FT) s.h2[e] *= 1.0f - s.h1[e] * s.h1[e];   // c_h1
        __syncthreads();
        for (int e = t; e < H * Dh; e += FT) {
            const int h = e / Dh, k = e % Dh;
            gW1[(int64_t)h * Dh + k] = rot_dot(s.h2 + h * FG, in + (aoff + k) * FG, lane);
        }
        row_sums<false>(s.h2, H, gb1, Dh, Dh4);
        cta_mm<false, false>(w + off.W1, H, Dh4, s.h2, s.ch, nullptr);
        __syncthreads();
        for (int e = t; e < Dh * FG; e += FT) s.c[aoff * FG + e] += s.ch[e];
        __syncthreads();
    }
}

// -------------------------------------------------------------- BF16 training
// The training step with every conditioner product on BF16 warp MMAs (FP32
// accumulation; master weights, bias sums, Adam and the coupling arithmetic
// stay FP32): the conditioner of the inverse pass and of the backward pass
// (as in the BF16 trajectories), the transposed products W3^T c_o, W2^T c_h2,
// W1^T c_h1 from the transposed fragments, and the weight gradients, which
// are products over the CTA's 32 particles, c [rows x 32] . act^T [32 x cols].
constexpr int WLD = FG + 8;      // row stride (BF16) of the weight-gradient operands

// FP32 rows X [R x 32] -> BF16 rows Y [Rpad][WLD] (particles contiguous),
// zero for R <= r < Rpad.  A thread converts eight particles of one row.
__device__ __noinline__ void to_rows(const float* X, int R, int Rpad, __nv_bfloat16* Y) {
    for (int e = threadIdx.x; e < Rpad * 4; e += FT) {
        const int r = e >> 2, p0 = 8 * (e & 3);
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (r < R) {
            const float4 a = *reinterpret_cast<const float4*>(X + r * FG + p0);
            const float4 b = *reinterpret_cast<const float4*>(X + r * FG + p0 + 4);
            const __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y), h1 = __floats2bfloat162_rn(a.z, a.w);
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(b.x, b.y), h3 = __floats2bfloat162_rn(b.z, b.w);
            w[0] = *reinterpret_cast<const uint32_t*>(&h0);
            w[1] = *reinterpret_cast<const uint32_t*>(&h1);
            w[2] = *reinterpret_cast<const uint32_t*>(&h2);
            w[3] = *reinterpret_cast<const uint32_t*>(&h3);
        }
        *reinterpret_cast<uint4*>(Y + r * WLD + p0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// out[row(m) * ldo + n] = sum over the CTA's 32 particles p of A[m][p] B[n][p]
// for m < 16 MT, n < min(16 NP, Nvalid); A, B BF16 rows [.][WLD] in shared
// memory (K = the particles: two k-steps of m16n8k16).  A warp takes one
// m-tile and four n-tiles.  CMAP: A's rows are the conditioner's padded
// output rows (s rows from 0, t rows from Dh4), stored at the canonical rows
// of W3 (s then t, Dh each); otherwise rows m < Mvalid are stored as they are.
template <bool CMAP>
__device__ __noinline__ void cta_wgrad(const __nv_bfloat16* A, int MT, const __nv_bfloat16* B, int NP, float* out,
                                       int ldo, int Mvalid, int Nvalid, int Dh, int Dh4) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int mi = lane >> 3, mr = lane & 7;
    const int NQ = (NP + 1) >> 1;
    const uint32_t abase = tc::smem_u32(A), bbase = tc::smem_u32(B);
    auto row_of = [&](int m) -> int {
        if (!CMAP) return m < Mvalid ? m : -1;
        return m < Dh ? m : (m >= Dh4 && m < Dh4 + Dh ? Dh + (m - Dh4) : -1);
    };
    for (int it = wid; it < MT * NQ; it += FT / 32) {
        const int mt = it / NQ, q = it % NQ;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            // A fragment: lanes 0-15 address rows 0-15 at k 0-7, lanes 16-31 the same rows at k 8-15
            uint32_t a[4];
            tc::ldsm4(a, abase + (uint32_t)(((16 * mt + (lane & 15)) * WLD + 16 * ks + 8 * (lane >> 4)) * 2));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int np = 2 * q + h;     // n-tiles 2 np and 2 np + 1
                if (np < NP) {
                    const int nrow = 16 * np + 8 * (mi >> 1) + mr;
                    const int kcol = 16 * ks + 8 * (mi & 1);
                    uint32_t b[4];
                    tc::ldsm4(b, bbase + (uint32_t)((nrow * WLD + kcol) * 2));
                    tc::mma_bf16_16816(acc[2 * h], a, b[0], b[1]);
                    tc::mma_bf16_16816(acc[2 * h + 1], a, b[2], b[3]);
                }
            }
        }
        const int r0 = row_of(16 * mt + g), r1 = row_of(16 * mt + g + 8);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (2 * q + (u >> 1) < NP) {
                const int c0 = 8 * (4 * q + u) + 2 * t;
                if (r0 >= 0) {
                    if (c0 < Nvalid) out[(int64_t)r0 * ldo + c0] = acc[u][0];
                    if (c0 + 1 < Nvalid) out[(int64_t)r0 * ldo + c0 + 1] = acc[u][1];
                }
                if (r1 >= 0) {
                    if (c0 < Nvalid) out[(int64_t)r1 * ldo + c0] = acc[u][2];
                    if (c0 + 1 < Nvalid) out[(int64_t)r1 * ldo + c0 + 1] = acc[u][3];
                }
            }
        }
    }
}

// Shared memory of the BF16 training kernel: FP32 x, c [D x 32], the layer
// inputs zl [L x D x 32], h1, h2 [H x 32], o [O4 x 32], ch [H x 32]; then the
// particle-major BF16 operand [32][<= 136] and the two row-major BF16
// operands of the weight-gradient products [128][WLD].
__device__ __forceinline__ FlowSmem flow_train_smem(unsigned char* base, int D, int H, int L, int O4,
                                                    __nv_bfloat16*& A16, __nv_bfloat16*& B16) {
    FlowSmem s{};
    float* f = reinterpret_cast<float*>(base);
    s.x = f;
    s.c = s.x + D * FG;
    s.zl = s.c + D * FG;
    s.h1 = s.zl + L * D * FG;
    s.h2 = s.h1 + H * FG;
    s.o = s.h2 + H * FG;
    s.ch = s.o + O4 * FG;
    s.pm = reinterpret_cast<__nv_bfloat16*>(s.ch + H * FG);
    A16 = s.pm + FG * (128 + 8);
    B16 = A16 + 128 * WLD;
    return s;
}

// The weighted-NLL gradient of k_flow_train with BF16 products; the same
// partials layout (canonical parameter order, one row per CTA).
__global__ void __launch_bounds__(FT, 1) k_flow_train_mma(DevFlow f, const float* theta, int64_t ld,
                                                          const int32_t* src, const double* W, FlowGate gate,
                                                          int64_t N, float* partials) {
    if (!gate.open()) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16 *A16, *B16;
    FlowSmem s = flow_train_smem(smem_raw, f.D, f.H, f.L, f.O4, A16, B16);
    __shared__ float w_s[FG];
    const int t = threadIdx.x, D = f.D, H = f.H, Dh = f.Dh, Dh4 = f.Dh4;
    const int64_t slot0 = (int64_t)blockIdx.x * FG;
    if (t < FG) {
        const int64_t j = slot0 + t;
        float wv = 0.0f;
        if (j < N) {
            wv = (gate.rs && gate.rs->resample) ? (float)(1.0 / (double)gate.rp->n) : (float)W[j];
        }
        w_s[t] = wv;
    }
    __syncthreads();
    for (int e = t; e < D * FG; e += FT) {
        const int d = e / FG, q = e % FG;
        const int64_t j = slot0 + q;
        s.x[e] = (j < N && w_s[q] != 0.0f) ? theta[(int64_t)d * ld + (src ? src[j] : j)] : 0.0f;
    }
    __syncthreads();
    for (int l = f.L - 1; l >= 0; --l) {
        for (int e = t; e < D * FG; e += FT) s.zl[l * D * FG + e] = s.x[e];
        __syncthreads();
        conditioner<true>(f, l, s.x, s);
        const int boff = (l & 1) ? 0 : Dh;
        for (int e = t; e < Dh * FG; e += FT) {
            const int k = e / FG, q = e % FG;
            const float sv = 2.0f * tanhf(s.o[k * FG + q]);
            const float tv = s.o[(Dh4 + k) * FG + q];
            s.x[(boff + k) * FG + q] = (s.x[(boff + k) * FG + q] - tv) * expf(-sv);
        }
        __syncthreads();
    }
    for (int e = t; e < D * FG; e += FT) s.c[e] = w_s[e % FG] * s.x[e];
    __syncthreads();
    const int64_t lsz = (int64_t)H * Dh + H + (int64_t)H * H + H + (int64_t)D * H + D;
    const FlowFragOff fo = flow_frag_off(H, f.kp1, f.o4p);
    float* part = partials + (int64_t)blockIdx.x * f.n_params;
    for (int l = 0; l < f.L; ++l) {
        const float* in = s.zl + l * D * FG;
        const uint4* fr = f.frag + (int64_t)l * f.layer_frag;
        float* gl = part + l * lsz;
        float *gW1 = gl, *gb1 = gW1 + (int64_t)H * Dh, *gW2 = gb1 + H, *gb2 = gW2 + (int64_t)H * H, *gW3 = gb2 + H,
              *gb3 = gW3 + (int64_t)D * H;
        conditioner<true>(f, l, in, s);
        const int boff = (l & 1) ? 0 : Dh, aoff = (l & 1) ? Dh : 0;
        for (int e = t; e < Dh4 * FG; e += FT) {
            const int k = e / FG, q = e % FG;
            float cs_raw = 0.0f, ct = 0.0f;
            if (k < Dh) {
                const float th = tanhf(s.o[k * FG + q]);
                const float ems = expf(-2.0f * th);
                const float b = (in[(boff + k) * FG + q] - s.o[(Dh4 + k) * FG + q]) * ems;
                const float cb = s.c[(boff + k) * FG + q];
                const float cs = fmaf(-cb, b, w_s[q]);
                cs_raw = cs * 2.0f * (1.0f - th * th);
                ct = -cb * ems;
                s.c[(boff + k) * FG + q] = cb * ems;
            }
            s.o[k * FG + q] = cs_raw;
            s.o[(Dh4 + k) * FG + q] = ct;
        }
        __syncthreads();
        // c_o: dW3 = c_o h2^T, db3 = row sums, c_h2 = (W3^T c_o) (1 - h2^2)
        to_rows(s.o, f.O4, f.o4p, A16);
        to_rows(s.h2, H, H, B16);
        to_pm(s.o, f.O4, f.o4p, s.pm, f.o4p + 8);
        __syncthreads();
        cta_wgrad<true>(A16, f.o4p / 16, B16, H / 16, gW3, H, 0, H, Dh, Dh4);
        row_sums<true>(s.o, D, gb3, Dh, Dh4);
        cta_mma<false, false>(fr + fo.W3t, H / 16, f.o4p / 16, s.pm, f.o4p + 8, s.ch, nullptr, H);
        __syncthreads();
        for (int e = t; e < H * FG; e += FT) s.ch[e] *= 1.0f - s.h2[e] * s.h2[e];
        __syncthreads();
        // c_h2: dW2 = c_h2 h1^T, db2, c_h1 = (W2^T c_h2) (1 - h1^2)
        to_rows(s.ch, H, H, A16);
        to_rows(s.h1, H, H, B16);
        to_pm(s.ch, H, H, s.pm, H + 8);
        __syncthreads();
        cta_wgrad<false>(A16, H / 16, B16, H / 16, gW2, H, H, H, Dh, Dh4);
        row_sums<false>(s.ch, H, gb2, Dh, Dh4);
        cta_mma<false, false>(fr + fo.W2t, H / 16, H / 16, s.pm, H + 8, s.h2, nullptr, H);   // h2 no longer needed
        __syncthreads();
        for (int e = t; e < H * FG; e += FT) s.h2[e] *= 1.0f - s.h1[e] * s.h1[e];
        __syncthreads();
        // c_h1: dW1 = c_h1 a^T, db1, c_a += W1^T c_h1
        to_rows(s.h2, H, H, A16);
        to_rows(in + aoff * FG, Dh, f.kp1, B16);
        to_pm(s.h2, H, H, s.pm, H + 8);
        __syncthreads();
        cta_wgrad<false>(A16, H / 16, B16, f.kp1 / 16, gW1, Dh, H, Dh, Dh, Dh4);
        row_sums<false>(s.h2, H, gb1, Dh, Dh4);
        cta_mma<false, false>(fr + fo.W1t, f.kp1 / 16, H / 16, s.pm, H + 8, s.ch, nullptr, Dh4);
        __syncthreads();
        for (int e = t; e < Dh * FG; e += FT) s.c[aoff * FG + e] += s.ch[e];
        __syncthreads();
    }
}

// grad[i] = sum over CTAs of partials[c][i], in CTA order.
__global__ void k_flow_reduce(const float* partials, int64_t n_blocks, int64_t n_params, float* grad,
                              FlowGate gate) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_params || !gate.open()) return;
    float acc = 0.0f;
    for (int64_t c = 0; c < n_blocks; ++c) acc += partials[c * n_params + i];
    grad[i] = acc;
}

__global__ void k_flow_adam(DevFlow f, float lr, FlowGate gate) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f.n_params || !gate.open()) return;
    const int32_t t = *f.adam_t + 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = f.grad[i];
    const float m = b1 * f.adam_m[i] + (1.0f - b1) * g;
    const float v = b2 * f.adam_v[i] + (1.0f - b2) * g * g;
    f.adam_m[i] = m;
    f.adam_v[i] = v;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    f.params[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

}  // namespace

bool flow_shape_ok(int64_t D, int64_t H, int64_t L) {
    if (D < 2 || (D & 1) || D > 128) return false;
    if (H < 4 || H > 128 || (H & 3) || L < 1 || L > 8) return false;
    const int64_t Dh4 = ((D / 2) + 3) & ~3ll;
    if (2 * Dh4 > 128) return false;
    if (H < Dh4) return false;   // the backward product into the input half writes Dh4 rows of an H-row buffer
    return flow_smem_bytes((int)D, (int)H, (int)L, (int)(2 * Dh4)) <= 220 * 1024;
}

bool flow_supported(const DevModel& m, int H, int L) {
    return (m.kind == GAUSS_DENSE || m.kind == BANANA) && flow_shape_ok(m.D, H, L);
}

bool flow_bf16_supported(int64_t D, int H, int L) {
    if (!flow_shape_ok(D, H, L) || !flow_bf16_ok(H)) return false;
    const int Dh4 = (int)(((D / 2) + 3) & ~3ll);
    return flow_smem_bytes((int)D, H, L, 2 * Dh4) + flow_pm_bytes() <= 226 * 1024;
}

static size_t flow_train_mma_smem_bytes(int D, int H, int L, int O4) {
    return sizeof(float) * (size_t)FG * (2 * D + L * D + 3 * H + O4) + flow_pm_bytes() +
           sizeof(uint16_t) * 2 * 128 * WLD;
}

bool flow_train_bf16_supported(int64_t D, int H, int L) {
    if (!flow_shape_ok(D, H, L) || !flow_bf16_ok(H)) return false;
    const int Dh4 = (int)(((D / 2) + 3) & ~3ll);
    return flow_train_mma_smem_bytes((int)D, H, L, 2 * Dh4) <= 226 * 1024;
}

DevFlow flow_shape(int D, int H, int L) {
    DevFlow f{};
    f.D = D;
    f.H = H;
    f.L = L;
    f.Dh = D / 2;
    f.Dh4 = (f.Dh + 3) & ~3;
    f.O4 = 2 * f.Dh4;
    f.kp1 = (f.Dh + 15) & ~15;
    f.o4p = (f.O4 + 15) & ~15;
    f.n_params = flow_num_params(D, H, L);
    f.layer_work = flow_layer_work(H, f.Dh, f.Dh4, f.O4);
    f.layer_frag = flow_bf16_ok(H) ? flow_frag_off(H, f.kp1, f.o4p).total : 0;
    return f;
}

cudaError_t flow_refresh(const DevFlow& f, cudaStream_t s, bool bump, FlowGate gate) {
    const int64_t total = (int64_t)f.L * f.layer_work;
    k_flow_refresh<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(f, bump, gate);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && f.frag && f.layer_frag > 0) {
        const int64_t nf = (int64_t)f.L * f.layer_frag;
        k_flow_frag<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(f);
        e = cudaGetLastError();
    }
    return e;
}

template <int TARGET, bool MMA>
static cudaError_t launch_flow_t(const DevModel& m, const DevFlow& f, const TrajArgs& a, float* z0, float* z1,
                                 int64_t grid, cudaStream_t s) {
    const size_t sm = flow_smem_bytes(f.D, f.H, f.L, f.O4) + (MMA ? flow_pm_bytes() : 0);
    auto kern = traj_flow_kernel<TARGET, MMA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, FT, sm, s>>>(m, f, a, z0, z1);
    return cudaGetLastError();
}

cudaError_t launch_traj_flow(const DevModel& m, const DevFlow& f, const TrajArgs& a, float* z0, float* z1,
                             cudaStream_t s) {
    const int64_t grid = (a.N + FG - 1) / FG;
    if (grid == 0) return cudaSuccess;
    const bool mma = f.bf16 != 0;
    if (mma && (!f.frag || f.layer_frag <= 0)) return cudaErrorInvalidValue;
    if (m.kind == GAUSS_DENSE)
        return mma ? launch_flow_t<0, true>(m, f, a, z0, z1, grid, s) : launch_flow_t<0, false>(m, f, a, z0, z1, grid, s);
    return mma ? launch_flow_t<1, true>(m, f, a, z0, z1, grid, s) : launch_flow_t<1, false>(m, f, a, z0, z1, grid, s);
}

int64_t flow_partials_floats(const DevFlow& f, int64_t N) { return ((N + FG - 1) / FG) * f.n_params; }

cudaError_t flow_loss_grad(const DevFlow& f, const float* theta, int64_t ld, const int32_t* src, const double* W,
                           FlowGate gate, int64_t N, float* partials, cudaStream_t s) {
    const int64_t grid = (N + FG - 1) / FG;
    if (grid == 0) return cudaSuccess;
    cudaError_t e;
    if (f.train_bf16) {
        if (!f.frag || f.layer_frag <= 0) return cudaErrorInvalidValue;
        const size_t sm = flow_train_mma_smem_bytes(f.D, f.H, f.L, f.O4);
        e = cudaFuncSetAttribute(k_flow_train_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_flow_train_mma<<<(unsigned)grid, FT, sm, s>>>(f, theta, ld, src, W, gate, N, partials);
    } else {
        const size_t sm = flow_smem_bytes(f.D, f.H, f.L, f.O4);
        e = cudaFuncSetAttribute(k_flow_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_flow_train<<<(unsigned)grid, FT, sm, s>>>(f, theta, ld, src, W, gate, N, partials);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_flow_reduce<<<(unsigned)((f.n_params + 255) / 256), 256, 0, s>>>(partials, grid, f.n_params, f.grad, gate);
    return cudaGetLastError();
}

cudaError_t flow_adam(const DevFlow& f, double lr, FlowGate gate, cudaStream_t s) {
    k_flow_adam<<<(unsigned)((f.n_params + 255) / 256), 256, 0, s>>>(f, (float)lr, gate);
    return cudaGetLastError();
}

}  // namespace smc
