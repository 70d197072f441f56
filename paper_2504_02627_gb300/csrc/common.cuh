// common.cuh -- device building blocks shared by the libsmcchees kernels.
//
// Counter-based random numbers (Philox4x32-10, Salmon et al., SC'11), the
// Box-Muller transform, the base-2 radical inverse used to jitter trajectory
// lengths (1-d Halton, Sec. 3.2 of arXiv 2504.02627), the step-count rule of
// Algorithm 2, and warp/block reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace smc {

// ---------------------------------------------------------------- run state
// Per-run parameters (read-only on the device during a step).
struct RunParams {
    int64_t off;            // first particle of the run in the global arrays
    int64_t n;              // particles in the run
    uint64_t seed;          // Philox key
    double eps;             // leapfrog step size
    double ess_frac;        // resampling threshold (fraction of n)
    double init_scale;      // q_init standard deviation
    double adam_lr, adam_b1, adam_b2, adam_eps;
    double log_L_lo, log_L_hi;   // clamp of log L: [log eps, log(max_steps * eps)]
    int32_t max_steps;
    int32_t jitter;
    int32_t adapt;
    int32_t n_tiles;        // resampling scan tiles of this run
    int64_t tile0;          // first global scan tile of the run
    int64_t n_iters, n_warmup;
    int32_t slice0;         // first particle slice (SLICE particles) of the run
    int32_t n_slices;
    int32_t accept_reject;  // 1: Metropolis select after the move, weight unchanged
    int32_t resample_scheme;   // 0 systematic, 1 multinomial
    double step_rate;       // optional warm-up step-size rule: log eps += step_rate (a_h - step_target)
    double step_target;
    int32_t mcmc;           // 1: Algorithm 2 as independent chains (no importance weights)
    int32_t init_general;   // 1: q_init = N(init_mean, init_chol init_chol') (either may be null)
    const double* init_mean;    // [D] device copy, or null (0)
    const double* init_chol;    // [D x D] device copy, row-major lower-triangular, or null (init_scale I)
    double init_logdet;     // sum_d log L_dd (D log init_scale without a factor)
};

constexpr int SLICE = 128;  // particles per CTA in the weight / statistics kernels (four warps:
                             // their FP64 work spreads over twice as many SMs as 256 would)

// Per-run mutable state (device).  The first 9 doubles are what
// smc_get_buffer(RUNSTATE) returns.
struct RunState {
    double log_z;       // running log evidence
    double log_L;       // log trajectory length (Adam variable)
    double adam_m, adam_v;
    double Lbar;        // moving average of L
    double adam_t;      // Adam step count (stored as double for the readout)
    double L_last;      // L used by the last completed iteration
    double ess;         // ESS after the last reweighting
    double eps;         // leapfrog step size of the iteration about to run (the
                        // configured one unless the step-size rule is on)
    // ---- decision for the iteration about to run (written by the previous
    //      iteration's finisher or by the initial weighting)
    double lse;         // log-sum-exp of the current log-weights
    double ess_pre;     // their ESS
    double L_used;      // L for this iteration's jitter
    unsigned long long T;   // sum of the fixed-point weights (atomic, exact)
    unsigned long long r64; // systematic-resampling uniform of this iteration
    int64_t k;          // 1-based iteration about to run
    int32_t resample;   // this iteration resamples
    int32_t status;     // 0 ok, -4 degenerate, -5 look-back gave up
    // ---- statistics of the last completed iteration
    double stat_ess_pre, log_z_inc, mean_alpha;
    int64_t grad_evals;
    int32_t stat_resampled, steps_min, steps_max, pad;
    // ---- cumulative counters since the initial draw
    int64_t iters_total, grad_evals_total, resamples_total;
    double ess_sum, ess_sum_post;
    // Adam bias-correction powers b1^t, b2^t, kept as running products
    double adam_b1t, adam_b2t;
};

// ---------------------------------------------------------------- Philox4x32-10
// Round: the 32x32->64 products of counter words 0 and 2 with the round
// multipliers; new words are (hi(c2*M1) ^ c1 ^ k0, lo(c2*M1), hi(c0*M0) ^ c3 ^ k1,
// lo(c0*M0)); the key advances by the Weyl increments (golden ratio and
// sqrt(3) - 1 as 32-bit fractions) after each of the ten rounds.
struct Philox4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ Philox4 philox4x32_10(Philox4 c, uint64_t seed) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        uint64_t a = (uint64_t)0xD2511F53u * c.x, b = (uint64_t)0xCD9E8D57u * c.z;
        uint32_t hi0 = (uint32_t)(a >> 32), lo0 = (uint32_t)a;
        uint32_t hi1 = (uint32_t)(b >> 32), lo1 = (uint32_t)b;
#endif
        c = Philox4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

enum : uint32_t { TAG_INIT = 1, TAG_MOM = 2, TAG_RESAMPLE = 3, TAG_MH = 4, TAG_JITTER = 5, TAG_SHUFFLE = 6 };

// Uniform on (0,1): 26 high bits of each word form a 52-bit integer m and the
// value is (m + 0.5) 2^-52, exact in FP64.
__device__ __forceinline__ double u01_52(uint32_t a, uint32_t b) {
    uint64_t m = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
    return ((double)m + 0.5) * 2.220446049250313080847263336181640625e-16;  // 2^-52
}

// Two standard normals from one Philox block by Box-Muller in FP64.
__device__ __forceinline__ void normal_pair(uint64_t seed, uint32_t i, uint32_t j, uint32_t k,
                                            uint32_t tag, double& z0, double& z1) {
    Philox4 w = philox4x32_10(Philox4{i, j, k, tag}, seed);
    double u1 = u01_52(w.x, w.y), u2 = u01_52(w.z, w.w);
    double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// The same pair from the same Philox block with the transform in FP32.  Each
// uniform is the FP64 pair's (m + 1/2) 2^-52 (m the same 52-bit integer)
// rounded to FP32 with relative error below 2^-23: the high 24 bits of m are
// exact in FP32, the low 28 bits plus the half are converted once and added
// with one rounding.  Keeping the relative precision of u1 matters in the
// tail, where log u1 amplifies it.  FP32 log, sqrt and sincospi then put the
// pair within about 1e-7 relative of the FP64 one; used where a thread draws
// whole particles' momenta, since FP64 runs at a small fraction of the FP32
// rate on this GPU.
__device__ __forceinline__ float u01_52_f32(uint32_t a, uint32_t b) {
    const float hi = (float)(a >> 8);                                    // bits 51..28 of m
    const float lo = (float)((((a >> 6) & 3u) << 26) | (b >> 6)) + 0.5f;  // bits 27..0, plus 1/2
    return fmaf(lo, 3.7252902984619140625e-9f, hi) * 5.9604644775390625e-8f;   // (hi + lo 2^-28) 2^-24
}
__device__ __forceinline__ void normal_pair_f32(uint64_t seed, uint32_t i, uint32_t j, uint32_t k,
                                                uint32_t tag, float& z0, float& z1) {
    Philox4 w = philox4x32_10(Philox4{i, j, k, tag}, seed);
    const float u1 = u01_52_f32(w.x, w.y), u2 = u01_52_f32(w.z, w.w);
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// ---------------------------------------------------------------- jitter
// Base-2 radical inverse of n: bit reversal of the 32-bit integer, times 2^-32
// (exact in FP64 for n < 2^32).
__device__ __forceinline__ double halton2(uint32_t n) {
    return (double)__brev(n) * 2.3283064365386962890625e-10;  // 2^-32
}

// Radical inverse of n in base b (Halton 1960): the base-b digits of n
// reversed behind the point, as the exact fraction rev / b^digits rounded once
// (both integers stay below 2^53 for n <= 2^30 and b below 2^20).
__device__ __forceinline__ double radical_inverse(uint64_t n, uint64_t b) {
    uint64_t num = 0, den = 1;
    while (n != 0) {
        num = num * b + n % b;
        den *= b;
        n /= b;
    }
    return __ddiv_rn((double)num, (double)den);
}

// Shuffle of iteration k, a bijection of {0..J-1} (1 <= J <= 2^30): a
// four-round Feistel network on 2 ceil(log4 J) bits, round r mixing in word 0
// of Philox block (x, r, k, SHUFFLE) masked to half the bits, applied to j
// until the value falls below J (cycle walking; the orbit of j < J returns
// below J, within the 2^bits bound of the loop).
__device__ __forceinline__ uint32_t shuffle_index(uint64_t seed, uint32_t k, uint32_t j, uint32_t J) {
    int m = 2;
    while ((1ull << m) < (unsigned long long)J) m += 2;
    const int half = m / 2;
    const uint32_t mask = (1u << half) - 1u;
    uint32_t v = j;
    for (uint64_t it = 0; it < (1ull << m); ++it) {
        uint32_t L = v >> half, R = v & mask;
#pragma unroll
        for (uint32_t r = 0; r < 4; ++r) {
            const uint32_t t = L ^ (philox4x32_10(Philox4{R, r, k, TAG_SHUFFLE}, seed).x & mask);
            L = R;
            R = t;
        }
        v = (L << half) | R;
        if (v < J) return v;
    }
    return j;
}

__device__ __forceinline__ double frac_rn(double x) { return __dsub_rn(x, floor(x)); }

// Jitter h of particle i (0-based within its run, the paper's j - 1) at
// iteration k (1-based), J particles, K iterations (Sec. 3.2.1): 0 none; 1
// 1-d Halton of n = iK + k; 2 uniform (Philox block (0, i, k, JITTER)); 3 / 4
// N-d Halton of i + 1 in base P_k / P_{K+1-k}; 5 / 6 N-d primes
// frac((i + 1) sqrt(P_k)) / P_{K+1-k}; 7 golden ratio frac((iK + k)(sqrt 5 -
// 1)/2); 8 equidistant (shuffle_k(i) + 1) / J; 9 offset equidistant: that +
// 0.1 u (Philox block (1, i, k, JITTER)); 10 1-d Sobol: radical inverse base
// 2 of the Gray code of iK + k; 11 1-d Halton in iteration-major order, base 2
// radical inverse of (k - 1) J + i + 1.  primes[m - 1] is the m-th prime (schemes
// 3-6, which reuse their K dimensions cyclically past iteration K).  Every
// FP64 operation is rounded once, in the order written.
__device__ __forceinline__ double jitter_h(int32_t scheme, uint64_t seed, int64_t i, int64_t k, int64_t J,
                                          int64_t K, const int32_t* primes) {
    if (scheme >= 3 && scheme <= 6) k = (k - 1) % K + 1;
    switch (scheme) {
        case 0: return 1.0;
        case 1: return halton2((uint32_t)(i * K + k));
        case 2: {
            const Philox4 w = philox4x32_10(Philox4{0u, (uint32_t)i, (uint32_t)k, TAG_JITTER}, seed);
            return u01_52(w.x, w.y);
        }
        case 3: return radical_inverse((uint64_t)(i + 1), (uint64_t)primes[k - 1]);
        case 4: return radical_inverse((uint64_t)(i + 1), (uint64_t)primes[K - k]);
        case 5:
        case 6: {
            const int32_t p = primes[scheme == 5 ? k - 1 : K - k];
            return frac_rn(__dmul_rn((double)(i + 1), __dsqrt_rn((double)p)));
        }
        case 7: {
            const double g = __dmul_rn(__dsub_rn(__dsqrt_rn(5.0), 1.0), 0.5);
            return frac_rn(__dmul_rn((double)(i * K + k), g));
        }
        case 8:
        case 9: {
            double h = __ddiv_rn((double)(shuffle_index(seed, (uint32_t)k, (uint32_t)i, (uint32_t)J) + 1), (double)J);
            if (scheme == 9) {
                const Philox4 w = philox4x32_10(Philox4{1u, (uint32_t)i, (uint32_t)k, TAG_JITTER}, seed);
                h = __dadd_rn(h, __dmul_rn(0.1, u01_52(w.x, w.y)));
            }
            return h;
        }
        case 10: {
            const uint32_t n = (uint32_t)(i * K + k);
            return halton2(n ^ (n >> 1));
        }
        case 11: return halton2((uint32_t)((k - 1) * J + i + 1));
        default: return 1.0;
    }
}

// Algorithm 2: ceil(h L / eps), at least 1 and at most max_steps.
__device__ __forceinline__ int32_t step_count(double h, double L, double eps, int32_t max_steps) {
    double s = ceil(__ddiv_rn(__dmul_rn(h, L), eps));
    if (!(s >= 1.0)) return 1;
    if (s >= (double)max_steps) return max_steps;
    return (int32_t)s;
}

// ---------------------------------------------------------------- FP32 pairs
// An unevaluated pair hi + lo of FP32 values carries about 48 significant
// bits.  Sums use Knuth's TwoSum and products the FMA form of Dekker's
// TwoProduct (both error-free transformations); pair + pair follows the
// accurate double-double addition of Hida, Li and Bailey.  On this GPU FP64
// runs at about 1/64 of the FP32 rate, so the statistics kernels accumulate
// in pairs and convert to FP64 once per partial sum.
struct f2sum {
    float hi, lo;
};
__device__ __forceinline__ f2sum two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ f2sum quick_two_sum(float a, float b) {   // needs |a| >= |b| or a = 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2sum f2_add(f2sum x, f2sum y) {
    f2sum s = two_sum(x.hi, y.hi);
    const f2sum t = two_sum(x.lo, y.lo);
    s = quick_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return quick_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ f2sum f2_add_f(f2sum x, float y) {
    const f2sum s = two_sum(x.hi, y);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
__device__ __forceinline__ f2sum f2_mul(f2sum x, f2sum y) {           // lo * lo dropped
    const float p = __fmul_rn(x.hi, y.hi);
    const float e = __fmaf_rn(x.hi, y.hi, -p);                          // exact error of p
    return quick_two_sum(p, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e)));
}
__device__ __forceinline__ double f2_to_double(f2sum x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ f2sum f2_from_double(double v) {
    const float hi = __double2float_rn(v);
    return {hi, __double2float_rn(v - (double)hi)};
}
// butterfly sum over the warp (pair addition is commutative bit for bit)
__device__ __forceinline__ f2sum warp_sum_f2(f2sum v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const f2sum w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = f2_add(v, w);
    }
    return v;
}

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Warp sums of 16 values per lane: on return each lane holds the total over
// the 32 lanes of value (lane >> 1) & 15.  A reduce-scatter butterfly: at
// each level a lane keeps half of its values and adds the partner's copy of
// that half, 16 additions per lane instead of 80 for 16 separate butterflies.
// The order is fixed, and both lanes of a pair get the same bits.
__device__ __forceinline__ double warp_sum16_scatter(double (&v)[16], int lane) {
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const bool up = (lane & (2 * h)) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const double send = up ? v[k] : v[k + h];
            const double keep = up ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * h);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Block-wide reduction through shared memory; every thread gets the result.
// `buf` needs blockDim.x / 32 entries.
template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, T* buf, Op op) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) buf[wid] = v;
    __syncthreads();
    T r = buf[0];
    for (int w = 1; w < nw; ++w) r = op(r, buf[w]);
    return r;
}

// N block reductions in one pass: every value goes through the same
// shuffle tree and the same warp-by-warp combination as block_reduce, so each
// result has the bits block_reduce would give it, while the N dependency
// chains overlap and share two barriers.  `buf` needs N * 32 entries.
template <int N, typename T, typename Op>
__device__ __forceinline__ void block_reduce_n(T (&v)[N], T* buf, Op op) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = op(v[i], __shfl_xor_sync(0xffffffffu, v[i], o));
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) buf[i * 32 + wid] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T r = buf[i * 32];
        for (int w = 1; w < nw; ++w) r = op(r, buf[i * 32 + w]);
        v[i] = r;
    }
}

struct OpSum { template <typename T> __device__ T operator()(T a, T b) const { return a + b; } };
struct OpMax { template <typename T> __device__ T operator()(T a, T b) const { return a > b ? a : b; } };
struct OpMin { template <typename T> __device__ T operator()(T a, T b) const { return a < b ? a : b; } };

}  // namespace smc
