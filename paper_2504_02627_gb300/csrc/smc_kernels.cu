// smc_kernels.cu -- the SMC stages around the trajectories (Algorithm 3 of
// arXiv 2504.02627): initial draw and weights, weight normalisation and ESS,
// fixed-point systematic resampling with a decoupled look-back scan, Halton
// jitter and step counts with a counting sort by step count, and the
// reweighting / evidence / ChEES-adaptation epilogue.
#include <math_constants.h>
#include "smc_kernels.cuh"

namespace smc {

constexpr int RUN_THREADS = 1024;
constexpr double LOG_2PI = 1.8378770664093454835606594728112;

// ============================================================ initial draw
// theta_0 ~ q_init = N(0, s^2 I) (Eq. for theta_0), and log q_init(theta_0)
// parked in logw until the target has been evaluated.
__global__ void k_init_draw(StepBufs b, float* theta) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= b.N) return;
    const int r = b.run_of[j];
    const RunParams rp = b.runs[r];
    const uint32_t jl = (uint32_t)(j - rp.off);
    double zz = 0.0;
    for (int64_t d = 0; d < b.D; d += 2) {
        double z0, z1;
        normal_pair(rp.seed, (uint32_t)(d >> 1), jl, 0u, TAG_INIT, z0, z1);
        theta[d * b.ld + j] = (float)(rp.init_scale * z0);
        zz += z0 * z0;
        if (d + 1 < b.D) {
            theta[(d + 1) * b.ld + j] = (float)(rp.init_scale * z1);
            zz += z1 * z1;
        }
    }
    b.logw[j] = -0.5 * zz - 0.5 * (double)b.D * (LOG_2PI + 2.0 * log(rp.init_scale));
}

// w_1 = pi(theta_0) / q_init(theta_0) (Eq. for w_1); log Z_0 = LSE(log w) - log J.
__global__ void __launch_bounds__(RUN_THREADS) k_init_finish(StepBufs b, const double* logpi) {
    __shared__ double buf[32];
    const int r = blockIdx.x;
    const RunParams rp = b.runs[r];
    double m = -CUDART_INF;
    for (int64_t i = threadIdx.x; i < rp.n; i += blockDim.x) {
        const int64_t j = rp.off + i;
        const double lp = logpi[j];
        const double lw = isfinite(lp) ? lp - b.logw[j] : -CUDART_INF;
        b.logw[j] = lw;
        m = fmax(m, lw);
    }
    m = block_reduce(m, buf, OpMax());
    double s = 0.0;
    if (m > -CUDART_INF)
        for (int64_t i = threadIdx.x; i < rp.n; i += blockDim.x) s += exp(b.logw[rp.off + i] - m);
    s = block_reduce(s, buf, OpSum());
    if (threadIdx.x == 0) {
        RunState& st = b.rstate[r];
        st.log_z = (m > -CUDART_INF) ? m + log(s) - log((double)rp.n) : -CUDART_INF;
        st.status = (m > -CUDART_INF) ? 0 : -4;
    }
}

// ============================================================ normalise + ESS
// Normalised weights W = w / sum w (Eq. for the normalised weights), J_eff =
// 1 / sum W^2 (Eq. for J_eff), the resampling test J_eff < frac J, and, when
// resampling, the fixed-point weights q_j = floor(W_j 2^S), their exact total
// T and the systematic offset U = floor(r64 T / 2^64).
__global__ void __launch_bounds__(RUN_THREADS) k_normalise(StepBufs b) {
    __shared__ double buf[32];
    __shared__ unsigned long long ubuf[32];
    const int r = blockIdx.x;
    const RunParams rp = b.runs[r];
    RunState& st = b.rstate[r];
    if (r == 0 && threadIdx.x == 0) {
        b.counter[0] = 0u;          // dynamic scan-tile counter
        b.counter[1] += 1u;         // look-back epoch: never repeats within a handle
    }
    if (st.status != 0) {
        if (threadIdx.x == 0) st.resample = 0;
        return;
    }
    const double* lw = b.logw + rp.off;
    double m = -CUDART_INF;
    for (int64_t i = threadIdx.x; i < rp.n; i += blockDim.x) m = fmax(m, lw[i]);
    m = block_reduce(m, buf, OpMax());
    if (!(m > -CUDART_INF)) {
        if (threadIdx.x == 0) {
            st.status = -4;
            st.resample = 0;
        }
        return;
    }
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < rp.n; i += blockDim.x) s += exp(lw[i] - m);
    s = block_reduce(s, buf, OpSum());
    const double lse = m + log(s);
    double s2 = 0.0;
    for (int64_t i = threadIdx.x; i < rp.n; i += blockDim.x) {
        const double w = exp(lw[i] - lse);
        b.W[rp.off + i] = w;
        s2 += w * w;
    }
    s2 = block_reduce(s2, buf, OpSum());
    const double ess = 1.0 / s2;
    const int resample = ess < rp.ess_frac * (double)rp.n;
    unsigned long long T = 0ull;
    if (resample) {
        int c = 0;
        while (((int64_t)1 << c) < rp.n) ++c;
        const double scale = ldexp(1.0, 62 - c);
        for (int64_t i = threadIdx.x; i < rp.n; i += blockDim.x) {
            const double v = b.W[rp.off + i] * scale;
            const unsigned long long qi = v > 0.0 ? __double2ull_rz(v) : 0ull;
            b.q[rp.off + i] = qi;
            T += qi;
        }
        T = block_reduce(T, ubuf, OpSum());
    }
    if (threadIdx.x == 0) {
        st.lse = lse;
        st.ess_pre = ess;
        st.resample = resample;
        st.L_used = exp(st.log_L);
        if (resample) {
            const Philox4 w = philox4x32_10(Philox4{0u, 0u, (uint32_t)st.k, TAG_RESAMPLE}, rp.seed);
            const unsigned long long r64 = ((unsigned long long)w.x << 32) | w.y;
            st.T = T;
            st.U = __umul64hi(r64, T);
            if (T == 0ull) {
                st.status = -4;
                st.resample = 0;
            }
        }
    }
}

// ============================================================ resampling scan
// Inclusive prefix C of q within each run by a single-pass decoupled
// look-back scan (tiles of SCAN_TILE elements; a tile id is taken from an
// atomic counter, so every predecessor tile has already started).  Each
// particle j then owns the output slots i with N C_{j-1} <= i T + U < N C_j,
// i.e. [cnt(C_{j-1}), cnt(C_j)) with cnt(C) = ceil((N C - U) / T) clipped to
// [0, N], and writes its own index there (systematic resampling).
constexpr long long LOOKBACK_SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ unsigned long long systematic_count(unsigned long long C, unsigned long long N,
                                                               unsigned long long T, unsigned long long U) {
    const unsigned long long NC = N * C;
    if (NC <= U) return 0ull;
    const unsigned long long c = (NC - U + T - 1ull) / T;
    return c < N ? c : N;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_resample_scan(StepBufs b) {
    __shared__ unsigned int tile_s;
    __shared__ unsigned long long wsum[SCAN_THREADS / 32];
    __shared__ unsigned long long excl_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) tile_s = atomicAdd(b.counter, 1u);
    __syncthreads();
    const int64_t g = tile_s;
    if (g >= b.n_tiles) return;
    const int r = b.tile_run ? b.tile_run[g] : 0;
    const RunParams rp = b.runs[r];
    RunState& st = b.rstate[r];
    if (!st.resample) return;
    const unsigned int epoch = b.counter[1] & 0x3fffffffu;
    const int64_t t_in_run = g - rp.tile0;
    const int64_t base = t_in_run * SCAN_TILE;
    const unsigned long long N = (unsigned long long)rp.n, T = st.T, U = st.U;

    // thread-local inclusive prefix of SCAN_ITEMS consecutive elements
    unsigned long long v[SCAN_ITEMS];
    unsigned long long acc = 0ull;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + (int64_t)tid * SCAN_ITEMS + k;
        const unsigned long long x = i < rp.n ? b.q[rp.off + i] : 0ull;
        acc += x;
        v[k] = acc;
    }
    // block exclusive scan of the per-thread totals
    unsigned long long x = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = lane < SCAN_THREADS / 32 ? wsum[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_THREADS / 32) wsum[lane] = w;
    }
    __syncthreads();
    const unsigned long long thread_excl = (x - acc) + (wid > 0 ? wsum[wid - 1] : 0ull);
    const unsigned long long tile_agg = wsum[SCAN_THREADS / 32 - 1];

    // look-back over predecessor tiles of the same run
    if (tid == 0) {
        TileDesc* me = b.tiles + g;
        unsigned long long excl = 0ull;
        if (t_in_run == 0) {
            me->incl = tile_agg;
            __threadfence();
            atomicExch(&me->flag, (epoch << 2) | 2u);
        } else {
            me->agg = tile_agg;
            __threadfence();
            atomicExch(&me->flag, (epoch << 2) | 1u);
            int64_t pred = g - 1;
            long long spins = 0;
            while (true) {
                const volatile TileDesc* pd = b.tiles + pred;
                const unsigned int f = pd->flag;
                if ((f >> 2) == epoch && (f & 3u) != 0u) {
                    __threadfence();
                    if ((f & 3u) == 2u) {
                        excl += pd->incl;
                        break;
                    }
                    excl += pd->agg;
                    --pred;
                    spins = 0;
                    continue;
                }
                if (++spins > LOOKBACK_SPIN_LIMIT) {   // bounded wait: report, never hang
                    st.status = -5;
                    break;
                }
                __nanosleep(64);
            }
            me->incl = excl + tile_agg;
            __threadfence();
            atomicExch(&me->flag, (epoch << 2) | 2u);
        }
        excl_s = excl;
    }
    __syncthreads();
    const unsigned long long off = excl_s + thread_excl;
    // scatter: particle i of the run owns output slots [cnt(C_{i-1}), cnt(C_i))
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + (int64_t)tid * SCAN_ITEMS + k;
        if (i >= rp.n) break;
        const unsigned long long Ci = off + v[k];
        const unsigned long long Cp = Ci - b.q[rp.off + i];
        const unsigned long long lo = systematic_count(Cp, N, T, U), hi = systematic_count(Ci, N, T, U);
        for (unsigned long long o = lo; o < hi; ++o) b.anc[rp.off + (int64_t)o] = (int32_t)i;
    }
}

// ============================================================ jitter + sort
// h_j = radical inverse base 2 of n = j K + k (1-d Halton, Sec. 3.2), S_j =
// ceil(h_j L / eps) (Algorithm 2), the source index of each particle after
// resampling, and a histogram of S_j for the counting sort.
__global__ void k_steps(StepBufs b) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= b.N) return;
    const int r = b.run_of[j];
    const RunParams& rp = b.runs[r];
    const RunState& st = b.rstate[r];
    const int64_t jl = j - rp.off;
    b.src[j] = st.resample ? (int32_t)(rp.off + b.anc[j]) : (int32_t)j;
    const double h = rp.jitter ? halton2((uint32_t)(jl * rp.n_iters + st.k)) : 1.0;
    const int32_t S = st.status == 0 ? step_count(h, st.L_used, rp.eps, rp.max_steps) : 0;
    b.steps[j] = S;
    atomicAdd(&b.hist[b.max_steps_all - S], 1);
}

// Exclusive scan of the histogram (one CTA), in place.
__global__ void __launch_bounds__(1024) k_hist_scan(StepBufs b) {
    __shared__ int wsum[32];
    const int nb = b.max_steps_all + 1;
    int carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? b.hist[i] : 0;
        int x = v;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int excl = carry + (x - v) + (wid > 0 ? wsum[wid - 1] : 0);
        const int total = wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
        if (i < nb) b.hist[i] = excl;
        carry += total;
    }
}

// Slot of each particle in descending-step order, so that particles with
// similar trajectory lengths share a CTA / warp in the trajectory kernels.
__global__ void k_sort_scatter(StepBufs b) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= b.N) return;
    const int slot = atomicAdd(&b.hist[b.max_steps_all - b.steps[j]], 1);
    b.perm[slot] = (int32_t)j;
}

// ============================================================ reweight + ChEES
// Incremental weight with the momentum change-of-variable L-kernel: the
// Jacobians cancel and log w += -Delta H (Sec. 3.1); the evidence factor is
// sum_j W_j exp(-Delta H_j).  During warm-up the ChEES gradient
// g_j = l_j (|t1_j - mean t1|^2 - |t0_j - mean t0|^2) (t1_j - mean t1)' p_j
// (Algorithm 2) is averaged with weights alpha_j and fed to Adam on log L;
// Lbar <- 0.9 Lbar + 0.1 L; at k = M_warmup, L <- Lbar.
__global__ void __launch_bounds__(RUN_THREADS) k_reweight_chees(StepBufs b) {
    __shared__ double buf[32];
    __shared__ int ibuf[32];
    __shared__ double mean0[1024], mean1[1024];
    const int r = blockIdx.x;
    const RunParams rp = b.runs[r];
    RunState& st = b.rstate[r];
    if (st.status != 0) return;
    const int64_t n = rp.n, off = rp.off;
    const int resample = st.resample;
    const double lse = st.lse, logn = log((double)n);

    // (f) evidence factor and new log-weights
    double m = -CUDART_INF;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t j = off + i;
        const double lw = (resample ? -logn : b.logw[j] - lse) - b.dH[j];
        m = fmax(m, lw);
    }
    m = block_reduce(m, buf, OpMax());
    double s = 0.0, sa = 0.0;
    long long ge = 0;
    int smin = 0x7fffffff, smax = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t j = off + i;
        const double lw = (resample ? -logn : b.logw[j] - lse) - b.dH[j];
        if (m > -CUDART_INF) s += exp(lw - m);
        sa += b.alpha[j];
        const int Sj = b.steps[j];
        ge += Sj;
        smin = min(smin, Sj);
        smax = max(smax, Sj);
    }
    s = block_reduce(s, buf, OpSum());
    sa = block_reduce(sa, buf, OpSum());
    ge = block_reduce(ge, reinterpret_cast<long long*>(buf), OpSum());
    smin = block_reduce(smin, ibuf, OpMin());
    smax = block_reduce(smax, ibuf, OpMax());
    const double log_z_inc = (m > -CUDART_INF) ? m + log(s) : -CUDART_INF;
    // new unnormalised log-weights, then their ESS
    double m2 = -CUDART_INF;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t j = off + i;
        const double lw = (resample ? -logn : b.logw[j]) - b.dH[j];
        b.logw[j] = lw;
        m2 = fmax(m2, lw);
    }
    m2 = block_reduce(m2, buf, OpMax());
    double e1 = 0.0, e2 = 0.0;
    if (m2 > -CUDART_INF)
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const double w = exp(b.logw[off + i] - m2);
            e1 += w;
            e2 += w * w;
        }
    e1 = block_reduce(e1, buf, OpSum());
    e2 = block_reduce(e2, buf, OpSum());

    // (g) ChEES adaptation during warm-up
    const int64_t k = st.k;
    if (rp.adapt && k < rp.n_warmup) {
        const int64_t D = b.D;
        for (int64_t d = threadIdx.x; d < D; d += blockDim.x) {
            mean0[d] = 0.0;
            mean1[d] = 0.0;
        }
        __syncthreads();
        for (int64_t d = 0; d < D; ++d) {
            double a0 = 0.0, a1 = 0.0;
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                const int64_t j = off + i;
                a0 += (double)b.theta_prev[d * b.ld + b.src[j]];
                a1 += (double)b.theta_new[d * b.ld + j];
            }
            a0 = warp_sum(a0);
            a1 = warp_sum(a1);
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&mean0[d], a0);
                atomicAdd(&mean1[d], a1);
            }
        }
        __syncthreads();
        for (int64_t d = threadIdx.x; d < D; d += blockDim.x) {
            mean0[d] /= (double)n;
            mean1[d] /= (double)n;
        }
        __syncthreads();
        double num = 0.0, den = 0.0;
        const double L = st.L_used;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const int64_t j = off + i;
            double sq0 = 0.0, sq1 = 0.0, proj = 0.0;
            for (int64_t d = 0; d < D; ++d) {
                const double e0 = (double)b.theta_prev[d * b.ld + b.src[j]] - mean0[d];
                const double e1v = (double)b.theta_new[d * b.ld + j] - mean1[d];
                sq0 += e0 * e0;
                sq1 += e1v * e1v;
                proj += e1v * (double)b.p_final[d * b.ld + j];
            }
            const double h = rp.jitter ? halton2((uint32_t)(i * rp.n_iters + k)) : 1.0;
            const double gj = (h * L) * (sq1 - sq0) * proj;
            num += b.alpha[j] * gj;
            den += b.alpha[j];
        }
        num = block_reduce(num, buf, OpSum());
        den = block_reduce(den, buf, OpSum());
        if (threadIdx.x == 0) {
            if (den > 0.0 && isfinite(num / den)) {
                const double gh = num / den;
                st.adam_t += 1.0;
                st.adam_m = rp.adam_b1 * st.adam_m + (1.0 - rp.adam_b1) * gh;
                st.adam_v = rp.adam_b2 * st.adam_v + (1.0 - rp.adam_b2) * gh * gh;
                const double mh = st.adam_m / (1.0 - pow(rp.adam_b1, st.adam_t));
                const double vh = st.adam_v / (1.0 - pow(rp.adam_b2, st.adam_t));
                st.log_L += rp.adam_lr * mh / (sqrt(vh) + rp.adam_eps);
                st.log_L = fmin(fmax(st.log_L, rp.log_L_lo), rp.log_L_hi);
            }
            st.Lbar = 0.9 * st.Lbar + 0.1 * exp(st.log_L);
        }
    }
    if (threadIdx.x == 0) {
        if (rp.adapt && k == rp.n_warmup && st.Lbar > 0.0) st.log_L = log(st.Lbar);
        st.log_z += log_z_inc;
        st.log_z_inc = log_z_inc;
        st.mean_alpha = sa / (double)n;
        st.ess = (m2 > -CUDART_INF) ? e1 * e1 / e2 : 0.0;
        st.grad_evals = ge;
        st.iters_total += 1;
        st.grad_evals_total += ge;
        st.resamples_total += resample;
        st.ess_sum += st.ess;
        if (k > rp.n_warmup) st.ess_sum_post += st.ess;
        st.steps_min = smin;
        st.steps_max = smax;
        st.k = k + 1;
    }
}

// ============================================================ launchers
cudaError_t launch_init_draw(const StepBufs& b, float* theta, cudaStream_t s) {
    const int bs = 256;
    k_init_draw<<<(unsigned)((b.N + bs - 1) / bs), bs, 0, s>>>(b, theta);
    return cudaGetLastError();
}
cudaError_t launch_init_finish(const StepBufs& b, const double* logpi, cudaStream_t s) {
    k_init_finish<<<(unsigned)b.n_runs, RUN_THREADS, 0, s>>>(b, logpi);
    return cudaGetLastError();
}
cudaError_t launch_normalise(const StepBufs& b, cudaStream_t s) {
    k_normalise<<<(unsigned)b.n_runs, RUN_THREADS, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_resample_scan(const StepBufs& b, cudaStream_t s) {
    k_resample_scan<<<(unsigned)b.n_tiles, SCAN_THREADS, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_steps_sort(const StepBufs& b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b.hist, 0, sizeof(int32_t) * (size_t)(b.max_steps_all + 1), s);
    if (e != cudaSuccess) return e;
    const int bs = 256;
    const unsigned grid = (unsigned)((b.N + bs - 1) / bs);
    k_steps<<<grid, bs, 0, s>>>(b);
    k_hist_scan<<<1, 1024, 0, s>>>(b);
    k_sort_scatter<<<grid, bs, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_reweight_chees(const StepBufs& b, cudaStream_t s) {
    if (b.D > 1024) return cudaErrorInvalidValue;
    k_reweight_chees<<<(unsigned)b.n_runs, RUN_THREADS, 0, s>>>(b);
    return cudaGetLastError();
}

// ============================================================ stand-alone stages
__global__ void k_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Philox4 w = philox4x32_10(Philox4{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]}, seed);
    out[4 * i] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
}
cudaError_t launch_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(seed, ctr, out, n);
    return cudaGetLastError();
}

__global__ void k_normals(uint64_t seed, uint32_t tag, uint32_t k, int64_t N, int64_t D, double* out,
                          int64_t ld) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    for (int64_t d = 0; d < D; d += 2) {
        double z0, z1;
        normal_pair(seed, (uint32_t)(d >> 1), (uint32_t)j, k, tag, z0, z1);
        out[d * ld + j] = z0;
        if (d + 1 < D) out[(d + 1) * ld + j] = z1;
    }
}
cudaError_t launch_normals(uint64_t seed, uint32_t tag, uint32_t k, int64_t N, int64_t D, double* out,
                           int64_t ld, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    k_normals<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(seed, tag, k, N, D, out, ld);
    return cudaGetLastError();
}

__global__ void k_steps_only(int64_t N, int64_t K, int64_t k, double L, double eps, int32_t max_steps,
                             int32_t jitter, double* out_h, int32_t* out_steps) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double h = jitter ? halton2((uint32_t)(j * K + k)) : 1.0;
    if (out_h) out_h[j] = h;
    out_steps[j] = step_count(h, L, eps, max_steps);
}
cudaError_t launch_steps_only(int64_t N, int64_t K, int64_t k, double L, double eps, int32_t max_steps,
                              int32_t jitter, double* out_h, int32_t* out_steps, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    k_steps_only<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, K, k, L, eps, max_steps, jitter, out_h,
                                                             out_steps);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(RUN_THREADS) k_normalise_flat(const double* logw, int64_t N, double* W,
                                                                double* lse_out, double* ess_out) {
    __shared__ double buf[32];
    double m = -CUDART_INF;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, logw[i]);
    m = block_reduce(m, buf, OpMax());
    if (!(m > -CUDART_INF)) {
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) W[i] = 0.0;
        if (threadIdx.x == 0) {
            *lse_out = -CUDART_INF;
            *ess_out = 0.0;
        }
        return;
    }
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += exp(logw[i] - m);
    s = block_reduce(s, buf, OpSum());
    const double lse = m + log(s);
    double s2 = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double w = exp(logw[i] - lse);
        W[i] = w;
        s2 += w * w;
    }
    s2 = block_reduce(s2, buf, OpSum());
    if (threadIdx.x == 0) {
        *lse_out = lse;
        *ess_out = 1.0 / s2;
    }
}
cudaError_t launch_normalise_flat(const double* logw, int64_t N, double* W, double* lse, double* ess,
                                  cudaStream_t s) {
    if (N <= 0) return cudaErrorInvalidValue;
    k_normalise_flat<<<1, RUN_THREADS, 0, s>>>(logw, N, W, lse, ess);
    return cudaGetLastError();
}

// Stand-alone systematic resampling of given normalised weights W.
struct FlatScratch {
    RunParams rp;
    RunState st;
    unsigned int counter[4];
};
static int64_t flat_tiles(int64_t N) { return (N + SCAN_TILE - 1) / SCAN_TILE; }
int64_t resample_scratch_bytes(int64_t N) {
    return (int64_t)(((sizeof(FlatScratch) + 255) / 256) * 256 + sizeof(TileDesc) * (size_t)flat_tiles(N));
}

__global__ void __launch_bounds__(RUN_THREADS) k_quantise_flat(const double* W, int64_t N, uint64_t r64,
                                                               unsigned long long* q, FlatScratch* fs,
                                                               int64_t n_tiles) {
    __shared__ unsigned long long ubuf[32];
    int c = 0;
    while (((int64_t)1 << c) < N) ++c;
    const double scale = ldexp(1.0, 62 - c);
    unsigned long long T = 0ull;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = W[i] * scale;
        const unsigned long long qi = v > 0.0 ? __double2ull_rz(v) : 0ull;
        q[i] = qi;
        T += qi;
    }
    T = block_reduce(T, ubuf, OpSum());
    if (threadIdx.x == 0) {
        RunParams rp = {};
        rp.off = 0;
        rp.n = N;
        rp.n_tiles = (int32_t)n_tiles;
        rp.tile0 = 0;
        fs->rp = rp;
        RunState st = {};
        st.k = 1;
        st.T = T;
        st.U = __umul64hi((unsigned long long)r64, T);
        st.resample = T != 0ull;
        st.status = T != 0ull ? 0 : -4;
        fs->st = st;
        fs->counter[0] = 0u;
        fs->counter[1] = 1u;        // tiles are zeroed before every call
    }
}

__global__ void k_copy_status(const FlatScratch* fs, int32_t* status) { *status = fs->st.status; }

cudaError_t launch_resample_flat(const double* W, int64_t N, uint64_t r64, unsigned long long* q,
                                 int32_t* anc, int32_t* status, void* scratch, cudaStream_t s) {
    if (N <= 0 || N > (1ll << 30)) return cudaErrorInvalidValue;
    const int64_t nt = flat_tiles(N);
    FlatScratch* fs = reinterpret_cast<FlatScratch*>(scratch);
    TileDesc* tiles = reinterpret_cast<TileDesc*>(reinterpret_cast<char*>(scratch) +
                                                  ((sizeof(FlatScratch) + 255) / 256) * 256);
    cudaError_t e = cudaMemsetAsync(tiles, 0, sizeof(TileDesc) * (size_t)nt, s);
    if (e != cudaSuccess) return e;
    k_quantise_flat<<<1, RUN_THREADS, 0, s>>>(W, N, r64, q, fs, nt);
    StepBufs b = {};
    b.runs = &fs->rp;
    b.rstate = &fs->st;
    b.tile_run = nullptr;
    b.n_runs = 1;
    b.N = N;
    b.q = q;
    b.anc = anc;
    b.counter = fs->counter;
    b.tiles = tiles;
    b.n_tiles = nt;
    k_resample_scan<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(b);
    k_copy_status<<<1, 1, 0, s>>>(fs, status);
    return cudaGetLastError();
}

}  // namespace smc
