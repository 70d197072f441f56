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
// theta_0 ~ q_init = N(0, s^2 I) (Eq. for theta_0), or N(m, L L') when the
// run has a general Gaussian initial distribution, and log q_init(theta_0)
// parked in logw until the target has been evaluated.
__global__ void k_init_draw(StepBufs b, float* theta) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= b.N) return;
    const int r = b.run_of[j];
    const RunParams rp = b.runs[r];
    const uint32_t jl = (uint32_t)(j - rp.off);
    if (rp.init_general) {
        // theta_d = m_d + L_d0 z_0 + ... + L_dd z_d in FP64, added column by
        // column (the same order for every d), every product and sum rounded
        // on its own (no contraction), so the result is that of the plain
        // sum written in this order
        double acc[MAX_CHEES_DIM];
        const int64_t D = b.D;
        for (int64_t d = 0; d < D; ++d) acc[d] = rp.init_mean ? rp.init_mean[d] : 0.0;
        double zz = 0.0;
        for (int64_t e = 0; e < D; e += 2) {
            double z[2];
            normal_pair(rp.seed, (uint32_t)(e >> 1), jl, 0u, TAG_INIT, z[0], z[1]);
            for (int u = 0; u < 2 && e + u < D; ++u) {
                const int64_t c = e + u;
                zz = __dadd_rn(zz, __dmul_rn(z[u], z[u]));
                if (rp.init_chol) {
                    for (int64_t d = c; d < D; ++d) acc[d] = __dadd_rn(acc[d], __dmul_rn(rp.init_chol[d * D + c], z[u]));
                } else {
                    acc[c] = __dadd_rn(acc[c], __dmul_rn(rp.init_scale, z[u]));
                }
            }
        }
        for (int64_t d = 0; d < D; ++d) theta[d * b.ld + j] = (float)acc[d];
        b.logw[j] = __dsub_rn(-0.5 * zz, __dadd_rn(__dmul_rn(0.5 * (double)D, LOG_2PI), rp.init_logdet));
        return;
    }
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

// Resampling uniform of iteration k: Philox block (0, 0, k, RESAMPLE).
__device__ __forceinline__ unsigned long long resample_r64(uint64_t seed, int64_t k) {
    const Philox4 w = philox4x32_10(Philox4{0u, 0u, (uint32_t)k, TAG_RESAMPLE}, seed);
    return ((unsigned long long)w.x << 32) | w.y;
}

// Decision for the next iteration from the current log-weights: LSE, ESS
// (Eqs. for W and J_eff) and the resampling test J_eff < frac J (Sec. 3).
__device__ __forceinline__ void set_decision(RunState& st, const RunParams& rp, double m, double e1, double e2) {
    if (!(m > -CUDART_INF)) {
        st.status = -4;
        st.resample = 0;
        return;
    }
    const double ess = e1 * e1 / e2;
    st.lse = m + log(e1);
    st.ess_pre = ess;
    st.resample = ess < rp.ess_frac * (double)rp.n;
    st.L_used = exp(st.log_L);
    st.T = 0ull;
    st.r64 = resample_r64(rp.seed, st.k);
}

// w_1 = pi(theta_0) / q_init(theta_0) (Eq. for w_1); log Z_0 = LSE(log w) - log J;
// and the weight decision of iteration 1.
__global__ void __launch_bounds__(RUN_THREADS) k_init_finish(StepBufs b, const double* logpi) {
    __shared__ double buf[32];
    const int r = blockIdx.x;
    const RunParams rp = b.runs[r];
    double m = -CUDART_INF;
    for (int64_t i = threadIdx.x; i < rp.n; i += blockDim.x) {
        const int64_t j = rp.off + i;
        const double lp = logpi[j];
        // independent chains (Algorithm 2) carry no importance weight
        const double lw = rp.mcmc ? 0.0 : (isfinite(lp) ? lp - b.logw[j] : -CUDART_INF);
        b.logw[j] = lw;
        m = fmax(m, lw);
    }
    m = block_reduce(m, buf, OpMax());
    double s = 0.0, s2 = 0.0;
    if (m > -CUDART_INF)
        for (int64_t i = threadIdx.x; i < rp.n; i += blockDim.x) {
            const double e = exp(b.logw[rp.off + i] - m);
            s += e;
            s2 += e * e;
        }
    s = block_reduce(s, buf, OpSum());
    s2 = block_reduce(s2, buf, OpSum());
    if (threadIdx.x == 0) {
        RunState& st = b.rstate[r];
        st.log_z = (m > -CUDART_INF) ? m + log(s) - log((double)rp.n) : -CUDART_INF;
        st.status = 0;
        set_decision(st, rp, m, s, s2);
        b.done[r] = 0u;
    }
}

// atomicAdd(&counter[key], number of active lanes with this key) once per
// distinct key in the warp; returns this lane's old-value-plus-rank (the
// warp-aggregated form: particles of a warp often share a step count)
__device__ __forceinline__ int warp_agg_inc(int* counter, int key) {
    const unsigned peers = __match_any_sync(__activemask(), key);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter + key, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

// ============================================================ weights + steps
// Per particle slice: normalised weight W_j = exp(log w_j - LSE), the
// fixed-point weight q_j = floor(W_j 2^S) with S = 62 - ceil(log2 N) when the
// run resamples (its slice total is added to T with an exact integer atomic),
// the 1-d Halton jitter h_j of n = j K + k (Sec. 3.2), the step count
// S_j = ceil(h_j L / eps) clipped to [1, max] (Algorithm 2), and the
// histogram of S_j for the counting sort.
__global__ void __launch_bounds__(SLICE) k_weights_steps(StepBufs b) {
    __shared__ unsigned long long ubuf[32];
    const int c = blockIdx.x;
    const int r = b.slice_run[c];
    const RunParams& rp = b.runs[r];
    RunState& st = b.rstate[r];
    if (c == 0 && threadIdx.x == 0) {
        b.counter[0] = 0u;      // dynamic scan-tile counter of the next launch
        b.counter[1] += 1u;     // look-back epoch: never repeats within a handle
    }
    const int64_t i = b.slice_start[c] + threadIdx.x;
    const bool valid = i < rp.n;
    const int64_t j = rp.off + i;
    const bool ok = st.status == 0;
    unsigned long long qi = 0ull;
    if (valid) {
        int32_t S = 0;
        if (ok) {
            const double w = exp(b.logw[j] - st.lse);
            b.W[j] = w;
            if (st.resample) {
                int sh = 0;
                while (((int64_t)1 << sh) < rp.n) ++sh;
                const double v = w * ldexp(1.0, 62 - sh);
                qi = v > 0.0 ? __double2ull_rz(v) : 0ull;
                b.q[j] = qi;
            }
            const double h = jitter_h(rp.jitter, rp.seed, i, st.k, rp.n, rp.n_iters, b.primes);
            S = step_count(h, st.L_used, st.eps, rp.max_steps);
        }
        b.steps[j] = S;
        warp_agg_inc(b.hist, b.max_steps_all - S);
    }
    if (ok && st.resample) {
        qi = block_reduce(qi, ubuf, OpSum());
        if (threadIdx.x == 0 && qi) atomicAdd(&st.T, qi);
    }
}

// ============================================================ resampling scan
// Inclusive prefix C of q within each run by a single-pass decoupled
// look-back scan (tiles of SCAN_TILE elements; a tile id is taken from an
// atomic counter, so every predecessor tile has already started).  Each
// particle j then owns the output slots i with N C_{j-1} <= i T + U < N C_j,
// i.e. [cnt(C_{j-1}), cnt(C_j)) with cnt(C) = ceil((N C - U) / T) clipped to
// [0, N], and writes its own index there (systematic resampling).  Runs that
// do not resample write the identity source index.
constexpr long long LOOKBACK_SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ unsigned long long systematic_count(unsigned long long C, unsigned long long N,
                                                               unsigned long long T, unsigned long long U) {
    const unsigned long long NC = N * C;
    if (NC <= U) return 0ull;
    const unsigned long long c = (NC - U + T - 1ull) / T;
    return c < N ? c : N;
}

// Decoupled look-back of tile g (thread 0 only): publishes the tile's
// aggregate, walks back over the predecessors of its run (tiles first .. g-1)
// summing aggregates until an inclusive prefix, and publishes its own
// inclusive prefix.  Every wait on a predecessor is bounded: after `limit`
// polls without progress it gives up, sets *failed (the caller has already
// stored the run's error status, which is ordered before the publication) and
// returns the partial sum; the tile still publishes, so no successor waits
// forever.  Returns the exclusive prefix of the tile.
__device__ unsigned long long lookback_prefix(TileDesc* tiles, int64_t g, int64_t first, unsigned int epoch,
                                              unsigned long long tile_agg, long long limit, int* status,
                                              bool& failed) {
    TileDesc* me = tiles + g;
    unsigned long long excl = 0ull;
    failed = false;
    if (g == first) {
        me->incl = tile_agg;
        __threadfence();
        atomicExch(&me->flag, (epoch << 2) | 2u);
        return 0ull;
    }
    me->agg = tile_agg;
    __threadfence();
    atomicExch(&me->flag, (epoch << 2) | 1u);
    int64_t pred = g - 1;
    long long spins = 0;
    while (true) {
        const volatile TileDesc* pd = tiles + pred;
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
        if (++spins > limit) {   // bounded wait: report, never hang
            *(volatile int*)status = -5;
            __threadfence();
            failed = true;
            break;
        }
        __nanosleep(64);
    }
    me->incl = excl + tile_agg;
    __threadfence();
    atomicExch(&me->flag, (epoch << 2) | 2u);
    return excl;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_resample_scan(StepBufs b) {
    __shared__ unsigned int tile_s;
    __shared__ unsigned long long wsum[SCAN_THREADS / 32];
    __shared__ unsigned long long excl_s;
    __shared__ int failed_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) tile_s = atomicAdd(b.counter, 1u);
    __syncthreads();
    const int64_t g = tile_s;
    if (g >= b.n_tiles) return;
    const int r = b.tile_run ? b.tile_run[g] : 0;
    const RunParams rp = b.runs[r];
    RunState& st = b.rstate[r];
    const int64_t t_in_run = g - rp.tile0;
    const int64_t base = t_in_run * SCAN_TILE;
    if (!st.resample || st.status != 0) {
        if (b.src)
            for (int k = 0; k < SCAN_ITEMS; ++k) {
                const int64_t i = base + (int64_t)k * SCAN_THREADS + tid;
                if (i < rp.n) b.src[rp.off + i] = (int32_t)(rp.off + i);
            }
        return;
    }
    const unsigned int epoch = b.counter[1] & 0x3fffffffu;
    const unsigned long long N = (unsigned long long)rp.n, T = st.T;
    if (T == 0ull) {                 // no mass at all: degenerate
        if (tid == 0) st.status = -4;
        return;
    }
    const unsigned long long U = __umul64hi(st.r64, T);

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
        bool failed;
        excl_s = lookback_prefix(b.tiles, g, rp.tile0, epoch, tile_agg, LOOKBACK_SPIN_LIMIT, &st.status, failed);
        // a run whose look-back gave up anywhere (here or in a predecessor,
        // whose status store precedes its publication) gets no resampling from
        // this tile on: identity source indices for the tile's own slots
        failed_s = failed || *(volatile int*)&st.status != 0;
    }
    __syncthreads();
    if (failed_s) {
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            const int64_t i = base + (int64_t)k * SCAN_THREADS + tid;
            if (i < rp.n) {
                b.anc[rp.off + i] = (int32_t)i;
                if (b.src) b.src[rp.off + i] = (int32_t)(rp.off + i);
            }
        }
        return;
    }
    const unsigned long long off = excl_s + thread_excl;
    // systematic: particle i of the run owns output slots [cnt(C_{i-1}),
    // cnt(C_i)); multinomial: the prefix is kept for k_multinomial_search
    const bool multi = rp.resample_scheme == 1;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + (int64_t)tid * SCAN_ITEMS + k;
        if (i >= rp.n) break;
        const unsigned long long Ci = off + v[k];
        if (multi) {
            b.cprefix[rp.off + i] = Ci;
            continue;
        }
        const unsigned long long Cp = Ci - b.q[rp.off + i];
        const unsigned long long lo = systematic_count(Cp, N, T, U), hi = systematic_count(Ci, N, T, U);
        for (unsigned long long o = lo; o < hi; ++o) {
            b.anc[rp.off + (int64_t)o] = (int32_t)i;
            if (b.src) b.src[rp.off + (int64_t)o] = (int32_t)(rp.off + i);
        }
    }
}

// Multinomial resampling (the paper's scheme, Sec. 3) after the scan: output
// i of a resampling run takes the first particle j whose inclusive prefix C_j
// exceeds P_i = floor(u_i T / 2^64), u_i the 64-bit word pair of Philox block
// (1, i, k, RESAMPLE): a binary search over the run's prefix (C_{n-1} = T > P_i).
__global__ void k_multinomial_search(StepBufs b) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= b.N) return;
    const int r = b.run_of ? b.run_of[o] : 0;
    const RunParams& rp = b.runs[r];
    const RunState& st = b.rstate[r];
    if (rp.resample_scheme != 1 || !st.resample || st.status != 0) return;
    const int64_t i = o - rp.off;
    const Philox4 w = philox4x32_10(Philox4{1u, (uint32_t)i, (uint32_t)st.k, TAG_RESAMPLE}, rp.seed);
    const unsigned long long u = ((unsigned long long)w.x << 32) | w.y;
    const unsigned long long P = __umul64hi(u, st.T);
    const unsigned long long* C = b.cprefix + rp.off;
    int64_t lo = 0, hi = rp.n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (C[mid] > P) hi = mid;
        else lo = mid + 1;
    }
    b.anc[o] = (int32_t)lo;
    if (b.src) b.src[o] = (int32_t)(rp.off + lo);
}

// ============================================================ sort by steps
// Exclusive scan of the step histogram (one CTA), in place.
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
    const int slot = warp_agg_inc(b.hist, b.max_steps_all - b.steps[j]);
    b.perm[slot] = (int32_t)j;
}

// ============================================================ move statistics
// Per particle slice (first pass): with the momentum change-of-variable
// L-kernel the Jacobians cancel and log w += -Delta H (Sec. 3.1); pieces of
// log sum_j W_j exp(-Delta H_j) (evidence factor), of the new ESS, sum alpha,
// sum S_j, and the ChEES column sums of the pre-move and proposed states.
struct SliceIdx {
    int r;
    int64_t i, j;
    bool valid;
};
__device__ __forceinline__ SliceIdx slice_idx(const StepBufs& b) {
    SliceIdx x;
    const int c = blockIdx.x;
    x.r = b.slice_run[c];
    x.i = b.slice_start[c] + threadIdx.x;
    x.valid = x.i < b.runs[x.r].n;
    x.j = b.runs[x.r].off + x.i;
    return x;
}

// (max, sum exp) pair of a block; returns (M, S) with S = sum exp(a - M).
__device__ __forceinline__ void block_lse(double a, double* buf, double& M, double& S) {
    M = block_reduce(a, buf, OpMax());
    S = block_reduce(M > -CUDART_INF ? exp(a - M) : 0.0, buf, OpSum());
}

__global__ void __launch_bounds__(SLICE) k_move_stats(StepBufs b) {
    __shared__ double buf[5 * 32];
    __shared__ long long lbuf[32];
    __shared__ int ibuf[2 * 32];
    const SliceIdx x = slice_idx(b);
    const RunParams& rp = b.runs[x.r];
    const RunState& st = b.rstate[x.r];
    if (st.status != 0) return;
    const int c = blockIdx.x;
    const double logn = log((double)rp.n);
    double za = -CUDART_INF, lw = -CUDART_INF, al = 0.0;
    long long S = 0;
    int smin = 0x7fffffff, smax = 0;
    if (x.valid) {
        // with the Metropolis select the incremental weight is one
        const double dH = rp.accept_reject ? 0.0 : b.dH[x.j];
        const double old = b.logw[x.j];
        za = (st.resample ? -logn : old - st.lse) - dH;
        lw = (st.resample ? -logn : old) - dH;
        b.logw[x.j] = lw;
        al = b.alpha[x.j];
        S = b.steps[x.j];
        smin = smax = (int)S;
    }
    // the slice's reductions, each with block_reduce's tree, in three passes:
    // the two maxima, then the five sums that need them; the integer parts
    SlicePart part;
    double mx[2] = {za, lw};
    block_reduce_n(mx, buf, OpMax());
    part.za_m = mx[0];
    part.w_m = mx[1];
    const double e = (x.valid && part.w_m > -CUDART_INF) ? exp(lw - part.w_m) : 0.0;
    const bool step_rule = rp.step_rate > 0.0 && st.k < rp.n_warmup;
    double sm[5] = {part.za_m > -CUDART_INF ? exp(za - part.za_m) : 0.0, e, e * e, al,
                    step_rule ? (x.valid ? 1.0 / al : 0.0) : 0.0};
    block_reduce_n(sm, buf, OpSum());
    part.za_s = sm[0];
    part.w_e1 = sm[1];
    part.w_e2 = sm[2];
    part.alpha_sum = sm[3];
    part.inv_alpha_sum = step_rule ? sm[4] : 0.0;
    long long ls[1] = {S};
    block_reduce_n(ls, lbuf, OpSum());
    part.steps_sum = ls[0];
    int mm[2] = {-smin, smax};   // min S as -max(-S)
    block_reduce_n(mm, ibuf, OpMax());
    part.smin = -mm[0];
    part.smax = mm[1];
    part.g_num = 0.0;
    part.g_den = 0.0;
    if (threadIdx.x == 0) b.parts[c] = part;
    if (rp.adapt && st.k < rp.n_warmup) {
        // ChEES column sums of the pre-move states (after resampling) and the
        // proposals: warp w takes dimensions w, w + SLICE / 32, ...; a lane
        // sums its particles lane, lane + 32, ... of the slice in order, then
        // the warp adds its lanes (fixed order)
        constexpr int PL = SLICE / 32;   // particles per lane
        const int D = (int)b.D, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const int64_t i0 = b.slice_start[c];
        int64_t jj[PL], ss[PL];
#pragma unroll
        for (int u = 0; u < PL; ++u) {
            const int64_t i = i0 + lane + 32 * u;
            jj[u] = i < rp.n ? rp.off + i : -1;
            ss[u] = (jj[u] >= 0 && !b.chees0) ? b.src[jj[u]] : 0;
        }
        // two dimensions per pass, their loads issued together
        const float* t0 = b.chees0 ? b.chees0 : b.theta_prev;
        const float* t1 = b.chees1 ? b.chees1 : b.theta_new;
        for (int d = wid; d < D; d += 2 * (SLICE / 32)) {
            const int d2 = d + SLICE / 32;
            float a0[2][PL], a1[2][PL];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int dd = h ? d2 : d;
                const int64_t o = (int64_t)dd * b.ld;
#pragma unroll
                for (int u = 0; u < PL; ++u) {
                    const bool in = jj[u] >= 0 && dd < D;
                    a0[h][u] = in ? t0[o + (b.chees0 ? jj[u] : ss[u])] : 0.0f;
                    a1[h][u] = in ? t1[o + jj[u]] : 0.0f;
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int dd = h ? d2 : d;
                f2sum v0{0.0f, 0.0f}, v1{0.0f, 0.0f};    // FP32 pairs (about 48 bits)
#pragma unroll
                for (int u = 0; u < PL; ++u) {
                    if (jj[u] < 0) continue;
                    v0 = f2_add_f(v0, a0[h][u]);
                    v1 = f2_add_f(v1, a1[h][u]);
                }
                v0 = warp_sum_f2(v0);
                v1 = warp_sum_f2(v1);
                if (lane == 0 && dd < D) {
                    b.colsum[(int64_t)c * 2 * D + dd] = f2_to_double(v0);
                    b.colsum[(int64_t)c * 2 * D + D + dd] = f2_to_double(v1);
                }
            }
        }
    }
}

// Second pass: ChEES gradient estimates g_j = l_j (|t1_j - mean t1|^2 -
// |t0_j - mean t0|^2) (t1_j - mean t1)' p_j weighted by alpha_j (Algorithm 2),
// then the last slice of each run combines every slice in a fixed order:
// evidence, log-weights' ESS, Adam ascent on log L, Lbar, the freeze at
// M_warmup, statistics, and the weight decision of the next iteration.
__global__ void __launch_bounds__(SLICE) k_chees_finish(StepBufs b) {
    __shared__ double buf[7 * 32];
    __shared__ long long lbuf[32];
    __shared__ int ibuf[2 * 32];
    __shared__ float mean_s[4 * MAX_CHEES_DIM];   // negated means as FP32 pairs: hi [2D], lo [2D]
    __shared__ bool last_s;
    const SliceIdx x = slice_idx(b);
    const RunParams& rp = b.runs[x.r];
    RunState& st = b.rstate[x.r];
    if (st.status != 0) return;
    const int c = blockIdx.x;
    const int D = (int)b.D;
    const bool adapting = rp.adapt && st.k < rp.n_warmup;
    if (adapting) {
        // loads are issued in batches ahead of the sums (the sums keep their
        // order): a serial load-then-add loop waits one L2 round trip per term
        constexpr int BQ = 8;
        for (int t = threadIdx.x; t < 2 * D; t += blockDim.x) {
            double s = 0.0;
            const double* cs = b.colsum + (int64_t)rp.slice0 * 2 * D + t;
            int q = 0;
            for (; q + BQ <= rp.n_slices; q += BQ) {
                double v[BQ];
#pragma unroll
                for (int u = 0; u < BQ; ++u) v[u] = cs[(int64_t)(q + u) * 2 * D];
#pragma unroll
                for (int u = 0; u < BQ; ++u) s += v[u];
            }
            for (; q < rp.n_slices; ++q) s += cs[(int64_t)q * 2 * D];
            // the mean as a negated FP32 pair, ready to add to each value
            const f2sum m = f2_from_double(s / (double)rp.n);
            mean_s[t] = -m.hi;
            mean_s[2 * D + t] = -m.lo;
        }
        __syncthreads();
        double num = 0.0, den = 0.0;
        if (x.valid) {
            const int64_t src = b.src[x.j];
            const int64_t j0 = b.chees0 ? x.j : src;
            const float* t0 = b.chees0 ? b.chees0 : b.theta_prev;
            const float* t1 = b.chees1 ? b.chees1 : b.theta_new;
            // |t - mean|^2 and the projection accumulated in FP32 pairs
            f2sum sq0{0.0f, 0.0f}, sq1{0.0f, 0.0f}, proj{0.0f, 0.0f};
            constexpr int BD = 8;
            for (int d0 = 0; d0 < D; d0 += BD) {
                float v0[BD], v1[BD], vp[BD];
#pragma unroll
                for (int u = 0; u < BD; ++u) {
                    const int64_t o = (int64_t)(d0 + u) * b.ld;
                    const bool in = d0 + u < D;
                    v0[u] = in ? t0[o + j0] : 0.0f;
                    v1[u] = in ? t1[o + x.j] : 0.0f;
                    vp[u] = in ? b.p_final[o + x.j] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < BD; ++u) {
                    const int d = d0 + u;
                    if (d >= D) break;
                    const f2sum e0 = f2_add_f(f2sum{mean_s[d], mean_s[2 * D + d]}, v0[u]);
                    const f2sum e1 = f2_add_f(f2sum{mean_s[D + d], mean_s[3 * D + d]}, v1[u]);
                    sq0 = f2_add(sq0, f2_mul(e0, e0));
                    sq1 = f2_add(sq1, f2_mul(e1, e1));
                    proj = f2_add(proj, f2_mul(e1, f2sum{vp[u], 0.0f}));
                }
            }
            const double h = jitter_h(rp.jitter, rp.seed, x.i, st.k, rp.n, rp.n_iters, b.primes);
            const double a = b.alpha[x.j];
            num = a * ((h * st.L_used) * (f2_to_double(sq1) - f2_to_double(sq0)) * f2_to_double(proj));
            den = a;
        }
        double nd[2] = {num, den};
        block_reduce_n(nd, buf, OpSum());
        if (threadIdx.x == 0) {
            b.parts[c].g_num = nd[0];
            b.parts[c].g_den = nd[1];
        }
    }
    // Metropolis variant (Eqs. for alpha and the select rule): keep the
    // proposal when u < alpha, otherwise restore the start state; the ChEES
    // statistics above used the proposals, as in Algorithm 2.
    if (rp.accept_reject && x.valid) {
        const Philox4 w = philox4x32_10(Philox4{0u, (uint32_t)x.i, (uint32_t)st.k, TAG_MH}, rp.seed);
        if (!(u01_52(w.x, w.y) < b.alpha[x.j])) {
            const int64_t src = b.src[x.j];
            for (int d = 0; d < D; ++d) {
                b.theta_new[(int64_t)d * b.ld + x.j] = b.theta_prev[(int64_t)d * b.ld + src];
                b.grad_new[(int64_t)d * b.ld + x.j] = b.grad_prev[(int64_t)d * b.ld + src];
            }
            b.logpi_new[x.j] = b.logpi_prev[src];
        }
    }
    // ticket: the last slice of the run to get here finishes the iteration
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(&b.done[x.r], 1u);
        last_s = (t == (unsigned int)rp.n_slices - 1u);
    }
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    // fixed-order combination of the run's slices: thread t takes slices
    // t, t + SLICE, ... and the block reduces in a fixed tree
    // (the other slices' parts are read from L2 with cache-global loads, after
    // the fence that followed the ticket, so no stale L1 copy is seen)
    double za_m = -CUDART_INF, w_m = -CUDART_INF;
    for (int q = threadIdx.x; q < rp.n_slices; q += blockDim.x) {
        const SlicePart* p = b.parts + rp.slice0 + q;
        za_m = fmax(za_m, __ldcg(&p->za_m));
        w_m = fmax(w_m, __ldcg(&p->w_m));
    }
    double mx[2] = {za_m, w_m};
    block_reduce_n(mx, buf, OpMax());
    za_m = mx[0];
    w_m = mx[1];
    double za_s = 0.0, w_e1 = 0.0, w_e2 = 0.0, asum = 0.0, gnum = 0.0, gden = 0.0, iasum = 0.0;
    long long ssum = 0;
    int smin = 0x7fffffff, smax = 0;
    for (int q = threadIdx.x; q < rp.n_slices; q += blockDim.x) {
        const SlicePart* pp = b.parts + rp.slice0 + q;
        SlicePart p;
        p.za_m = __ldcg(&pp->za_m);
        p.za_s = __ldcg(&pp->za_s);
        p.w_m = __ldcg(&pp->w_m);
        p.w_e1 = __ldcg(&pp->w_e1);
        p.w_e2 = __ldcg(&pp->w_e2);
        p.alpha_sum = __ldcg(&pp->alpha_sum);
        p.inv_alpha_sum = __ldcg(&pp->inv_alpha_sum);
        p.g_num = __ldcg(&pp->g_num);
        p.g_den = __ldcg(&pp->g_den);
        p.steps_sum = __ldcg(&pp->steps_sum);
        p.smin = __ldcg(&pp->smin);
        p.smax = __ldcg(&pp->smax);
        if (p.za_m > -CUDART_INF) za_s += p.za_s * exp(p.za_m - za_m);
        if (p.w_m > -CUDART_INF) {
            const double f = exp(p.w_m - w_m);
            w_e1 += p.w_e1 * f;
            w_e2 += p.w_e2 * f * f;
        }
        asum += p.alpha_sum;
        iasum += p.inv_alpha_sum;
        gnum += p.g_num;
        gden += p.g_den;
        ssum += p.steps_sum;
        smin = min(smin, p.smin);
        smax = max(smax, p.smax);
    }
    // the run's sums, each with block_reduce's tree, in one pass per type
    double sm[7] = {za_s, w_e1, w_e2, asum, iasum, gnum, gden};
    block_reduce_n(sm, buf, OpSum());
    za_s = sm[0];
    w_e1 = sm[1];
    w_e2 = sm[2];
    asum = sm[3];
    iasum = sm[4];
    gnum = sm[5];
    gden = sm[6];
    long long ls[1] = {ssum};
    block_reduce_n(ls, lbuf, OpSum());
    ssum = ls[0];
    int mm[2] = {-smin, smax};   // min S as -max(-S)
    block_reduce_n(mm, ibuf, OpMax());
    smin = -mm[0];
    smax = mm[1];
    if (threadIdx.x != 0) return;
    const int64_t k = st.k;
    if (adapting) {
        if (gden > 0.0 && isfinite(gnum / gden)) {
            const double gh = gnum / gden;
            st.adam_t += 1.0;
            st.adam_m = rp.adam_b1 * st.adam_m + (1.0 - rp.adam_b1) * gh;
            st.adam_v = rp.adam_b2 * st.adam_v + (1.0 - rp.adam_b2) * gh * gh;
            st.adam_b1t *= rp.adam_b1;     // b1^t, b2^t by running products (no FP64 pow)
            st.adam_b2t *= rp.adam_b2;
            const double mh = st.adam_m / (1.0 - st.adam_b1t);
            const double vh = st.adam_v / (1.0 - st.adam_b2t);
            st.log_L += rp.adam_lr * mh / (sqrt(vh) + rp.adam_eps);
            // clamp L to [eps, max_steps eps] of this iteration's step size
            const double lo = rp.step_rate > 0.0 ? log(st.eps) : rp.log_L_lo;
            const double hi = rp.step_rate > 0.0 ? log((double)rp.max_steps * st.eps) : rp.log_L_hi;
            st.log_L = fmin(fmax(st.log_L, lo), hi);
        }
        st.Lbar = 0.9 * st.Lbar + 0.1 * exp(st.log_L);
    }
    if (rp.adapt && k == rp.n_warmup && st.Lbar > 0.0) st.log_L = log(st.Lbar);
    // optional warm-up step-size rule (not in the paper), after the ChEES
    // update: log eps += rate (a_h - target), a_h = n / sum 1/alpha_j the
    // harmonic mean (0 when some alpha_j = 0: the sum is +inf)
    if (rp.step_rate > 0.0 && k < rp.n_warmup)
        st.eps = exp(log(st.eps) + rp.step_rate * ((double)rp.n / iasum - rp.step_target));
    const double inc = za_m > -CUDART_INF ? za_m + log(za_s) : -CUDART_INF;
    st.log_z += inc;
    st.log_z_inc = inc;
    st.mean_alpha = asum / (double)rp.n;
    st.ess = w_m > -CUDART_INF ? w_e1 * w_e1 / w_e2 : 0.0;
    st.stat_ess_pre = st.ess_pre;
    st.stat_resampled = st.resample;
    st.L_last = st.L_used;
    st.grad_evals = ssum;
    st.steps_min = smin;
    st.steps_max = smax;
    st.iters_total += 1;
    st.grad_evals_total += ssum;
    st.resamples_total += st.resample;
    st.ess_sum += st.ess;
    if (k > rp.n_warmup) st.ess_sum_post += st.ess;
    st.k = k + 1;
    set_decision(st, rp, w_m, w_e1, w_e2);
    b.done[x.r] = 0u;
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
cudaError_t launch_weights_steps(const StepBufs& b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b.hist, 0, sizeof(int32_t) * (size_t)(b.max_steps_all + 1), s);
    if (e != cudaSuccess) return e;
    k_weights_steps<<<(unsigned)b.n_slices, SLICE, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_resample_scan(const StepBufs& b, cudaStream_t s) {
    k_resample_scan<<<(unsigned)b.n_tiles, SCAN_THREADS, 0, s>>>(b);
    if (b.any_multinomial && b.N > 0) k_multinomial_search<<<(unsigned)((b.N + 255) / 256), 256, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_sort(const StepBufs& b, cudaStream_t s) {
    const int bs = 256;
    k_hist_scan<<<1, 1024, 0, s>>>(b);
    k_sort_scatter<<<(unsigned)((b.N + bs - 1) / bs), bs, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_move_stats(const StepBufs& b, cudaStream_t s) {
    if (b.D > MAX_CHEES_DIM) return cudaErrorInvalidValue;
    k_move_stats<<<(unsigned)b.n_slices, SLICE, 0, s>>>(b);
    k_chees_finish<<<(unsigned)b.n_slices, SLICE, 0, s>>>(b);
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

__global__ void k_jitter_only(int32_t scheme, uint64_t seed, int64_t J, int64_t K, int64_t k,
                              const int32_t* primes, double* out_h) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= J) return;
    out_h[i] = jitter_h(scheme, seed, i, k, J, K, primes);
}
cudaError_t launch_jitter_only(int32_t scheme, uint64_t seed, int64_t J, int64_t K, int64_t k,
                               const int32_t* primes, double* out_h, cudaStream_t s) {
    if (J <= 0) return cudaSuccess;
    k_jitter_only<<<(unsigned)((J + 255) / 256), 256, 0, s>>>(scheme, seed, J, K, k, primes, out_h);
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
        st.r64 = (unsigned long long)r64;
        st.resample = T != 0ull;
        st.status = T != 0ull ? 0 : -4;
        fs->st = st;
        fs->counter[0] = 0u;
        fs->counter[1] = 1u;        // tiles are zeroed before every call
    }
}

__global__ void k_copy_status(const FlatScratch* fs, int32_t* status) { *status = fs->st.status; }

// The look-back wait of the resampling scan against a predecessor that never
// publishes: tile 1 of a two-tile run whose tile 0 descriptor holds no flag
// of the current epoch, with the caller's poll limit; the wait must give up
// and report -5 in *status (device), never hang.
__global__ void k_lookback_wait_check(TileDesc* tiles, long long limit, int* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    tiles[0].flag = 0u;   // epoch 0, not ready: nothing will ever publish it
    tiles[0].agg = tiles[0].incl = 0ull;
    *status = 0;
    __threadfence();
    bool failed;
    (void)lookback_prefix(tiles, 1, 0, 1u, 1ull, limit, status, failed);
    if (!failed) *status = 1;   // cannot happen: the predecessor never publishes
}
cudaError_t launch_lookback_wait_check(long long limit, TileDesc* tiles, int* status, cudaStream_t s) {
    k_lookback_wait_check<<<1, 32, 0, s>>>(tiles, limit, status);
    return cudaGetLastError();
}

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
