// smc_api.cu -- host driver behind include/smc.h: device memory, the
// per-iteration launch sequence of Algorithm 3, statistics, and the
// kernel-level entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/smc.h"
#include "common.cuh"
#include "flow.cuh"
#include "smc_kernels.cuh"
#include "traj.cuh"

using namespace smc;

namespace {
constexpr double LOG_2PI = 1.8378770664093454835606594728112;

struct DevAlloc {
    std::vector<void*> ptrs;
    cudaStream_t s = nullptr;
    cudaError_t err = cudaSuccess;
    template <typename T>
    T* get(size_t count) {
        void* p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMallocAsync(&p, count * sizeof(T), s);
        if (e != cudaSuccess) {
            err = e;
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    void release() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
        ptrs.clear();
    }
};

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// The first m primes (sieve of Eratosthenes), for the N-d jitter schemes.
std::vector<int32_t> first_primes(int64_t m) {
    std::vector<int32_t> out;
    if (m < 1) return out;
    out.reserve((size_t)m);
    int64_t top = 64;
    for (;;) {
        std::vector<char> comp((size_t)top + 1, 0);
        out.clear();
        for (int64_t p = 2; p <= top && (int64_t)out.size() < m; ++p) {
            if (comp[(size_t)p]) continue;
            out.push_back((int32_t)p);
            for (int64_t q = p * p; q <= top; q += p) comp[(size_t)q] = 1;
        }
        if ((int64_t)out.size() == m) return out;
        top *= 2;
    }
}

bool jitter_needs_primes(int32_t scheme) { return scheme >= 3 && scheme <= 6; }
constexpr int64_t MAX_JITTER_PRIME_INDEX = 65536;   // P_m < 2^20: radical inverses stay exact

}  // namespace

// Per-move reference arrays of the centred tensor-core path (TrajArgs::c_*).
struct CentredScratch {
    float* centre = nullptr;
    float* gref = nullptr;
    float2* refs = nullptr;
    double* part = nullptr;
    int32_t runs = 0;
    float* sth = nullptr;     // the move's theta and p in slot order, [D x s_ld] (handles only)
    float* sp = nullptr;
    int64_t s_ld = 0;
    // several runs (handles only): run-uniform particle tiles (TrajArgs::c_tiles)
    int2* tiles = nullptr;
    int32_t* perm = nullptr;
    int32_t* padoff = nullptr;
    int32_t* pcnt = nullptr;
    int64_t ntiles = 0;
    std::vector<int2> h_tiles;        // host copies, uploaded once on the handle's stream
    std::vector<int32_t> h_padoff;
};

struct smc_dev_model {
    DevModel m{};
    DevAlloc mem;
    CentredScratch cs1;   // one run: the stage-level calls on caller buffers
};

namespace {
// sizes (a handle's particles per run) adds the slot-ordered state buffers
// and, with several runs, the run-uniform tile layout: run r's slots start at
// a multiple of 128, and the tiles are listed by their relative rank within
// their run (then by run), so that every run's longest trajectories start
// first.
CentredScratch alloc_centred(DevAlloc& A, const DevModel& m, int32_t runs,
                             const std::vector<int64_t>* sizes = nullptr) {
    CentredScratch c;
    if (!traj_centred_supported(m)) return c;
    c.centre = A.get<float>((size_t)(runs * m.dk));
    c.gref = A.get<float>((size_t)(runs * m.dk));
    c.refs = A.get<float2>((size_t)centred_refs_elems(m, runs));
    c.part = A.get<double>((size_t)centred_part_elems(m, runs));
    c.runs = (c.centre && c.gref && c.refs && c.part) ? runs : 0;
    if (!sizes) return c;
    int64_t N = 0;
    for (int64_t n : *sizes) N += n;
    int64_t slots = round_up(N, 32);
    if (runs > 1) {
        struct T { double key; int32_t r; int64_t i; };
        std::vector<T> tl;
        int64_t P = 0;
        c.h_padoff.resize((size_t)runs);
        for (int32_t r = 0; r < runs; ++r) {
            c.h_padoff[(size_t)r] = (int32_t)P;
            const int64_t nt = ((*sizes)[(size_t)r] + 127) / 128;
            for (int64_t i = 0; i < nt; ++i) tl.push_back({((double)i + 0.5) / (double)nt, r, i});
            P += nt * 128;
        }
        std::stable_sort(tl.begin(), tl.end(), [](const T& x, const T& y) {
            return x.key < y.key || (x.key == y.key && x.r < y.r);
        });
        for (const T& t : tl) c.h_tiles.push_back(make_int2(t.r, c.h_padoff[(size_t)t.r] + (int32_t)(128 * t.i)));
        c.ntiles = (int64_t)tl.size();
        slots = P;
        const int64_t nblk = (N + 1023) / 1024;
        c.tiles = A.get<int2>((size_t)c.ntiles);
        c.perm = A.get<int32_t>((size_t)P);
        c.padoff = A.get<int32_t>((size_t)runs);
        c.pcnt = A.get<int32_t>((size_t)(2 * nblk * runs));
    }
    c.sth = A.get<float>((size_t)(m.D * slots));
    c.sp = A.get<float>((size_t)(m.D * slots));
    c.s_ld = (c.sth && c.sp) ? slots : 0;
    return c;
}
// The tile table and run offsets, and -1 in every slot (the pads stay -1).
void upload_centred(const CentredScratch& c, cudaStream_t s) {
    if (!c.tiles) return;
    cudaMemcpyAsync(c.tiles, c.h_tiles.data(), sizeof(int2) * c.h_tiles.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c.padoff, c.h_padoff.data(), sizeof(int32_t) * c.h_padoff.size(), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(c.perm, 0xff, sizeof(int32_t) * (size_t)c.s_ld, s);
}
// Call after a.ld is set: the slot-ordered buffers serve only launches with
// the stride they were sized for.
void set_centred(TrajArgs& a, const CentredScratch& c) {
    a.c_centre = c.centre;
    a.c_gref = c.gref;
    a.c_refs = c.refs;
    a.c_part = c.part;
    a.c_runs = c.runs;
    a.c_sth = c.s_ld > 0 ? c.sth : nullptr;
    a.c_sp = c.s_ld > 0 ? c.sp : nullptr;
    a.c_sld = c.s_ld;
    a.c_tiles = c.tiles;
    a.c_perm = c.perm;
    a.c_padoff = c.padoff;
    a.c_pcnt = c.pcnt;
    a.c_ntiles = c.ntiles;
}
}  // namespace

struct smc_handle {
    cudaStream_t stream = nullptr;
    int64_t n_runs = 0, N = 0, ld = 0, D = 0, K = 0;
    int32_t precision = 0;
    smc_dev_model model;
    DevAlloc mem;
    std::vector<RunParams> h_runs;
    RunParams* d_runs = nullptr;
    RunState* d_rstate = nullptr;
    int32_t* d_run_of = nullptr;
    int32_t* d_primes = nullptr;   // N-d jitter schemes only
    int32_t* d_tile_run = nullptr;
    float* theta[2] = {nullptr, nullptr};
    float* grad[2] = {nullptr, nullptr};
    double* logpi[2] = {nullptr, nullptr};
    int cur = 0;
    float* p_final = nullptr;
    double *logw = nullptr, *W = nullptr, *dH = nullptr, *alpha = nullptr;
    unsigned long long* q = nullptr;
    unsigned long long* cprefix = nullptr;   // multinomial runs only
    int32_t *anc = nullptr, *src = nullptr, *steps = nullptr, *perm = nullptr, *hist = nullptr;
    unsigned int* counter = nullptr;
    TileDesc* tiles = nullptr;
    int32_t *slice_run = nullptr, *slice_start = nullptr;
    int64_t n_slices = 0;
    SlicePart* parts = nullptr;
    double* colsum = nullptr;
    unsigned int* done = nullptr;
    int* dev_err = nullptr;     // set by a bounded device wait that gave up
    unsigned int* work = nullptr;   // tile counter of persistent trajectory launches
    int64_t n_tiles = 0;
    int32_t max_steps_all = 0;
    int64_t iters_done = 0;
    int sticky = 0;
    std::string err;
    std::vector<smc_config> cfg;       // init_mean / init_chol cleared: they were the caller's
    std::vector<std::vector<double>> init_host;   // staged copies of the initial distributions
    // profiling: events around trajectory launches, launch counter
    bool profiling = false;
    // CUDA graph of two consecutive iterations (buffer parity 0 -> 1 -> 0)
    cudaGraphExec_t graph2 = nullptr;
    bool graph_flow = false;               // whether graph2 runs the preconditioned move
    cudaStream_t graph_stream = nullptr;   // private stream the graph is captured and replayed on
    cudaEvent_t fork = nullptr, join = nullptr;
    std::vector<cudaEvent_t> events;
    size_t n_event_pairs = 0;
    int64_t kernel_launches = 0;
    // learned preconditioner (transport map) and its training state
    bool flow_on = false;
    DevFlow flow{};
    smc_flow_config flow_cfg{};
    std::vector<float> flow_init;   // parameters at smc_flow_enable, restored by smc_reset
    float* flow_partials = nullptr;
    float* z0 = nullptr;            // latent start / end points of the last move
    float* z1 = nullptr;
    // launch plan chosen by the autotuner
    int32_t traj_tile = 0, n_traj_tiles = 1;
    std::vector<double> tile_ms;
    CentredScratch cs;   // centred precision: reference arrays of every run
};

namespace {

smc_status fail(smc_handle* h, smc_status st, const std::string& msg) {
    if (h) {
        h->err = msg;
        if (st == SMC_E_CUDA || st == SMC_E_TIMEOUT || st == SMC_E_DEGENERATE) h->sticky = st;
    }
    return st;
}

smc_status cuda_fail(smc_handle* h, cudaError_t e, const char* where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? SMC_E_NOMEM : SMC_E_CUDA, msg);
}

std::vector<float> to_f32(const double* x, size_t n) {
    std::vector<float> v(n);
    for (size_t i = 0; i < n; ++i) v[i] = (float)x[i];
    return v;
}

uint16_t f32_to_bf16_rn(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);   // NaN stays NaN
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_to_f32(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Validates a model description and uploads it.  Returns an error text or "".
std::string upload_model(smc_dev_model* dm, const smc_model* md, cudaStream_t s) {
    if (!md) return "model is NULL";
    if (md->dim < 1 || md->dim > 1024) return "dim must be in [1, 1024]";
    DevModel& m = dm->m;
    m = DevModel{};
    m.kind = md->kind;
    m.D = (int32_t)md->dim;
    m.Dp = (int32_t)round_up(md->dim, 4);
    m.n = (int32_t)md->n_obs;
    m.h0 = md->hyper[0];
    m.h1 = md->hyper[1];
    dm->mem.s = s;
    auto up = [&](const std::vector<float>& v) -> float* {
        float* p = dm->mem.get<float>(v.size());
        if (p) cudaMemcpyAsync(p, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice, s);
        return p;
    };
    const int64_t D = md->dim;
    switch (md->kind) {
        case SMC_MODEL_GAUSS_DENSE: {
            if (!md->mu || !md->prec) return "GAUSS_DENSE needs mu and prec";
            m.mu = up(to_f32(md->mu, (size_t)D));
            m.P = up(to_f32(md->prec, (size_t)(D * D)));
            m.lconst = md->c;
            break;
        }
        case SMC_MODEL_LOGISTIC:
        case SMC_MODEL_LINEAR_GAUSS: {
            if (!md->X || !md->y || md->n_obs < 1) return "regression models need X, y and n_obs >= 1";
            const bool logit = md->kind == SMC_MODEL_LOGISTIC;
            const double tau = logit ? md->hyper[0] : md->hyper[1];
            if (!(tau > 0.0)) return "prior scale tau must be > 0";
            if (!logit && !(md->hyper[0] > 0.0)) return "noise scale sigma must be > 0";
            const int64_t n = md->n_obs, Dp = m.Dp;
            std::vector<float> X((size_t)(n * Dp), 0.0f);
            std::vector<uint16_t> Xh((size_t)(n * Dp), 0), Xl((size_t)(n * Dp), 0);
            for (int64_t i = 0; i < n; ++i)
                for (int64_t d = 0; d < D; ++d) {
                    const float x = (float)md->X[i * D + d];
                    X[(size_t)(i * Dp + d)] = x;
                    const uint16_t hi = f32_to_bf16_rn(x);
                    Xh[(size_t)(i * Dp + d)] = hi;
                    Xl[(size_t)(i * Dp + d)] = f32_to_bf16_rn(x - bf16_to_f32(hi));
                }
            m.X = up(X);
            m.y = up(to_f32(md->y, (size_t)n));
            uint16_t* xh = dm->mem.get<uint16_t>(Xh.size());
            uint16_t* xl = dm->mem.get<uint16_t>(Xl.size());
            if (xh) cudaMemcpyAsync(xh, Xh.data(), Xh.size() * 2, cudaMemcpyHostToDevice, s);
            if (xl) cudaMemcpyAsync(xl, Xl.data(), Xl.size() * 2, cudaMemcpyHostToDevice, s);
            m.Xbf = xh;
            m.Xbf_lo = xl;
            if (D <= 32 && n <= 4096 && xh && xl) {   // the warp-MMA kernel keeps X on chip
                uint16_t* img = dm->mem.get<uint16_t>((size_t)glm_mma_image_elems(n));
                if (img && build_glm_mma_image(xh, xl, n, (int)D, (int)Dp, img, s) == cudaSuccess) m.xmma_img = img;
            }
            if (D <= 128) {
                // per-chunk shared-memory images for the streamed tensor-core path:
                // 128-byte swizzle (16-byte unit u of row r stored at unit u ^ (r & 7))
                const int64_t C = STREAM_CHUNK, nch = (n + C - 1) / C, dk = round_up(D, 16);
                std::vector<uint16_t> xk((size_t)(nch * 2 * C * 64), 0), xt((size_t)(nch * dk * C), 0);
                std::vector<float> yi((size_t)(nch * C), 0.0f);
                for (int64_t i = 0; i < n; ++i) {
                    const int64_t c = i / C, r = i % C;
                    yi[(size_t)i] = (float)md->y[i];
                    for (int64_t d = 0; d < D; ++d) {
                        const uint16_t v = Xh[(size_t)(i * Dp + d)];
                        const int64_t atom = d / 64, u = (d % 64) / 8, e = d % 8;
                        const int64_t bk = c * (2 * C * 128) + atom * (C * 128) + r * 128 + ((u ^ (r & 7)) << 4) + 2 * e;
                        xk[(size_t)(bk / 2)] = v;
                        const int64_t ut = r / 8, et = r % 8;
                        const int64_t bt = c * (dk * 128) + d * 128 + ((ut ^ (d & 7)) << 4) + 2 * et;
                        xt[(size_t)(bt / 2)] = v;
                    }
                }
                uint16_t* xkd = dm->mem.get<uint16_t>(xk.size());
                uint16_t* xtd = dm->mem.get<uint16_t>(xt.size());
                if (xkd) cudaMemcpyAsync(xkd, xk.data(), xk.size() * 2, cudaMemcpyHostToDevice, s);
                if (xtd) cudaMemcpyAsync(xtd, xt.data(), xt.size() * 2, cudaMemcpyHostToDevice, s);
                m.xk_img = xkd;
                m.xt_img = xtd;
                m.y_img = up(yi);
                m.dk = (int32_t)dk;
                m.n_chunks = (int32_t)nch;
                // tiles of CENTRED_CHUNK observations for the centred path:
                // [atoms][CENTRED_CHUNK rows][128 B], same swizzle
                const int64_t CT = CENTRED_CHUNK, nt = (n + CT - 1) / CT, atoms = (dk + 63) / 64;
                std::vector<uint16_t> xc((size_t)(nt * atoms * CT * 64), 0);
                for (int64_t i = 0; i < n; ++i) {
                    const int64_t c = i / CT, r = i % CT;
                    for (int64_t d = 0; d < D; ++d) {
                        const int64_t atom = d / 64, u = (d % 64) / 8, e = d % 8;
                        const int64_t b = c * (atoms * CT * 128) + atom * (CT * 128) + r * 128 + ((u ^ (r & 7)) << 4) + 2 * e;
                        xc[(size_t)(b / 2)] = Xh[(size_t)(i * Dp + d)];
                    }
                }
                uint16_t* xcd = dm->mem.get<uint16_t>(xc.size());
                if (xcd) cudaMemcpyAsync(xcd, xc.data(), xc.size() * 2, cudaMemcpyHostToDevice, s);
                m.xc_img = xcd;
                m.n_tiles128 = (int32_t)nt;
                cudaStreamSynchronize(s);   // the staging vectors are pageable and local
                dm->cs1 = alloc_centred(dm->mem, m, 1);
            }
            if (logit) {
                m.lconst = -0.5 * (double)D * (LOG_2PI + 2.0 * std::log(tau));
            } else {
                const double sigma = md->hyper[0];
                m.lconst = -0.5 * (double)n * (LOG_2PI + 2.0 * std::log(sigma)) -
                           0.5 * (double)D * (LOG_2PI + 2.0 * std::log(tau));
            }
            // the host synchronises before the staging vectors go out of scope
            cudaStreamSynchronize(s);
            break;
        }
        case SMC_MODEL_HIER_NORMAL: {
            const int64_t G = md->n_obs;
            if (G < 1 || D != G + 2) return "HIER_NORMAL needs dim == n_obs + 2";
            if (!md->group_mean || !md->group_n || !md->group_ss) return "HIER_NORMAL needs group statistics";
            if (!(md->hyper[0] > 0.0)) return "sigma must be > 0";
            m.gmean = up(to_f32(md->group_mean, (size_t)G));
            m.gn = up(to_f32(md->group_n, (size_t)G));
            m.gss = up(to_f32(md->group_ss, (size_t)G));
            const double sigma = md->hyper[0];
            double c = -LOG_2PI;   // priors on mu and log tau
            for (int64_t g = 0; g < G; ++g)
                c += -0.5 * md->group_n[g] * (LOG_2PI + 2.0 * std::log(sigma)) - 0.5 * LOG_2PI;
            m.lconst = c;
            break;
        }
        case SMC_MODEL_BANANA: {
            if (D % 2 != 0) return "BANANA needs an even dim";
            if (!(md->hyper[0] > 0.0)) return "BANANA variance a must be > 0";
            m.lconst = -(double)(D / 2) * (0.5 * (LOG_2PI + std::log(md->hyper[0])) + 0.5 * LOG_2PI);
            break;
        }
        default: return "unknown model kind";
    }
    if (dm->mem.err != cudaSuccess) return std::string("device allocation failed: ") + cudaGetErrorString(dm->mem.err);
    cudaStreamSynchronize(s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return std::string("model upload: ") + cudaGetErrorString(e);
    return "";
}

std::string check_config(const smc_config& c) {
    if (c.n_particles < 1 || c.n_particles > (1ll << 30)) return "n_particles must be in [1, 2^30]";
    if (c.n_iters < 1) return "n_iters must be >= 1";
    if (c.n_iters * c.n_particles + c.n_iters >= (1ll << 32)) return "n_particles * n_iters must be < 2^32 (Halton index)";
    if (!(c.step_size > 0.0) || !std::isfinite(c.step_size)) return "step_size must be > 0";
    if (!(c.traj_len0 > 0.0)) return "traj_len0 must be > 0";
    if (c.max_steps < 1 || c.max_steps > 65536) return "max_steps must be in [1, 65536]";
    if (c.jitter < 0 || c.jitter > 11) return "jitter must be in [0, 11]";
    if (jitter_needs_primes(c.jitter) && c.n_iters > MAX_JITTER_PRIME_INDEX)
        return "the N-d jitter schemes need n_iters <= 65536";
    if (c.accept_reject != 0 && c.accept_reject != 1) return "accept_reject must be 0 or 1";
    if (!(c.init_scale > 0.0)) return "init_scale must be > 0";
    if (!(c.ess_frac >= 0.0 && c.ess_frac <= 1.0)) return "ess_frac must be in [0, 1]";
    if (!(c.step_adapt_rate >= 0.0) || !std::isfinite(c.step_adapt_rate)) return "step_adapt_rate must be >= 0";
    if (c.resample_scheme != 0 && c.resample_scheme != 1) return "resample_scheme must be 0 or 1";
    if (c.mcmc != 0 && c.mcmc != 1) return "mcmc must be 0 or 1";
    if (c.step_adapt_rate > 0.0 && !(c.step_adapt_target > 0.0 && c.step_adapt_target < 1.0))
        return "step_adapt_target must be in (0, 1)";
    if (c.precision < 0 || c.precision > 4) return "unknown precision";
    return "";
}

// The optional Gaussian initial distribution N(m, L L') of one run.
std::string check_init_dist(const smc_config& c, int64_t D) {
    if (c.init_mean)
        for (int64_t d = 0; d < D; ++d)
            if (!std::isfinite(c.init_mean[d])) return "init_mean must be finite";
    if (c.init_chol)
        for (int64_t d = 0; d < D; ++d) {
            const double l = c.init_chol[d * D + d];
            if (!(l > 0.0) || !std::isfinite(l)) return "init_chol needs a positive, finite diagonal";
            for (int64_t e = 0; e < d; ++e)
                if (!std::isfinite(c.init_chol[d * D + e])) return "init_chol must be finite";
        }
    return "";
}

StepBufs make_bufs(smc_handle* h) {
    StepBufs b{};
    b.runs = h->d_runs;
    b.rstate = h->d_rstate;
    b.run_of = h->d_run_of;
    b.tile_run = h->d_tile_run;
    b.n_runs = h->n_runs;
    b.N = h->N;
    b.ld = h->ld;
    b.D = h->D;
    b.logw = h->logw;
    b.W = h->W;
    b.q = h->q;
    b.cprefix = h->cprefix;
    b.primes = h->d_primes;
    b.any_multinomial = h->cprefix != nullptr;
    b.anc = h->anc;
    b.src = h->src;
    b.steps = h->steps;
    b.perm = h->perm;
    b.hist = h->hist;
    b.counter = h->counter;
    b.tiles = h->tiles;
    b.n_tiles = h->n_tiles;
    b.max_steps_all = h->max_steps_all;
    b.slice_run = h->slice_run;
    b.slice_start = h->slice_start;
    b.n_slices = h->n_slices;
    b.parts = h->parts;
    b.colsum = h->colsum;
    b.done = h->done;
    b.theta_prev = h->theta[h->cur];
    b.theta_new = h->theta[1 - h->cur];
    b.grad_prev = h->grad[h->cur];
    b.grad_new = h->grad[1 - h->cur];
    b.logpi_prev = h->logpi[h->cur];
    b.logpi_new = h->logpi[1 - h->cur];
    b.p_final = h->p_final;
    b.dH = h->dH;
    b.alpha = h->alpha;
    b.chees0 = h->flow_on ? h->z0 : nullptr;
    b.chees1 = h->flow_on ? h->z1 : nullptr;
    return b;
}

// Whether iteration k trains the transport map (warm-up, every train_every).
bool flow_trains_at(const smc_handle* h, int64_t k) {
    const smc_flow_config& fc = h->flow_cfg;
    return h->flow_on && fc.train_every > 0 && fc.epochs > 0 && k < h->cfg[0].n_warmup &&
           (k - 1) % fc.train_every == 0;
}

// `epochs` Adam steps on the weighted NLL of the current particles (after
// resampling: positions through src, weights 1/J or W), each followed by a
// rebuild of the work copies; every kernel of it is a no-op on the device
// when the tested ESS is below min_ess_frac * J.
cudaError_t flow_train(smc_handle* h, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    const FlowGate gate{h->d_rstate, h->d_runs, h->flow_cfg.min_ess_frac};
    for (int32_t ep = 0; ep < h->flow_cfg.epochs && e == cudaSuccess; ++ep) {
        e = flow_loss_grad(h->flow, h->theta[h->cur], h->ld, h->src, h->W, gate, h->N, h->flow_partials, s);
        if (e == cudaSuccess) e = flow_adam(h->flow, h->flow_cfg.lr, gate, s);
        if (e == cudaSuccess) e = flow_refresh(h->flow, s, true, gate);   // the next gradient sees the new map
    }
    if (h->profiling) h->kernel_launches += (4 + (h->flow.frag ? 1 : 0)) * (int64_t)h->flow_cfg.epochs;
    return e;
}

// Initial draw, target evaluation and initial weights (Algorithm 3, first
// lines) into buffer 0; the run state must already hold k = 1 and log L_0.
cudaError_t initial_draw(smc_handle* h) {
    cudaStream_t s = h->stream;
    h->cur = 0;
    StepBufs b = make_bufs(h);
    cudaError_t ce = launch_init_draw(b, h->theta[0], s);
    if (ce == cudaSuccess) {
        TrajArgs a{};
        a.theta_in = h->theta[0];
        a.grad_out = h->grad[0];
        a.logpi_out = h->logpi[0];
        a.run_of = h->d_run_of;
        a.runs = h->d_runs;
        a.rstate = h->d_rstate;
        a.N = h->N;
        a.ld = h->ld;
        a.eval_only = 1;
        a.dev_err = h->dev_err;
        a.work = h->work;
        set_centred(a, h->cs);
        ce = launch_traj(h->model.m, a, h->precision, s);
    }
    if (ce == cudaSuccess) ce = launch_init_finish(b, h->logpi[0], s);
    if (h->profiling) h->kernel_launches += 3;
    return ce;
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// The autotuner: every launch variant of the model's trajectory kernel runs a
// 16-step trajectory (capped at the largest step count) from the initial
// particles in buffer 0 into buffer 1, p_final, dH and alpha, all of which
// the first iteration rewrites before reading; best of three event-timed
// launches per variant.  Variants share their arithmetic, so nothing here
// can change a result.
cudaError_t autotune(smc_handle* h) {
    const int32_t nt = traj_tile_count(h->model.m, h->precision);
    h->n_traj_tiles = nt;
    h->traj_tile = 0;
    h->tile_ms.assign((size_t)nt, 0.0);
    if (nt <= 1 || h->N == 0) return cudaSuccess;
    cudaStream_t s = h->stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) return e;   // keep the default
    const int32_t S = std::max<int32_t>(1, std::min<int32_t>(16, h->max_steps_all));
    k_fill_i32<<<(unsigned)((h->N + 255) / 256), 256, 0, s>>>(h->steps, h->N, S);
    e = cudaGetLastError();
    TrajArgs a{};
    a.theta_in = h->theta[0];
    a.grad_in = h->grad[0];
    a.logpi_in = h->logpi[0];
    a.theta_out = h->theta[1];
    a.grad_out = h->grad[1];
    a.logpi_out = h->logpi[1];
    a.p_out = h->p_final;
    a.dH = h->dH;
    a.alpha = h->alpha;
    a.steps = h->steps;
    a.run_of = h->d_run_of;
    a.runs = h->d_runs;
    a.rstate = h->d_rstate;
    a.N = h->N;
    a.ld = h->ld;
    a.dev_err = h->dev_err;
    a.work = h->work;
    set_centred(a, h->cs);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int32_t v = 0; v < nt && e == cudaSuccess; ++v) {   // first launches (function attributes) untimed
        a.tile = v;
        e = launch_traj(h->model.m, a, h->precision, s);
    }
    std::vector<double> best((size_t)nt, 1e30);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        for (int32_t v = 0; v < nt && e == cudaSuccess; ++v) {
            a.tile = v;
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch_traj(h->model.m, a, h->precision, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess) best[(size_t)v] = std::min(best[(size_t)v], (double)ms);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    int32_t arg = 0;
    for (int32_t v = 1; v < nt; ++v)
        if (best[(size_t)v] < best[(size_t)arg]) arg = v;
    h->traj_tile = arg;
    h->tile_ms = best;
    return cudaSuccess;
}

RunState initial_state(const RunParams& rp, const smc_config& c) {
    RunState st{};
    st.log_L = std::fmin(std::fmax(std::log(c.traj_len0), rp.log_L_lo), rp.log_L_hi);
    st.k = 1;
    st.L_used = std::exp(st.log_L);
    st.eps = rp.eps;
    st.adam_b1t = 1.0;
    st.adam_b2t = 1.0;
    return st;
}

smc_status create(smc_handle** out, int64_t n_runs, const smc_config* cfg, const smc_model* model,
                  void* stream) {
    if (!out) return SMC_E_INVAL;
    *out = nullptr;
    if (n_runs < 1 || !cfg) return SMC_E_INVAL;
    smc_handle* h = new smc_handle();
    h->stream = static_cast<cudaStream_t>(stream);
    h->mem.s = h->stream;
    for (int64_t r = 0; r < n_runs; ++r) {
        std::string e = check_config(cfg[r]);
        if (!e.empty()) {
            fprintf(stderr, "smc_init: run %lld: %s\n", (long long)r, e.c_str());
            delete h;
            return SMC_E_INVAL;
        }
        if (cfg[r].n_iters != cfg[0].n_iters || cfg[r].n_warmup != cfg[0].n_warmup ||
            cfg[r].precision != cfg[0].precision) {
            fprintf(stderr, "smc_init_batch: runs must share n_iters, n_warmup and precision\n");
            delete h;
            return SMC_E_INVAL;
        }
    }
    std::string e = upload_model(&h->model, model, h->stream);
    if (!e.empty()) {
        fprintf(stderr, "smc_init: %s\n", e.c_str());
        h->model.mem.release();
        delete h;
        return SMC_E_INVAL;
    }
    h->precision = cfg[0].precision;
    if (h->precision == SMC_PREC_BF16C && n_runs > CENTRED_MAX_RUNS) {
        fprintf(stderr, "smc_init_batch: the centred precision serves at most %d runs per handle\n", CENTRED_MAX_RUNS);
        h->model.mem.release();
        delete h;
        return SMC_E_INVAL;
    }
    if (!traj_supported(h->model.m, h->precision)) {
        fprintf(stderr, "smc_init: no kernel for this model / dimension / precision\n");
        h->model.mem.release();
        delete h;
        return SMC_E_INVAL;
    }
    if (model->dim > MAX_CHEES_DIM) {
        fprintf(stderr, "smc_init: dim must be <= %d\n", MAX_CHEES_DIM);
        h->model.mem.release();
        delete h;
        return SMC_E_INVAL;
    }
    for (int64_t r = 0; r < n_runs; ++r) {
        const std::string ei = check_init_dist(cfg[r], model->dim);
        if (!ei.empty()) {
            fprintf(stderr, "smc_init: run %lld: %s\n", (long long)r, ei.c_str());
            h->model.mem.release();
            delete h;
            return SMC_E_INVAL;
        }
    }
    h->n_runs = n_runs;
    h->D = model->dim;
    h->K = cfg[0].n_iters;
    int64_t N = 0, tiles = 0, slices = 0;
    int32_t smax = 0;
    h->h_runs.resize((size_t)n_runs);
    std::vector<RunState> h_state((size_t)n_runs);
    for (int64_t r = 0; r < n_runs; ++r) {
        RunParams& rp = h->h_runs[(size_t)r];
        rp = RunParams{};
        rp.off = N;
        rp.n = cfg[r].n_particles;
        rp.seed = cfg[r].seed;
        rp.eps = cfg[r].step_size;
        rp.ess_frac = cfg[r].ess_frac;
        rp.init_scale = cfg[r].init_scale;
        rp.adam_lr = cfg[r].adam_lr;
        rp.adam_b1 = cfg[r].adam_b1;
        rp.adam_b2 = cfg[r].adam_b2;
        rp.adam_eps = cfg[r].adam_eps;
        rp.log_L_lo = std::log(cfg[r].step_size);
        rp.log_L_hi = std::log((double)cfg[r].max_steps * cfg[r].step_size);
        rp.max_steps = cfg[r].max_steps;
        rp.jitter = cfg[r].jitter;
        rp.adapt = cfg[r].adapt;
        rp.n_tiles = (int32_t)((rp.n + SCAN_TILE - 1) / SCAN_TILE);
        rp.tile0 = tiles;
        rp.n_iters = cfg[r].n_iters;
        rp.n_warmup = cfg[r].n_warmup;
        rp.accept_reject = cfg[r].accept_reject || cfg[r].mcmc;
        rp.mcmc = cfg[r].mcmc;
        rp.step_rate = cfg[r].step_adapt_rate;
        rp.resample_scheme = cfg[r].resample_scheme;
        rp.step_target = cfg[r].step_adapt_target;
        if (cfg[r].init_mean || cfg[r].init_chol) {
            // log |det L| summed over d in order (D log s without a factor)
            rp.init_general = 1;
            double ldet = 0.0;
            if (cfg[r].init_chol)
                for (int64_t d = 0; d < model->dim; ++d) ldet += std::log(cfg[r].init_chol[d * model->dim + d]);
            else
                ldet = (double)model->dim * std::log(cfg[r].init_scale);
            rp.init_logdet = ldet;
        }
        rp.slice0 = (int32_t)slices;
        rp.n_slices = (int32_t)((rp.n + SLICE - 1) / SLICE);
        slices += rp.n_slices;
        h_state[(size_t)r] = initial_state(rp, cfg[r]);
        N += rp.n;
        tiles += rp.n_tiles;
        smax = std::max(smax, rp.max_steps);
    }
    h->N = N;
    h->ld = round_up(N, 32);
    h->n_tiles = tiles;
    h->max_steps_all = smax;
    h->n_slices = slices;
    std::vector<int32_t> run_of((size_t)N), tile_run((size_t)tiles), slice_run((size_t)slices),
        slice_start((size_t)slices);
    for (int64_t r = 0; r < n_runs; ++r) {
        const RunParams& rp = h->h_runs[(size_t)r];
        for (int64_t i = 0; i < rp.n; ++i) run_of[(size_t)(rp.off + i)] = (int32_t)r;
        for (int64_t t = 0; t < rp.n_tiles; ++t) tile_run[(size_t)(rp.tile0 + t)] = (int32_t)r;
        for (int64_t q = 0; q < rp.n_slices; ++q) {
            slice_run[(size_t)(rp.slice0 + q)] = (int32_t)r;
            slice_start[(size_t)(rp.slice0 + q)] = (int32_t)(q * SLICE);
        }
    }
    DevAlloc& A = h->mem;
    const size_t nd = (size_t)(h->D * h->ld);
    h->d_runs = A.get<RunParams>((size_t)n_runs);
    h->d_rstate = A.get<RunState>((size_t)n_runs);
    h->d_run_of = A.get<int32_t>((size_t)N);
    h->d_tile_run = A.get<int32_t>((size_t)tiles);
    for (int b = 0; b < 2; ++b) {
        h->theta[b] = A.get<float>(nd);
        h->grad[b] = A.get<float>(nd);
        h->logpi[b] = A.get<double>((size_t)h->ld);
    }
    h->p_final = A.get<float>(nd);
    h->logw = A.get<double>((size_t)h->ld);
    h->W = A.get<double>((size_t)h->ld);
    h->dH = A.get<double>((size_t)h->ld);
    h->alpha = A.get<double>((size_t)h->ld);
    h->q = A.get<unsigned long long>((size_t)h->ld);
    for (int64_t r = 0; r < n_runs; ++r)
        if (cfg[r].resample_scheme == 1) {
            h->cprefix = A.get<unsigned long long>((size_t)h->ld);
            break;
        }
    {
        int64_t kp = 0;
        for (int64_t r = 0; r < n_runs; ++r)
            if (jitter_needs_primes(cfg[r].jitter)) kp = std::max(kp, cfg[r].n_iters);
        if (kp > 0) {
            const std::vector<int32_t> pr = first_primes(kp);
            int32_t* d = A.get<int32_t>(pr.size());
            if (d) cudaMemcpyAsync(d, pr.data(), pr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
            h->d_primes = d;
        }
    }
    h->anc = A.get<int32_t>((size_t)h->ld);
    h->src = A.get<int32_t>((size_t)h->ld);
    h->steps = A.get<int32_t>((size_t)h->ld);
    h->perm = A.get<int32_t>((size_t)h->ld);
    h->hist = A.get<int32_t>((size_t)smax + 1);
    h->counter = A.get<unsigned int>(4);
    h->tiles = A.get<TileDesc>((size_t)tiles);
    h->slice_run = A.get<int32_t>((size_t)slices);
    h->slice_start = A.get<int32_t>((size_t)slices);
    h->parts = A.get<SlicePart>((size_t)slices);
    h->colsum = A.get<double>((size_t)(slices * 2 * h->D));
    h->done = A.get<unsigned int>((size_t)n_runs);
    h->dev_err = A.get<int>(1);
    h->work = A.get<unsigned int>(1);
    if (h->precision == SMC_PREC_BF16C) {
        std::vector<int64_t> sizes((size_t)n_runs);
        for (int64_t r = 0; r < n_runs; ++r) sizes[(size_t)r] = cfg[r].n_particles;
        h->cs = alloc_centred(A, h->model.m, (int32_t)n_runs, &sizes);
    }
    for (int64_t r = 0; r < n_runs; ++r) {
        RunParams& rp = h->h_runs[(size_t)r];
        const int64_t D = h->D;
        if (cfg[r].init_mean) {
            h->init_host.emplace_back(cfg[r].init_mean, cfg[r].init_mean + D);
            rp.init_mean = A.get<double>((size_t)D);
        }
        if (cfg[r].init_chol) {
            h->init_host.emplace_back(cfg[r].init_chol, cfg[r].init_chol + D * D);
            rp.init_chol = A.get<double>((size_t)(D * D));
        }
    }
    if (A.err != cudaSuccess) {
        smc_status st = cuda_fail(h, A.err, "smc_init allocation");
        smc_destroy(h);
        return st;
    }
    cudaStream_t s = h->stream;
    upload_centred(h->cs, s);
    {
        // the staged initial distributions, in the order they were staged
        size_t k = 0;
        for (int64_t r = 0; r < n_runs; ++r) {
            const RunParams& rp = h->h_runs[(size_t)r];
            if (cfg[r].init_mean) {
                cudaMemcpyAsync(const_cast<double*>(rp.init_mean), h->init_host[k].data(),
                                sizeof(double) * h->init_host[k].size(), cudaMemcpyHostToDevice, s);
                ++k;
            }
            if (cfg[r].init_chol) {
                cudaMemcpyAsync(const_cast<double*>(rp.init_chol), h->init_host[k].data(),
                                sizeof(double) * h->init_host[k].size(), cudaMemcpyHostToDevice, s);
                ++k;
            }
        }
    }
    cudaMemcpyAsync(h->d_runs, h->h_runs.data(), sizeof(RunParams) * (size_t)n_runs, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->d_rstate, h_state.data(), sizeof(RunState) * (size_t)n_runs, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->d_run_of, run_of.data(), sizeof(int32_t) * (size_t)N, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->d_tile_run, tile_run.data(), sizeof(int32_t) * (size_t)tiles, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(h->tiles, 0, sizeof(TileDesc) * (size_t)tiles, s);
    cudaMemsetAsync(h->counter, 0, sizeof(unsigned int) * 4, s);
    cudaMemsetAsync(h->done, 0, sizeof(unsigned int) * (size_t)n_runs, s);
    cudaMemsetAsync(h->dev_err, 0, sizeof(int), s);
    cudaMemcpyAsync(h->slice_run, slice_run.data(), sizeof(int32_t) * (size_t)slices, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->slice_start, slice_start.data(), sizeof(int32_t) * (size_t)slices, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(h->theta[0], 0, nd * sizeof(float), s);
    cudaMemsetAsync(h->theta[1], 0, nd * sizeof(float), s);
    cudaMemsetAsync(h->grad[0], 0, nd * sizeof(float), s);
    cudaMemsetAsync(h->grad[1], 0, nd * sizeof(float), s);
    cudaMemsetAsync(h->p_final, 0, nd * sizeof(float), s);

    h->cfg.assign(cfg, cfg + n_runs);
    for (smc_config& c : h->cfg) c.init_mean = c.init_chol = nullptr;   // the caller's memory
    cudaError_t ce = initial_draw(h);
    if (ce == cudaSuccess) ce = autotune(h);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
        smc_status st = cuda_fail(h, ce, "smc_init");
        fprintf(stderr, "%s\n", h->err.c_str());
        smc_destroy(h);
        return st;
    }
    *out = h;
    return SMC_OK;
}

smc_status read_stats(smc_handle* h, smc_stats* stats) {
    std::vector<RunState> st((size_t)h->n_runs);
    cudaError_t e = cudaMemcpyAsync(st.data(), h->d_rstate, sizeof(RunState) * (size_t)h->n_runs,
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "smc_step stats");
    smc_status ret = SMC_OK;
    int derr = 0;
    if (cudaMemcpy(&derr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && derr)
        ret = fail(h, SMC_E_TIMEOUT, "a bounded device wait in the trajectory kernel gave up");
    for (int64_t r = 0; r < h->n_runs; ++r) {
        const RunState& s = st[(size_t)r];
        if (stats) {
            smc_stats& o = stats[r];
            o.ess = s.ess;
            o.ess_pre = s.stat_ess_pre;
            o.log_z_inc = s.log_z_inc;
            o.mean_alpha = s.mean_alpha;
            o.traj_len = s.L_last;
            o.grad_evals = s.grad_evals;
            o.steps_min = s.steps_min;
            o.steps_max = s.steps_max;
            o.resampled = s.stat_resampled;
            o.pad = 0;
        }
        if (s.status == -4) ret = fail(h, SMC_E_DEGENERATE, "all weights are zero in run " + std::to_string(r));
        if (s.status == -5) ret = fail(h, SMC_E_TIMEOUT, "resampling look-back gave up in run " + std::to_string(r));
    }
    return ret;
}

}  // namespace

extern "C" {

smc_status smc_init(smc_handle** out, const smc_config* cfg, const smc_model* model, void* stream) {
    return create(out, 1, cfg, model, stream);
}

smc_status smc_init_batch(smc_handle** out, int64_t n_runs, const smc_config* cfg, const smc_model* model,
                          void* stream) {
    return create(out, n_runs, cfg, model, stream);
}

smc_status smc_step(smc_handle* h, smc_stats* stats) {
    if (!h) return SMC_E_INVAL;
    if (h->sticky) return SMC_E_STATE;
    cudaStream_t s = h->stream;
    StepBufs b = make_bufs(h);
    cudaError_t e = launch_weights_steps(b, s);
    if (e == cudaSuccess) e = launch_resample_scan(b, s);
    if (e == cudaSuccess) e = launch_sort(b, s);
    if (e == cudaSuccess && flow_trains_at(h, h->iters_done + 1)) e = flow_train(h, s);
    if (e == cudaSuccess) {
        TrajArgs a{};
        a.theta_in = h->theta[h->cur];
        a.grad_in = h->grad[h->cur];
        a.logpi_in = h->logpi[h->cur];
        a.theta_out = h->theta[1 - h->cur];
        a.grad_out = h->grad[1 - h->cur];
        a.logpi_out = h->logpi[1 - h->cur];
        a.p_out = h->p_final;
        a.dH = h->dH;
        a.alpha = h->alpha;
        a.steps = h->steps;
        a.perm = h->perm;
        a.src = h->src;
        a.run_of = h->d_run_of;
        a.runs = h->d_runs;
        a.rstate = h->d_rstate;
        a.N = h->N;
        a.ld = h->ld;
        a.dev_err = h->dev_err;
        a.work = h->work;
        a.tile = h->traj_tile;
        set_centred(a, h->cs);
        if (h->profiling) {
            const size_t i = 2 * h->n_event_pairs;
            while (h->events.size() < i + 2) {
                cudaEvent_t ev;
                e = cudaEventCreate(&ev);
                if (e != cudaSuccess) return cuda_fail(h, e, "smc_step profiling");
                h->events.push_back(ev);
            }
            cudaEventRecord(h->events[i], s);
            e = h->flow_on ? launch_traj_flow(h->model.m, h->flow, a, h->z0, h->z1, s)
                           : launch_traj(h->model.m, a, h->precision, s);
            cudaEventRecord(h->events[i + 1], s);
            h->n_event_pairs += 1;
            // + the centred form's reference kernels, and its run partition with several runs
            h->kernel_launches += KERNELS_PER_ITERATION +
                                  (h->precision == SMC_PREC_BF16C ? (h->n_runs > 1 ? 6 : 3) : 0);
        } else {
            e = h->flow_on ? launch_traj_flow(h->model.m, h->flow, a, h->z0, h->z1, s)
                           : launch_traj(h->model.m, a, h->precision, s);
        }
    }
    if (e == cudaSuccess) e = launch_move_stats(b, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "smc_step launch");
    h->cur = 1 - h->cur;
    h->iters_done += 1;
    if (stats) return read_stats(h, stats);
    return SMC_OK;
}

// Captures two consecutive iterations (starting from buffer parity 0) into a
// CUDA graph, so that a run replays one graph launch per two iterations
// instead of 2 x 7 kernel launches.
// The capture happens on the handle's private stream (the caller's stream may
// be the legacy default stream, which cannot be captured).
static smc_status capture_two_steps(smc_handle* h) {
    cudaStream_t s = h->graph_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "smc_run capture");
    cudaStream_t user = h->stream;
    h->stream = s;
    smc_status st = smc_step(h, nullptr);
    if (st == SMC_OK) st = smc_step(h, nullptr);
    h->stream = user;
    e = cudaStreamEndCapture(s, &graph);
    h->iters_done -= 2;   // captured, not executed
    if (st != SMC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "smc_run capture");
    e = cudaGraphInstantiate(&h->graph2, graph, 0);
    cudaGraphDestroy(graph);
    h->graph_flow = h->flow_on;
    if (e != cudaSuccess) {
        h->graph2 = nullptr;
        return cuda_fail(h, e, "smc_run graph instantiate");
    }
    return SMC_OK;
}

smc_status smc_run(smc_handle* h, int64_t n_iters, smc_stats* per_iter) {
    if (!h || n_iters < 0) return SMC_E_INVAL;
    if (h->sticky) return SMC_E_STATE;
    // Graph replay when nothing has to be read back between iterations.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(h->stream, &cap);
    int64_t k = 0;
    if (!per_iter && h->flow_on) {
        // iterations that train the map are not graph-replayable (host loop of
        // epochs, Adam step counts): run them one by one
        while (k < n_iters && h->iters_done + 1 < h->cfg[0].n_warmup && h->flow_cfg.train_every > 0 &&
               h->flow_cfg.epochs > 0) {
            smc_status st = smc_step(h, nullptr);
            if (st != SMC_OK) return st;
            ++k;
        }
    }
    const bool graphs = !per_iter && !h->profiling && n_iters - k >= 2 && cap == cudaStreamCaptureStatusNone;
    if (graphs) {
        if (h->cur != 0) {   // align to the captured buffer parity
            smc_status st = smc_step(h, nullptr);
            if (st != SMC_OK) return st;
            ++k;
        }
        if (h->graph2 && h->graph_flow != h->flow_on) {   // captured before the map was enabled
            cudaGraphExecDestroy(h->graph2);
            h->graph2 = nullptr;
        }
        if (!h->graph_stream) {
            cudaError_t e = cudaStreamCreateWithFlags(&h->graph_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(h, e, "smc_run graph stream");
        }
        if (!h->graph2) {
            smc_status st = capture_two_steps(h);
            if (st != SMC_OK) return st;
        }
        // caller's stream -> private stream -> caller's stream
        cudaError_t e = cudaEventRecord(h->fork, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->graph_stream, h->fork, 0);
        for (; e == cudaSuccess && k + 2 <= n_iters; k += 2) {
            e = cudaGraphLaunch(h->graph2, h->graph_stream);
            h->iters_done += 2;
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->join, h->graph_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->join, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "smc_run graph launch");
    }
    for (; k < n_iters; ++k) {
        smc_status st = smc_step(h, per_iter ? per_iter + k * h->n_runs : nullptr);
        if (st != SMC_OK) return st;
    }
    return SMC_OK;
}

smc_status smc_log_evidence(const smc_handle* hc, double* out) {
    smc_handle* h = const_cast<smc_handle*>(hc);
    if (!h || !out) return SMC_E_INVAL;
    std::vector<RunState> st((size_t)h->n_runs);
    cudaError_t e = cudaMemcpyAsync(st.data(), h->d_rstate, sizeof(RunState) * (size_t)h->n_runs,
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "smc_log_evidence");
    smc_status ret = SMC_OK;
    for (int64_t r = 0; r < h->n_runs; ++r) {
        out[r] = st[(size_t)r].log_z;
        if (st[(size_t)r].status == -4) ret = fail(h, SMC_E_DEGENERATE, "all weights are zero");
        if (st[(size_t)r].status == -5) ret = fail(h, SMC_E_TIMEOUT, "resampling look-back gave up");
    }
    return ret;
}

smc_status smc_get_layout(const smc_handle* h, int64_t* ld, int64_t* n_total, int64_t* n_runs) {
    if (!h) return SMC_E_INVAL;
    if (ld) *ld = h->ld;
    if (n_total) *n_total = h->N;
    if (n_runs) *n_runs = h->n_runs;
    return SMC_OK;
}

smc_status smc_get_buffer(const smc_handle* hc, int32_t which, void* dst, int64_t bytes, int32_t device_ptrs) {
    smc_handle* h = const_cast<smc_handle*>(hc);
    if (!h || !dst || bytes < 0) return SMC_E_INVAL;
    const void* srcp = nullptr;
    int64_t avail = 0;
    const int64_t nd = h->D * h->ld;
    std::vector<double> runstate;
    switch (which) {
        case SMC_BUF_THETA: srcp = h->theta[h->cur]; avail = nd * 4; break;
        case SMC_BUF_GRAD: srcp = h->grad[h->cur]; avail = nd * 4; break;
        case SMC_BUF_LOGPI: srcp = h->logpi[h->cur]; avail = h->N * 8; break;
        case SMC_BUF_LOGW: srcp = h->logw; avail = h->N * 8; break;
        case SMC_BUF_W: srcp = h->W; avail = h->N * 8; break;
        case SMC_BUF_ANCESTORS: srcp = h->anc; avail = h->N * 4; break;
        case SMC_BUF_STEPS: srcp = h->steps; avail = h->N * 4; break;
        case SMC_BUF_P_FINAL: srcp = h->p_final; avail = nd * 4; break;
        case SMC_BUF_DH: srcp = h->dH; avail = h->N * 8; break;
        case SMC_BUF_ALPHA: srcp = h->alpha; avail = h->N * 8; break;
        case SMC_BUF_THETA_PREV: srcp = h->theta[1 - h->cur]; avail = nd * 4; break;
        case SMC_BUF_Z0: srcp = h->z0; avail = h->flow_on ? nd * 4 : 0; break;
        case SMC_BUF_Z1: srcp = h->z1; avail = h->flow_on ? nd * 4 : 0; break;
        case SMC_BUF_ORDER: srcp = h->perm; avail = h->N * 4; break;
        case SMC_BUF_RUNSTATE: {
            std::vector<RunState> st((size_t)h->n_runs);
            cudaError_t e = cudaMemcpyAsync(st.data(), h->d_rstate, sizeof(RunState) * (size_t)h->n_runs,
                                            cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "smc_get_buffer");
            runstate.resize((size_t)(9 * h->n_runs));
            for (int64_t r = 0; r < h->n_runs; ++r) std::memcpy(&runstate[(size_t)(9 * r)], &st[(size_t)r], 72);
            if (bytes > (int64_t)(runstate.size() * 8)) return SMC_E_INVAL;
            if (device_ptrs) {
                e = cudaMemcpyAsync(dst, runstate.data(), (size_t)bytes, cudaMemcpyHostToDevice, h->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
                return e == cudaSuccess ? SMC_OK : cuda_fail(h, e, "smc_get_buffer");
            }
            std::memcpy(dst, runstate.data(), (size_t)bytes);
            return SMC_OK;
        }
        default: return SMC_E_INVAL;
    }
    if (bytes > avail) return SMC_E_INVAL;
    cudaError_t e = cudaMemcpyAsync(dst, srcp, (size_t)bytes,
                                    device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? SMC_OK : cuda_fail(h, e, "smc_get_buffer");
}

smc_status smc_get_particles(const smc_handle* hc, float* theta, double* logw, int32_t device_ptrs) {
    smc_handle* h = const_cast<smc_handle*>(hc);
    if (!h) return SMC_E_INVAL;
    const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    if (theta)
        e = cudaMemcpy2DAsync(theta, (size_t)h->N * sizeof(float), h->theta[h->cur], (size_t)h->ld * sizeof(float),
                              (size_t)h->N * sizeof(float), (size_t)h->D, kind, h->stream);
    if (e == cudaSuccess && logw) e = cudaMemcpyAsync(logw, h->logw, (size_t)h->N * 8, kind, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? SMC_OK : cuda_fail(h, e, "smc_get_particles");
}

smc_status smc_moments(const smc_handle* hc, double* mean, double* var) {
    smc_handle* h = const_cast<smc_handle*>(hc);
    if (!h || !mean) return SMC_E_INVAL;
    const int64_t n = h->h_runs[0].n, D = h->D;
    std::vector<float> th((size_t)(D * h->N));
    std::vector<double> lw((size_t)h->N);
    smc_status st = smc_get_particles(h, th.data(), lw.data(), 0);
    if (st != SMC_OK) return st;
    double m = -INFINITY;
    for (int64_t j = 0; j < n; ++j) m = std::fmax(m, lw[(size_t)j]);
    if (!(m > -INFINITY)) return fail(h, SMC_E_DEGENERATE, "all weights are zero");
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += std::exp(lw[(size_t)j] - m);
    // particles of zero weight are left out (their positions may be non-finite)
    for (int64_t d = 0; d < D; ++d) {
        double mu = 0.0;
        for (int64_t j = 0; j < n; ++j)
            if (lw[(size_t)j] > -INFINITY) mu += std::exp(lw[(size_t)j] - m) / s * th[(size_t)(d * h->N + j)];
        double v = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (!(lw[(size_t)j] > -INFINITY)) continue;
            const double e = th[(size_t)(d * h->N + j)] - mu;
            v += std::exp(lw[(size_t)j] - m) / s * e * e;
        }
        mean[d] = mu;
        if (var) var[d] = v;
    }
    return SMC_OK;
}

smc_status smc_reset(smc_handle* h, uint64_t seed) {
    if (!h) return SMC_E_INVAL;
    if (h->sticky == SMC_E_CUDA) return SMC_E_STATE;
    std::vector<RunState> st((size_t)h->n_runs);
    for (int64_t r = 0; r < h->n_runs; ++r) {
        h->h_runs[(size_t)r].seed = seed + (uint64_t)r;
        st[(size_t)r] = initial_state(h->h_runs[(size_t)r], h->cfg[(size_t)r]);
    }
    cudaStream_t s = h->stream;
    cudaError_t e = cudaMemcpyAsync(h->d_runs, h->h_runs.data(), sizeof(RunParams) * (size_t)h->n_runs,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_rstate, st.data(), sizeof(RunState) * (size_t)h->n_runs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && h->flow_on) {
        e = cudaMemcpyAsync(h->flow.params, h->flow_init.data(), sizeof(float) * h->flow_init.size(),
                            cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->flow.adam_m, 0, sizeof(float) * h->flow_init.size(), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->flow.adam_v, 0, sizeof(float) * h->flow_init.size(), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->flow.adam_t, 0, sizeof(int32_t), s);
        if (e == cudaSuccess) e = flow_refresh(h->flow, s);
    }
    // the staging vectors are pageable: the copies have consumed them on return
    if (e == cudaSuccess) e = initial_draw(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "smc_reset");
    h->sticky = 0;
    h->err.clear();
    h->iters_done = 0;
    return SMC_OK;
}

smc_status smc_get_summary(const smc_handle* hc, smc_summary* out) {
    smc_handle* h = const_cast<smc_handle*>(hc);
    if (!h || !out) return SMC_E_INVAL;
    std::vector<RunState> st((size_t)h->n_runs);
    cudaError_t e = cudaMemcpyAsync(st.data(), h->d_rstate, sizeof(RunState) * (size_t)h->n_runs,
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "smc_get_summary");
    for (int64_t r = 0; r < h->n_runs; ++r) {
        const RunState& x = st[(size_t)r];
        out[r].iterations = x.iters_total;
        out[r].grad_evals = x.grad_evals_total;
        out[r].ess_sum = x.ess_sum;
        out[r].ess_sum_post_warmup = x.ess_sum_post;
        out[r].log_z = x.log_z;
        out[r].resamples = x.resamples_total;
    }
    return SMC_OK;
}

smc_status smc_profile(smc_handle* h, int32_t enable) {
    if (!h) return SMC_E_INVAL;
    h->profiling = enable != 0;
    if (enable) {
        h->n_event_pairs = 0;
        h->kernel_launches = 0;
    }
    return SMC_OK;
}

smc_status smc_get_profile(smc_handle* h, double* traj_ms, int64_t* traj_launches, int64_t* kernel_launches) {
    if (!h) return SMC_E_INVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "smc_get_profile");
    double total = 0.0;
    for (size_t i = 0; i < h->n_event_pairs; ++i) {
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, h->events[2 * i], h->events[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(h, e, "smc_get_profile");
        total += ms;
    }
    if (traj_ms) *traj_ms = total;
    if (traj_launches) *traj_launches = (int64_t)h->n_event_pairs;
    if (kernel_launches) *kernel_launches = h->kernel_launches;
    return SMC_OK;
}

smc_status smc_get_plan(const smc_handle* h, int32_t* traj_tile, int32_t* n_tiles, double* tile_ms) {
    if (!h) return SMC_E_INVAL;
    if (traj_tile) *traj_tile = h->traj_tile;
    if (n_tiles) *n_tiles = h->n_traj_tiles;
    if (tile_ms)
        for (int32_t v = 0; v < h->n_traj_tiles; ++v)
            tile_ms[v] = (size_t)v < h->tile_ms.size() ? h->tile_ms[(size_t)v] : 0.0;
    return SMC_OK;
}

smc_status smc_set_plan(smc_handle* h, int32_t traj_tile) {
    if (!h || traj_tile < 0 || traj_tile >= h->n_traj_tiles) return SMC_E_INVAL;
    if (traj_tile != h->traj_tile && h->graph2) {   // the captured graph launches the old variant
        if (h->graph_stream) cudaStreamSynchronize(h->graph_stream);
        cudaGraphExecDestroy(h->graph2);
        h->graph2 = nullptr;
    }
    h->traj_tile = traj_tile;
    return SMC_OK;
}

smc_status smc_last_error(const smc_handle* h, char* buf, int64_t len) {
    if (!h || !buf || len < 1) return SMC_E_INVAL;
    std::snprintf(buf, (size_t)len, "%s", h->err.c_str());
    return SMC_OK;
}

void smc_destroy(smc_handle* h) {
    if (!h) return;
    for (cudaEvent_t ev : h->events) cudaEventDestroy(ev);
    if (h->graph2) cudaGraphExecDestroy(h->graph2);
    if (h->graph_stream) {
        cudaStreamSynchronize(h->graph_stream);
        cudaStreamDestroy(h->graph_stream);
    }
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    h->mem.release();
    h->model.mem.release();
    cudaStreamSynchronize(h->stream);
    delete h;
}

// ------------------------------------------------------------------ kernel-level
smc_status smc_model_create(smc_dev_model** out, const smc_model* model, void* stream) {
    if (!out) return SMC_E_INVAL;
    *out = nullptr;
    smc_dev_model* m = new smc_dev_model();
    std::string e = upload_model(m, model, static_cast<cudaStream_t>(stream));
    if (!e.empty()) {
        fprintf(stderr, "smc_model_create: %s\n", e.c_str());
        m->mem.release();
        delete m;
        return SMC_E_INVAL;
    }
    *out = m;
    return SMC_OK;
}

void smc_model_destroy(smc_dev_model* m) {
    if (!m) return;
    cudaStream_t s = m->mem.s;
    m->mem.release();
    cudaStreamSynchronize(s);
    delete m;
}

static smc_status kstatus(cudaError_t e) {
    if (e == cudaSuccess) return SMC_OK;
    fprintf(stderr, "libsmcchees: %s\n", cudaGetErrorString(e));
    return e == cudaErrorInvalidValue ? SMC_E_INVAL : SMC_E_CUDA;
}

smc_status smc_k_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return SMC_E_INVAL;
    return kstatus(launch_philox(seed, ctr, out, n, static_cast<cudaStream_t>(stream)));
}

smc_status smc_k_normals(uint64_t seed, uint32_t tag, uint32_t k, int64_t N, int64_t D, double* out, int64_t ld,
                         void* stream) {
    if (N < 0 || D < 1 || ld < N || (N > 0 && !out)) return SMC_E_INVAL;
    return kstatus(launch_normals(seed, tag, k, N, D, out, ld, static_cast<cudaStream_t>(stream)));
}

smc_status smc_k_steps(int64_t N, int64_t K, int64_t k, double L, double eps, int32_t max_steps, int32_t jitter,
                       double* out_h, int32_t* out_steps, void* stream) {
    if (N < 0 || K < 1 || k < 0 || !(eps > 0.0) || max_steps < 1 || (N > 0 && !out_steps)) return SMC_E_INVAL;
    if (N * K + k >= (1ll << 32) || jitter < 0 || jitter > 1) return SMC_E_INVAL;
    return kstatus(launch_steps_only(N, K, k, L, eps, max_steps, jitter, out_h, out_steps,
                                     static_cast<cudaStream_t>(stream)));
}

smc_status smc_k_jitter(int32_t scheme, uint64_t seed, int64_t J, int64_t K, int64_t k, double* out_h,
                        void* stream) {
    if (scheme < 0 || scheme > 11 || J < 0 || J > (1ll << 30) || K < 1 || k < 1 || k > K) return SMC_E_INVAL;
    if (J > 0 && !out_h) return SMC_E_INVAL;
    if (J * K + k >= (1ll << 32)) return SMC_E_INVAL;
    if (jitter_needs_primes(scheme) && K > MAX_JITTER_PRIME_INDEX) return SMC_E_INVAL;
    if (J == 0) return SMC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t* d = nullptr;
    if (jitter_needs_primes(scheme)) {
        const std::vector<int32_t> pr = first_primes(K);
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), pr.size() * sizeof(int32_t), s);
        if (e != cudaSuccess) return kstatus(e);
        // pageable source: the call returns once the host data is staged
        e = cudaMemcpyAsync(d, pr.data(), pr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaFreeAsync(d, s);
            return kstatus(e);
        }
    }
    cudaError_t e = launch_jitter_only(scheme, seed, J, K, k, d, out_h, s);
    if (d) cudaFreeAsync(d, s);
    return kstatus(e);
}

smc_status smc_k_target(const smc_dev_model* m, const float* theta, int64_t N, int64_t ld, double* logpi,
                        float* grad, int32_t precision, void* stream) {
    if (!m || N < 0 || ld < N || (N > 0 && (!theta || !logpi || !grad))) return SMC_E_INVAL;
    if (!traj_supported(m->m, precision)) return SMC_E_INVAL;
    TrajArgs a{};
    a.theta_in = theta;
    a.grad_out = grad;
    a.logpi_out = logpi;
    a.N = N;
    a.ld = ld;
    a.eval_only = 1;
    set_centred(a, m->cs1);
    return kstatus(launch_traj(m->m, a, precision, static_cast<cudaStream_t>(stream)));
}

smc_status smc_k_leapfrog(const smc_dev_model* m, float* theta, float* p, float* grad, double* logpi,
                          const int32_t* steps, double eps, int64_t N, int64_t ld, int32_t precision, void* stream) {
    if (!m || N < 0 || ld < N || !(eps > 0.0)) return SMC_E_INVAL;
    if (N > 0 && (!theta || !p || !grad || !logpi || !steps)) return SMC_E_INVAL;
    if (!traj_supported(m->m, precision)) return SMC_E_INVAL;
    TrajArgs a{};
    a.theta_in = theta;
    a.grad_in = grad;
    a.logpi_in = logpi;
    a.theta_out = theta;
    a.grad_out = grad;
    a.logpi_out = logpi;
    a.p_in = p;
    a.p_out = p;
    a.steps = steps;
    a.eps_fixed = eps;
    a.N = N;
    a.ld = ld;
    set_centred(a, m->cs1);
    return kstatus(launch_traj(m->m, a, precision, static_cast<cudaStream_t>(stream)));
}

smc_status smc_k_normalise(const double* logw, int64_t N, double* W, double* lse, double* ess, void* stream) {
    if (N < 1 || !logw || !W || !lse || !ess) return SMC_E_INVAL;
    return kstatus(launch_normalise_flat(logw, N, W, lse, ess, static_cast<cudaStream_t>(stream)));
}

int64_t smc_k_resample_scratch_bytes(int64_t N) { return N < 1 ? 0 : resample_scratch_bytes(N); }

smc_status smc_k_resample(const double* W, int64_t N, uint64_t r64, uint64_t* q, int32_t* ancestors,
                          int32_t* status_out, void* scratch, void* stream) {
    if (N < 1 || N > (1ll << 30) || !W || !q || !ancestors || !status_out || !scratch) return SMC_E_INVAL;
    return kstatus(launch_resample_flat(W, N, r64, reinterpret_cast<unsigned long long*>(q), ancestors, status_out,
                                        scratch, static_cast<cudaStream_t>(stream)));
}

smc_status smc_k_lookback_wait_check(int64_t poll_limit, int32_t* status_out, void* scratch, void* stream) {
    if (poll_limit < 1 || poll_limit > (1ll << 40) || !status_out || !scratch) return SMC_E_INVAL;
    return kstatus(launch_lookback_wait_check((long long)poll_limit, reinterpret_cast<TileDesc*>(scratch),
                                              status_out, static_cast<cudaStream_t>(stream)));
}

// ------------------------------------------------------------------ transport map
int64_t smc_flow_num_params(int64_t dim, int32_t hidden, int32_t layers) {
    if (dim < 2 || hidden < 1 || layers < 1) return 0;
    return flow_num_params(dim, hidden, layers);
}

smc_status smc_flow_enable(smc_handle* h, const smc_flow_config* fc, const double* params) {
    if (!h || !fc || !params) return SMC_E_INVAL;
    if (h->sticky) return SMC_E_STATE;
    auto reject = [&](const char* why) { return fail(h, SMC_E_INVAL, std::string("smc_flow_enable: ") + why); };
    if (h->flow_on) return reject("already enabled");
    if (h->iters_done != 0) return reject("must be called before the first iteration");
    if (h->n_runs != 1) return reject("single-run handles only");
    if (h->precision != SMC_PREC_FP32) return reject("precision must be SMC_PREC_FP32");
    if (!flow_supported(h->model.m, fc->hidden, fc->layers))
        return reject("needs a GAUSS_DENSE or BANANA model with even dim <= 128, hidden a multiple of 4 "
                      "in [4, 128] and at least dim / 2 rounded up to 4, and layers in [1, 8]");
    if (fc->train_every < 0 || fc->epochs < 0 || !(fc->lr > 0.0) || !std::isfinite(fc->lr))
        return reject("train_every and epochs must be >= 0 and lr > 0");
    if (!(fc->min_ess_frac >= 0.0 && fc->min_ess_frac <= 1.0)) return reject("min_ess_frac must be in [0, 1]");
    if (fc->precision != SMC_PREC_FP32 && fc->precision != SMC_PREC_BF16)
        return reject("precision must be SMC_PREC_FP32 or SMC_PREC_BF16");
    if (fc->precision == SMC_PREC_BF16 && !flow_bf16_supported(h->D, fc->hidden, fc->layers))
        return reject("the BF16 form needs hidden a multiple of 16 in [16, 128]");
    if (fc->train_precision != SMC_PREC_FP32 && fc->train_precision != SMC_PREC_BF16)
        return reject("train_precision must be SMC_PREC_FP32 or SMC_PREC_BF16");
    if (fc->train_precision == SMC_PREC_BF16 && !flow_train_bf16_supported(h->D, fc->hidden, fc->layers))
        return reject("BF16 training needs hidden a multiple of 16 in [16, 128]");
    DevFlow f = flow_shape((int)h->D, fc->hidden, fc->layers);
    f.bf16 = fc->precision == SMC_PREC_BF16 ? 1 : 0;
    f.train_bf16 = fc->train_precision == SMC_PREC_BF16 ? 1 : 0;
    std::vector<float> p32((size_t)f.n_params);
    for (int64_t i = 0; i < f.n_params; ++i) {
        if (!std::isfinite(params[i])) return reject("non-finite parameter");
        p32[(size_t)i] = (float)params[i];
    }
    DevAlloc& A = h->mem;
    f.params = A.get<float>((size_t)f.n_params);
    f.adam_m = A.get<float>((size_t)f.n_params);
    f.adam_v = A.get<float>((size_t)f.n_params);
    f.grad = A.get<float>((size_t)f.n_params);
    f.work = A.get<float>((size_t)(f.L * f.layer_work));
    if (f.bf16 || f.train_bf16) f.frag = A.get<uint4>((size_t)(f.L * f.layer_frag));
    f.adam_t = A.get<int32_t>(1);
    float* partials = A.get<float>((size_t)flow_partials_floats(f, h->N));
    float* z0 = A.get<float>((size_t)(h->D * h->ld));
    float* z1 = A.get<float>((size_t)(h->D * h->ld));
    if (A.err != cudaSuccess) {
        cudaError_t e = A.err;
        A.err = cudaSuccess;
        return cuda_fail(h, e, "smc_flow_enable allocation");
    }
    cudaStream_t s = h->stream;
    cudaError_t e = cudaMemcpyAsync(f.params, p32.data(), sizeof(float) * p32.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f.adam_m, 0, sizeof(float) * p32.size(), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f.adam_v, 0, sizeof(float) * p32.size(), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f.adam_t, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(z0, 0, sizeof(float) * (size_t)(h->D * h->ld), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(z1, 0, sizeof(float) * (size_t)(h->D * h->ld), s);
    if (e == cudaSuccess) e = flow_refresh(f, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // p32 is pageable
    if (e != cudaSuccess) return cuda_fail(h, e, "smc_flow_enable");
    h->flow = f;
    h->flow_cfg = *fc;
    h->flow_init = std::move(p32);
    h->flow_partials = partials;
    h->z0 = z0;
    h->z1 = z1;
    h->flow_on = true;
    return SMC_OK;
}

smc_status smc_flow_get_params(const smc_handle* hc, double* params, int64_t n) {
    smc_handle* h = const_cast<smc_handle*>(hc);
    if (!h || !params) return SMC_E_INVAL;
    if (!h->flow_on || n != h->flow.n_params) return SMC_E_INVAL;
    std::vector<float> p32((size_t)n);
    cudaError_t e = cudaMemcpyAsync(p32.data(), h->flow.params, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "smc_flow_get_params");
    for (int64_t i = 0; i < n; ++i) params[i] = p32[(size_t)i];
    return SMC_OK;
}

// Stand-alone flow of the given shape over caller-owned device parameters:
// stream-ordered work copies (and partials) that the caller frees with release().
namespace {
struct TmpFlow {
    DevFlow f{};
    DevAlloc mem;
    bool make(int64_t D, int32_t H, int32_t L, const float* params, int64_t n_partial_rows, cudaStream_t s,
              bool bf16 = false) {
        mem.s = s;
        f = flow_shape((int)D, H, L);
        f.params = const_cast<float*>(params);
        f.work = mem.get<float>((size_t)(f.L * f.layer_work));
        if (bf16) {
            f.bf16 = 1;
            f.frag = mem.get<uint4>((size_t)(f.L * f.layer_frag));
        }
        partials = n_partial_rows > 0 ? mem.get<float>((size_t)flow_partials_floats(f, n_partial_rows)) : nullptr;
        return mem.err == cudaSuccess;
    }
    float* partials = nullptr;
};
}  // namespace

smc_status smc_k_flow_loss_grad(int64_t dim, int32_t hidden, int32_t layers, const float* params,
                                const float* theta, const double* W, int64_t N, int64_t ld, float* grad,
                                int32_t precision, void* stream) {
    if (!flow_shape_ok(dim, hidden, layers) || !params || !grad || N < 0 || ld < N) return SMC_E_INVAL;
    if (N > 0 && (!theta || !W)) return SMC_E_INVAL;
    if (precision != SMC_PREC_FP32 && precision != SMC_PREC_BF16) return SMC_E_INVAL;
    const bool bf16 = precision == SMC_PREC_BF16;
    if (bf16 && !flow_train_bf16_supported(dim, hidden, layers)) return SMC_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TmpFlow t;
    if (!t.make(dim, hidden, layers, params, std::max<int64_t>(N, 1), s, bf16)) {
        t.mem.release();
        return SMC_E_NOMEM;
    }
    t.f.bf16 = 0;   // the fragments serve the training products only
    t.f.train_bf16 = bf16 ? 1 : 0;
    t.f.grad = grad;
    cudaError_t e = flow_refresh(t.f, s);
    if (e == cudaSuccess && N == 0) e = cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)t.f.n_params, s);
    if (e == cudaSuccess && N > 0) e = flow_loss_grad(t.f, theta, ld, nullptr, W, FlowGate{}, N, t.partials, s);
    t.mem.release();
    return kstatus(e);
}

smc_status smc_k_flow_leapfrog(const smc_dev_model* m, int32_t hidden, int32_t layers, const float* params,
                               float* theta, float* p, float* grad, double* logpi, const int32_t* steps, double eps,
                               int64_t N, int64_t ld, float* z0, float* z1, double* dH, int32_t precision,
                               void* stream) {
    if (!m || !params || N < 0 || ld < N || !(eps > 0.0)) return SMC_E_INVAL;
    if (N > 0 && (!theta || !p || !grad || !logpi || !steps)) return SMC_E_INVAL;
    if (!flow_supported(m->m, hidden, layers)) return SMC_E_INVAL;
    if (precision != SMC_PREC_FP32 && precision != SMC_PREC_BF16) return SMC_E_INVAL;
    const bool bf16 = precision == SMC_PREC_BF16;
    if (bf16 && !flow_bf16_supported(m->m.D, hidden, layers)) return SMC_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TmpFlow t;
    if (!t.make(m->m.D, hidden, layers, params, 0, s, bf16)) {
        t.mem.release();
        return SMC_E_NOMEM;
    }
    TrajArgs a{};
    a.theta_in = theta;
    a.grad_in = grad;
    a.logpi_in = logpi;
    a.theta_out = theta;
    a.grad_out = grad;
    a.logpi_out = logpi;
    a.p_in = p;
    a.p_out = p;
    a.dH = dH;
    a.steps = steps;
    a.eps_fixed = eps;
    a.N = N;
    a.ld = ld;
    cudaError_t e = flow_refresh(t.f, s);
    if (e == cudaSuccess) e = launch_traj_flow(m->m, t.f, a, z0, z1, s);
    t.mem.release();
    return kstatus(e);
}

}  // extern "C"
