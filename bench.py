"""Benchmark of the SMC-ChEES hot path on GB300 (one JSON line on rank 0).

Workload (default): Bayesian logistic regression, n=1000 observations, D=25
(intercept + 24 N(0,1) features), N=4096 particles, K=50 SMC iterations,
1-d Halton jitter, eps=1e-3, L0=5, at most 500 leapfrog steps.  One "step"
is one complete sampler run (initial draw + K iterations: every stage of the
path), restarted on the device with a new seed (smc_reset) each step.

value      = real particle-gradient evaluations (sum of leapfrog steps over
             particles and iterations, all ranks) / device time of the timed
             steps (CUDA events on the library's stream, L2 flushed between
             steps outside the events, max over ranks).
e2e        = the same metric through the public C-ABI from host memory:
             smc_init (host model data copied in) -> smc_run -> particles,
             log-weights and evidence copied back -> smc_destroy.
roofline   = the trajectory kernel (dominant): algorithmic FLOPs per launch
             (4 n D per particle-gradient + 2 n D per particle for the endpoint
             energy) / its mean event-timed duration.
cpu_baseline / --impl reference = the FP64 C oracle on the host cores.
large_logistic = the n=1e5, D=100, 16384-particle regression on the streamed
             tensor-core kernel (BF16x2), with its roofline.
preconditioner = the learned transport map against the plain identity-metric
             sampler on the 8192-particle 100-d Gaussian (condition number
             1e4) and 50-d banana targets: ESS/s, grad-evals/s, acceptance,
             moment accuracy against the closed forms, and the achieved
             FLOP rate of the latent-space trajectory kernel.

N > 1 (torchrun): independent replicas, one per GPU, different seeds
("replicas only": the method's particle sets do not exchange data).
"""
from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

FP32_FMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 x max SM clock


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _workload(name):
    if name == "logistic":
        return workloads.logistic()
    if name == "gauss10":
        return workloads.gauss10()
    if name == "hier":
        return workloads.hier()
    if name == "logistic_large":
        return workloads.logistic_large()
    raise ValueError(name)


def aggregate_ranks(torch, dist, dev_ms, grad_evals, ess, device):
    """Whole-job numbers of independent replicas: the device time is the
    slowest rank's (max over ranks), work and ESS add up (sum over ranks).
    Without a process group the rank's own numbers are returned."""
    if not dist:
        return float(dev_ms), float(grad_evals), float(ess)
    t = torch.tensor([dev_ms, float(grad_evals), ess], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1]), float(t[2])


def _timed_runs(torch, smp, K, seeds, flush, moments=None):
    """One full sampler run per seed, each bracketed by CUDA events on the
    sampler's stream after an L2 flush; returns (device ms, gradient
    evaluations, post-warm-up ESS sum, log Z per run).  With a list in
    `moments`, the weighted posterior mean and variance of every run are
    appended to it (read back after the events)."""
    ms, ge, ess, lz = 0.0, 0, 0.0, []
    for sd in seeds:
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        smp.reset(sd)
        smp.run(K)                              # smc_run replays CUDA graphs
        e1.record()
        summ = smp.summary()                    # synchronises after the step; outside the events
        ms += e0.elapsed_time(e1)
        ge += sum(x["grad_evals"] for x in summ)
        ess += sum(x["ess_sum_post_warmup"] for x in summ)
        lz.append(summ[0]["log_z"])
        if moments is not None:
            moments.append(smp.moments())
    torch.cuda.synchronize()
    return ms, ge, ess, lz


def _profiled_run(smp, K, seed, flush):
    """Trajectory-kernel time and launch count: one more run with in-library
    events around every trajectory launch (no graphs), outside the timed region."""
    smp.profile(True)
    flush.zero_()
    smp.reset(seed)
    smp.run(K)
    ge = sum(x["grad_evals"] for x in smp.summary())
    prof = smp.get_profile()
    smp.profile(False)
    return prof, ge


def _mma_flops_per_grad(w, prec):
    """MMA FLOPs the warp-level tensor-core kernel issues per gradient (two
    products over the padded dimension 32 and observations padded to 16, three
    BF16 products each in the compensated form) and per end point (none: the
    end point is FP32)."""
    if w["kind"] not in ("logistic", "linear_gauss") or w["D"] > 32 or prec not in (1, 2):
        return None
    n16 = -(-w["n"] // 16) * 16
    return 2 * 2.0 * 32 * n16 * (3 if prec == 1 else 1), 0.0


def _flops_per_grad(w):
    if w["kind"] in ("logistic", "linear_gauss"):
        return 4.0 * w["n"] * w["D"], 2.0 * w["n"] * w["D"]
    if w["kind"] == "gauss_dense":
        return 2.0 * w["D"] ** 2, 2.0 * w["D"] ** 2
    if w["kind"] == "hier_normal":
        # per group: b = mu + tau eta (2), ybar - b (1), n (.)/s^2 (2), sum (1),
        # tau eta r into d/dlog tau (3), r tau - eta (2)
        return 11.0 * w["n"] + 4.0, 14.0 * w["n"]
    return 0.0, 0.0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _traffic_for(kernel_file, workload):
    """Per-launch DRAM bytes of the trajectory kernel from a committed ncu
    summary, if it was taken on the current source of that kernel and for
    this bench workload (one file holds the kernels of several models)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        src = os.path.join(ROOT, "paper_2504_02627_gb300", "csrc", kernel_file)
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        e = t.get(kernel_file)
        if e and e.get("source_sha256_16") == h and e.get("bench_workload") == workload:
            return e.get("bytes_per_launch_full")
    except (OSError, ValueError):
        pass
    return None


def cpu_oracle_rate(w, run, seconds_target=20.0, iters=2):
    """The FP64 oracle on the host cores: the first `iters` SMC iterations of
    the same workload (all particles, full data); returns grad-evals/s."""
    import oracle
    if w["kind"] == "logistic":
        t = oracle.TargetSpec.logistic(w["X"], w["y"], w.get("tau", 1.0))
    elif w["kind"] == "gauss_dense":
        t = oracle.TargetSpec.gauss_dense(w["mu"], w["P"])
    else:
        t = oracle.TargetSpec.hier_normal(w["ybar"], w["n_g"], w["ss"], w["sigma"])
    cores = os.cpu_count() or 1
    cfg = oracle.SMCConfig(seed=999, **dict(run))
    t0 = time.perf_counter()
    st = oracle.smc_init(t, cfg, nthreads=cores)
    st["chees"] = oracle.initial_chees_state(cfg)
    ge, done = 0, 0
    for k in range(1, iters + 1):
        out = oracle.smc_iteration(t, cfg, k, st, nthreads=cores)
        ge += out["stats"]["grad_evals"]
        done += 1
        if time.perf_counter() - t0 > seconds_target:
            break
    dt = time.perf_counter() - t0
    return ge / dt, cores, dt, done


def _c5_truth(w):
    """Closed-form log Z, mean and marginal variances of the C5 targets."""
    D = w["D"]
    if w["kind"] == "gauss_dense":
        P = np.asarray(w["P"], np.float32).astype(np.float64)
        _, ld = np.linalg.slogdet(P)
        return 0.5 * D * np.log(2 * np.pi) - 0.5 * ld, np.zeros(D), np.diag(np.linalg.inv(P))
    a, b = w["a"], w["b"]
    return 0.0, np.zeros(D), np.tile([a, 1.0 + 2.0 * b * b * a * a], D // 2)


def _flow_flops_per_grad(w, H, L):
    """Algorithmic FLOPs of one latent-space gradient: per coupling layer the
    conditioner forward 2(Dh H + H^2 + H D) and its vector-Jacobian product
    (the same), plus the target's gradient."""
    D, Dh = w["D"], w["D"] // 2
    tgt = 2.0 * D * D if w["kind"] == "gauss_dense" else 8.0 * D
    return L * 4.0 * (Dh * H + H * H + H * D) + tgt


def precond_compare(g, torch, stream, flush, K=50, M=25, H=128, L=4):
    """The learned preconditioner against the plain identity-metric sampler
    on the two 8192-particle targets of the preconditioner workload: one
    complete run each (K iterations, training during warm-up), device-timed,
    L2 flushed before each; ESS/s, grad-evals/s, acceptance and the accuracy
    of the posterior moments against the closed forms."""
    out = {}
    for name, w, eps in (("gauss100_cond1e4", workloads.gauss100_cond(), 0.01),
                         ("banana50", workloads.banana50(), 0.05)):
        lz_t, m_t, v_t = _c5_truth(w)
        run = dict(w["run"], step_size=eps, n_iters=K, n_warmup=M)
        md = g.ModelData.from_workload(w)
        res = {}
        arms = ("plain", "plain_bf16x3", "flow", "flow_bf16") if w["kind"] == "gauss_dense" else \
            ("plain", "flow", "flow_bf16")
        for arm in arms:
            prec = 1 if arm == "plain_bf16x3" else 0
            smp = g.Sampler(md, g.make_config(seed=4242, precision=prec, **run), stream)
            if arm.startswith("flow"):
                smp.enable_flow(workloads.flow_init(w["D"], H, L, seed=5), H, L, train_every=2, epochs=20,
                                lr=1e-3, min_ess_frac=0.25, precision=2 if arm == "flow_bf16" else 0)
            smp.run(2)                      # first launches (function attributes, graph capture) untimed
            smp.reset(777)
            smp.profile(True)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            stats = smp.run(K, with_stats=True)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            prof = smp.get_profile()
            smp.profile(False)
            summ = smp.summary()[0]
            m, v = smp.moments()
            smp.close()
            r = {"ms": ms, "ess_per_s": summ["ess_sum_post_warmup"] / (ms / 1e3),
                 "grad_evals_per_s": summ["grad_evals"] / (ms / 1e3),
                 "mean_alpha_post_warmup": float(np.mean([x["mean_alpha"] for x in stats[M:]])),
                 "mean_ess_post_warmup": float(np.mean([x["ess"] for x in stats[M:]])),
                 "mean_err_sd_units": float(np.sqrt(np.mean((m - m_t) ** 2 / v_t))),
                 "var_rel_err": float(np.sqrt(np.mean((v / v_t - 1.0) ** 2))),
                 "log_z": summ["log_z"], "log_z_closed_form": lz_t,
                 "traj_share": prof["traj_ms"] / ms}
            if arm.startswith("flow"):
                fl = _flow_flops_per_grad(w, H, L) * (summ["grad_evals"] + run["n_particles"] * K)
                r["flow_traj_tflops"] = fl / (prof["traj_ms"] / 1e3) / 1e12
                if arm == "flow":
                    r["flow_traj_frac_of_fp32_peak"] = r["flow_traj_tflops"] / FP32_FMA_PEAK_TFLOPS
                else:
                    pk = _peaks()[0]
                    r["flow_traj_frac_of_bf16_peak"] = r["flow_traj_tflops"] / pk.get("bf16_tflops_sustained",
                                                                                   pk["bf16_tflops"])
            res[arm] = r
        res["config"] = {"N": run["n_particles"], "K": K, "M_warmup": M, "eps": eps, "flow": f"{L} coupling layers, "
                         f"width {H}, tanh, Adam lr 1e-3, 20 epochs every 2 warm-up iterations, ESS gate 0.25 J; "
                         f"flow: FP32 conditioner products, flow_bf16: BF16 warp-MMA products (training FP32); "
                         f"plain_bf16x3: no map, the Gaussian's P (theta - mu) on BF16x3 warp MMAs"}
        out[name] = res
    return out


def large_logistic_line(g, torch, stream, flush, precision=3):
    """The large Bayesian logistic regression (n = 1e5 observations, D = 100,
    correlated features, 16384 particles, 30 iterations) on the streamed
    tensor-core kernel: one untimed iteration (first launches), then one
    complete device-timed run with the trajectory launches timed by events
    inside the library.  Roofline of the trajectory kernel against the
    sustained BF16 tensor peak: algorithmic FLOPs are 4 n D per gradient
    (X theta and X' r) plus 2 n D per particle for the FP32 end-point energy."""
    w = workloads.logistic_large()
    run = dict(w["run"])
    K, n, D = run["n_iters"], w["n"], w["D"]
    md = g.ModelData.from_workload(w)
    smp = g.Sampler(md, g.make_config(seed=5151, precision=precision, **run), stream)
    smp.run(1)
    smp.reset(6161)
    smp.profile(True)
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    smp.run(K)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = smp.get_profile()
    smp.profile(False)
    summ = smp.summary()[0]
    N = smp.n_total
    smp.close()
    peaks, kind = _peaks()
    flops = 4.0 * n * D * summ["grad_evals"] + 2.0 * n * D * N * K
    achieved = flops / (prof["traj_ms"] / 1e3) / 1e12
    pk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    # chosen vs plain on the same first iterations: the FP32 streamed kernel
    # is ~16x slower per step, so both arms run the first `k_cmp` iterations
    k_cmp = 2
    cmp = {}
    for name, prec in (("bf16x2", precision), ("fp32", 0)):
        sv = g.Sampler(md, g.make_config(seed=5151, precision=prec, **run), stream)
        flush.zero_()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        sv.run(k_cmp)
        c1.record()
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1)
        sm_ = sv.summary()[0]
        sv.close()
        cmp[name] = {"ms": cms, "grad_evals": sm_["grad_evals"], "value": sm_["grad_evals"] / (cms / 1e3),
                     "unit": "particle-grad-evals/s"}
    cmp["iterations"] = k_cmp
    cmp["note"] = "first iterations of the same run (seed 5151): chosen BF16x2 tensor cores vs plain FP32 SIMT"
    return {"workload": WORKLOAD_DESC["logistic_large"], "precision": ["fp32", "bf16x3", "bf16", "bf16x2"][precision],
            "chosen_vs_plain": cmp,
            "value": summ["grad_evals"] / (ms / 1e3), "unit": "particle-grad-evals/s", "ms_per_run": ms,
            "ess_per_s": summ["ess_sum_post_warmup"] / (ms / 1e3), "log_z": summ["log_z"],
            "grad_evals": summ["grad_evals"], "traj_share": prof["traj_ms"] / ms,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                         "peak_source": f"bf16 dense sustained, {kind}",
                         "kernel": "streamed tcgen05 trajectory kernel",
                         "note": "algorithmic FLOPs; the kernel issues 2 products per GEMM (split state operands) "
                                 "and pads D=100 to 112"},
            "l2": "flushed before the run (256 MB write, outside the events)"}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle as it stands, on the host cores, one
    SMC iteration of the workload per step (bounded sample)."""
    import oracle
    w = _workload(args.workload)
    run = dict(w["run"])
    if rank != 0:
        return None
    t = oracle.TargetSpec.logistic(w["X"], w["y"], w.get("tau", 1.0)) if w["kind"] == "logistic" else \
        oracle.TargetSpec.gauss_dense(w["mu"], w["P"])
    cores = os.cpu_count() or 1
    cfg = oracle.SMCConfig(seed=2024, **run)
    st = oracle.smc_init(t, cfg, nthreads=cores)
    st["chees"] = oracle.initial_chees_state(cfg)
    k = 1
    for _ in range(args.warmup):
        oracle.smc_iteration(t, cfg, k, st, nthreads=cores)
        k += 1
    t0 = time.perf_counter()
    ge, ess = 0, 0.0
    for _ in range(args.steps):
        out = oracle.smc_iteration(t, cfg, k, st, nthreads=cores)
        ge += out["stats"]["grad_evals"]
        ess += out["stats"]["ess"]
        k += 1
    dt = time.perf_counter() - t0
    val = ge / dt
    sample = (f"{args.steps} SMC iterations (k={args.warmup + 1}..{k - 1}) of the {args.workload} workload "
              f"after {args.warmup} untimed, N={run['n_particles']}, FP64 C oracle, OpenMP")
    return {"metric": METRIC, "value": val, "unit": "particle-grad-evals/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC[args.workload]},
            "cpu_baseline": {"value": val, "unit": "particle-grad-evals/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "particle-grad-evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "ess_per_s": ess / dt}


METRIC = "particle-grad-evals/s & ESS/s at fixed log-Z error, chosen vs plain FP32 on 1 GB300"
WORKLOAD_DESC = {
    "logistic": "Bayesian logistic regression, synthetic, n=1000, D=25 (intercept + 24 N(0,1) features), "
                "N=4096 particles, K=50 SMC iterations, ChEES-HMC eps=1e-3 L0=5 max 500 steps, 1-d Halton",
    "gauss10": "10-d correlated Gaussian, N=256, K=20",
    "hier": "batched hierarchical normal (non-centred, 50 groups x 20 obs, D=52), 64 independent runs with "
            "particle counts uniform on 512..8192 (seeded, 278k particles) in every launch, K=50, eps=0.01, L0=1, FP32",
    "logistic_large": "Bayesian logistic regression, synthetic, n=100000, D=100 (N(0,1) features with pairwise "
                      "correlation 0.3), N=16384 particles, K=30 SMC iterations, eps=1e-3 L0=5 max 500 steps, "
                      "1-d Halton, streamed tcgen05 BF16x2 gradients",
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="logistic")
    ap.add_argument("--precision", type=int, default=None,
                    help="timed main line: 0 FP32 SIMT, 1 BF16x3 tensor cores (compensated), 2 BF16 tensor "
                         "cores; default: the chosen form, BF16x3 where the model has a tensor-core kernel, "
                         "else FP32")
    ap.add_argument("--variants", default="2",
                    help="precisions also measured (fewer steps) and reported under 'variants'")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-precond", action="store_true",
                    help="skip the learned-preconditioner comparison (two 8192-particle targets)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large logistic regression line (n=1e5, D=100, 16384 particles)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    import torch
    import paper_2504_02627_gb300 as g

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream().cuda_stream

    w = _workload(args.workload)
    run = dict(w["run"])
    K = run["n_iters"]
    md = g.ModelData.from_workload(w)
    batched = "run_sizes" in w

    def make_configs(seed0, precision):
        if not batched:
            return g.make_config(seed=seed0, precision=precision, **run)
        # uneven independent runs in one handle (particle counts from the workload)
        return [g.make_config(seed=seed0 + r, precision=precision, **dict(run, n_particles=int(nr)))
                for r, nr in enumerate(w["run_sizes"])]

    prec = args.precision
    if prec is None:
        prec = 1
        try:
            g.Sampler(md, make_configs(1, 1), stream).close()
        except RuntimeError:
            prec = 0    # no tensor-core kernel for this model: the chosen form is FP32
    smp = g.Sampler(md, make_configs(1000 + 1000 * rank, prec), stream)
    n_runs = smp.n_runs

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    seeds = [20_000 + 1000 * rank + i for i in range(args.steps)]

    for i in range(args.warmup):
        smp.reset(10_000 + 1000 * rank + i)
        smp.run(K)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    mom_c = [] if not batched else None
    dev_ms, ge_total, ess_post, lz = _timed_runs(torch, smp, K, seeds, flush, mom_c)
    if dist:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    # the paper's Table 1 quantities for the last timed run (outside the events)
    paper_q = None
    s_last = smp.summary()
    n_it = sum(x["iterations"] for x in s_last)
    if n_it > 0:
        n_part = sum(c.n_particles for c in smp._cfg)
        grads_paper = sum(x["grad_evals"] for x in s_last) + n_part * (n_it // len(s_last))
        paper_q = {"grad_evals_per_particle": grads_paper / (n_part * (n_it // len(s_last))),
                   "ess_per_grad_eval": sum(x["ess_sum"] for x in s_last) / grads_paper,
                   "note": "the paper's Table 1 quantities for the last timed run: gradient evaluations per "
                           "particle per iteration counting S_j + 1 (the paper's convention), and J_eff per "
                           "gradient evaluation (sums over the iterations)"}
    prof, prof_ge = _profiled_run(smp, K, 30_000 + rank, flush)
    dev_ms, ge_all, ess_all = aggregate_ranks(torch, dist, dev_ms, ge_total, ess_post, "cuda")
    value = ge_all / (dev_ms / 1e3)

    # ---------------- plain FP32 on the same seeds: the comparison the metric names
    plain = None
    if prec != 0:
        sp = g.Sampler(md, make_configs(1000 + 1000 * rank, 0), stream)
        sp.reset(10_000 + 1000 * rank)
        sp.run(K)
        torch.cuda.synchronize()
        mom_p = [] if not batched else None
        p_ms, p_ge, p_ess, p_lz = _timed_runs(torch, sp, K, seeds, flush, mom_p)
        p_prof, p_prof_ge = _profiled_run(sp, K, 30_000 + rank, flush)
        sp.close()
        fl_grad, fl_end = _flops_per_grad(w)
        p_flops = fl_grad * p_prof_ge + fl_end * smp.n_total * K
        p_ach = p_flops / (p_prof["traj_ms"] / 1e3) / 1e12
        d = np.asarray(lz) - np.asarray(p_lz)
        plain = {"value": p_ge / (p_ms / 1e3), "unit": "particle-grad-evals/s", "ms_per_step": p_ms / len(seeds),
                 "ess_per_s": p_ess / (p_ms / 1e3),
                 "log_z": {"mean": float(np.mean(p_lz)), "sd": float(np.std(p_lz, ddof=1)) if len(p_lz) > 1 else None},
                 "roofline": {"bound": "alu", "achieved": p_ach, "peak": FP32_FMA_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": p_ach / FP32_FMA_PEAK_TFLOPS, "kernel": "FP32 SIMT trajectory kernel"},
                 "log_z_paired_diff": {"mean": float(np.mean(d)),
                                       "sd": float(np.std(d, ddof=1)) if len(d) > 1 else None,
                                       "note": "chosen minus plain, same seeds (same initial particles and "
                                               "momentum streams); compare with the between-seed sd"},
                 "seeds": "the timed seeds of the main line"}
        if mom_c and mom_p:
            # posterior means, chosen minus plain per seed, in posterior sd units
            dm = [np.max(np.abs(mc[0] - mp[0]) / np.sqrt(mp[1])) for mc, mp in zip(mom_c, mom_p)]
            plain["mean_paired_diff_sd_units"] = {"max_over_dims_mean_over_seeds": float(np.mean(dm)),
                                                  "note": "compare with the Monte Carlo error of a mean, "
                                                          "about 1/sqrt(ESS) sd"}

    # ---------------- other precisions of the same workload (tensor-core forms)
    variants = {}
    for pv in [int(x) for x in args.variants.split(",") if x.strip() != ""]:
        if pv == prec or pv == 0:
            continue
        try:
            sv = g.Sampler(md, make_configs(1000 + 1000 * rank, pv), stream)
        except RuntimeError:
            continue    # no kernel for this model at that precision
        sv.reset(5_000 + rank)
        sv.run(K)
        torch.cuda.synchronize()
        nv = max(1, args.steps // 2)
        ms_v, ge_v, ess_v = 0.0, 0, 0.0
        for i in range(nv):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sv.reset(40_000 + 1000 * rank + i)
            sv.run(K)
            e1.record()
            sm_ = sv.summary()
            ms_v += e0.elapsed_time(e1)
            ge_v += sum(x["grad_evals"] for x in sm_)
            ess_v += sum(x["ess_sum_post_warmup"] for x in sm_)
        sv.close()
        variants[["fp32", "bf16x3", "bf16"][pv]] = {
            "value": ge_v / (ms_v / 1e3), "unit": "particle-grad-evals/s", "ms_per_step": ms_v / nv,
            "ess_per_s": ess_v / (ms_v / 1e3), "steps": nv}

    # ---------------- roofline of the trajectory kernel
    peaks, peak_kind = _peaks()
    fl_grad, fl_end = _flops_per_grad(w)
    n_part = smp.n_total
    traj_flops = fl_grad * prof_ge + fl_end * n_part * K
    traj_ms = prof["traj_ms"]
    traj_n = max(1, prof["traj_launches"])
    achieved = traj_flops / traj_n / (traj_ms / traj_n / 1e3) / 1e12
    if prec == 0:
        roof = {"bound": "alu", "achieved": achieved, "peak": FP32_FMA_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_FMA_PEAK_TFLOPS,
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x 2070 MHz (max SM clock)"}
        kfile = "traj_simt.cu"
    else:
        # a kernel inside a long step: the sustained bf16 peak
        pk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                "peak_source": f"bf16 dense sustained, {peak_kind}"}
        kfile = "traj_glm_mma.cu" if w["kind"] in ("logistic", "linear_gauss") and w["D"] <= 32 else "traj_tc.cu"
        ex = _mma_flops_per_grad(w, prec)
        if ex is not None:
            roof["executed"] = (ex[0] * prof_ge + ex[1] * n_part * K) / (traj_ms / 1e3) / 1e12
            roof["executed_note"] = ("MMA FLOP/s actually issued: the three BF16 products of the compensated "
                                     "form, the dimension padded to 32 and the observations to 16")
            ceil = C.c_double()
            if g.lib().smc_k_mma_peak(1 << 14, C.byref(ceil), C.c_void_p(stream)) == 0:
                roof["warp_mma_ceiling"] = ceil.value
                roof["executed_frac_of_warp_mma_ceiling"] = roof["executed"] / ceil.value
                roof["ceiling_note"] = ("issue-rate ceiling of warp-level BF16 MMAs (mma.sync m16n8k16) measured "
                                        "live by smc_k_mma_peak; the kernel's MMAs are of that kind")
    tr = _traffic_for(kfile, args.workload)
    roof["traffic"] = tr
    roof["kernel"] = "trajectory (leapfrog) kernel"
    roof["launches_profiled"] = prof["traj_launches"]
    roof["mean_launch_ms"] = traj_ms / traj_n
    roof["share_of_step_time"] = traj_ms / (dev_ms / args.steps) if dev_ms > 0 else None

    # ---------------- learned preconditioner vs the plain sampler (rank 0, N=1)
    precond = None
    if not args.no_precond and world == 1 and args.workload == "logistic":
        precond = precond_compare(g, torch, stream, flush)
    large = None
    if not args.no_large and world == 1 and args.workload == "logistic":
        large = large_logistic_line(g, torch, stream, flush)

    # ---------------- end to end through the C-ABI with host buffers
    e2e = None
    if not args.no_e2e:
        lib = g.lib()
        h2d = 0
        for a in md.arrays:
            if a is not None:
                h2d += a.nbytes
        D = w["D"]
        theta_h = np.empty((D, n_part), dtype=np.float32)
        logw_h = np.empty(n_part)
        lz_h = np.empty(n_runs)
        times, ge_e = [], 0
        for i in range(max(2, args.steps // 2)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = C.c_void_p()
            c2 = make_configs(30_000 + 100 * i + 1000 * rank, prec)
            if batched:
                arr = (g._binding.SmcConfig * len(c2))(*c2)
                g.check(lib.smc_init_batch(C.byref(h), len(c2), arr, C.byref(md.struct), C.c_void_p(stream)),
                        "smc_init_batch")
            else:
                g.check(lib.smc_init(C.byref(h), C.byref(c2), C.byref(md.struct), C.c_void_p(stream)), "smc_init")
            g.check(lib.smc_run(h, K, None), "smc_run", h)
            g.check(lib.smc_get_particles(h, theta_h.ctypes.data, logw_h.ctypes.data, 0), "particles", h)
            g.check(lib.smc_log_evidence(h, lz_h.ctypes.data_as(C.POINTER(C.c_double))), "evidence", h)
            summ = (g._binding.SmcSummary * n_runs)()
            g.check(lib.smc_get_summary(h, summ), "summary", h)
            lib.smc_destroy(h)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            ge_e += sum(x.grad_evals for x in summ)
        e2e = {"value": ge_e * world / sum(times), "unit": "particle-grad-evals/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(theta_h.nbytes + logw_h.nbytes + lz_h.nbytes),
               "steps": len(times)}

    if dist:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return

    # ---------------- CPU baseline (oracle on the host cores), rank 0, N=1 only
    cpu = None
    if world == 1 and not args.no_cpu_baseline and not batched:
        rate, cores, dt, iters = cpu_oracle_rate(w, run)
        cpu = {"value": rate, "unit": "particle-grad-evals/s", "cores": cores, "kind": "oracle",
               "sample": f"first {iters} SMC iterations of the same workload (N={n_part}, full data), "
                         f"FP64 C oracle, OpenMP, {dt:.1f} s wall"}

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "particle-grad-evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dev_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == 0 else "bf16",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC[args.workload], "step": f"one full sampler run ({K} iterations)",
                   "precision": ["fp32", "bf16x3", "bf16"][prec],
                   "l2": "flushed between timed steps (256 MB write, outside the events)",
                   "parallelism": f"replicas x{world}"},
        "ess_per_s": {"value": ess_all / (dev_ms / 1e3), "unit": "ESS/s",
                      "note": "sum of post-warm-up J_eff over iterations / device time"},
        "log_z": {"mean": float(np.mean(lz)), "sd": float(np.std(lz, ddof=1)) if len(lz) > 1 else None},
        "paper_metrics": paper_q,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "plain_fp32": plain,
        "chosen_vs_plain": None if plain is None else {
            "throughput": value / plain["value"], "ess_per_s": (ess_all / (dev_ms / 1e3)) / plain["ess_per_s"]},
        "variants": variants,
        "preconditioner": precond,
        "large_logistic": large,
        "autotune": smp.plan(),
        "gpu_launches": prof["kernel_launches"] * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
