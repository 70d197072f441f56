"""Single-launch kernel timings through the kernel-level entry points (a
micro-benchmark and the profiling driver for one trajectory kernel at a time).

    python kernel_bench.py stream --n 20000 --particles 16384 --steps 40
    python kernel_bench.py flow --particles 8192 --steps 8
    python kernel_bench.py flow_train --particles 8192 --precision 2
    python kernel_bench.py latency --iters 20
    python kernel_bench.py glm --particles 4096 --steps 20
    python kernel_bench.py gauss --particles 8192 --steps 20 --eps 0.005 --precision 1

Each run makes seeded synthetic inputs (the workloads of this repository),
launches one target evaluation, then leapfrog trajectories of `--steps` steps
for every particle (one untimed, ten timed back to back, each continuing
from the last), and prints the average event-timed duration of a trajectory
launch as one JSON line.  Under a profiler, the first trajectory launch is
the second launch of the kernel (skip one with `-s 1`).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


def _setup():
    root = os.path.dirname(os.path.abspath(__file__))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    import workloads
    from paper_2504_02627_gb300 import _binding as B
    return torch, workloads, B


def _time(torch, fn, reps=10):
    """Device time of one call: one untimed call, then `reps` back-to-back
    calls between two events on the current stream, averaged (the host's
    launch latency overlaps the previous call's execution)."""
    fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_glm_like(args, streamed):
    torch, workloads, B = _setup()
    s = torch.cuda.current_stream().cuda_stream
    if streamed:
        w = workloads.logistic_large(n=args.n, D=args.dim)
        prec = B.PREC_BF16X2 if args.precision is None else args.precision
    else:
        w = workloads.logistic()
        prec = B.PREC_FP32 if args.precision is None else args.precision
    N, D = args.particles, w["D"]
    dm = B.DevModel(B.ModelData.from_workload(w), s)
    rng = np.random.default_rng(0)
    centre = w.get("beta_true", np.zeros(D))
    th = torch.tensor((centre[None, :] + 0.01 * rng.standard_normal((N, D))).T.astype(np.float32)).cuda()
    th = th.contiguous()
    p = torch.randn(D, N, device="cuda")
    gr = torch.zeros(D, N, device="cuda")
    lp = torch.zeros(N, dtype=torch.float64, device="cuda")
    steps = torch.full((N,), args.steps, dtype=torch.int32, device="cuda")
    lib = B.lib()
    B.check(lib.smc_k_target(dm.h, th.data_ptr(), N, N, lp.data_ptr(), gr.data_ptr(), prec, s), "smc_k_target")
    ms = _time(torch, lambda: B.check(lib.smc_k_leapfrog(dm.h, th.data_ptr(), p.data_ptr(), gr.data_ptr(),
                                                         lp.data_ptr(), steps.data_ptr(), args.eps, N, N, prec, s),
                                      "smc_k_leapfrog"))
    n = w["n"]
    flops = 4.0 * n * D * N * args.steps + 2.0 * n * D * N
    kname = "streamed tcgen05" if streamed else ("FP32 SIMT GLM" if prec == 0 else "warp-MMA GLM")
    return {"kernel": kname, "n": n, "D": D, "particles": N,
            "steps": args.steps, "precision": prec, "ms": ms, "tflops_algorithmic": flops / (ms / 1e3) / 1e12}


def run_gauss(args):
    """The 100-d Gaussian (condition 1e4): FP32 dense kernel (precision 0) or
    the warp-MMA kernel (1: BF16x3, 2: BF16)."""
    torch, workloads, B = _setup()
    s = torch.cuda.current_stream().cuda_stream
    w = workloads.gauss100_cond()
    prec = B.PREC_FP32 if args.precision is None else args.precision
    N, D = args.particles, w["D"]
    dm = B.DevModel(B.ModelData.from_workload(w), s)
    rng = np.random.default_rng(2)
    th = torch.tensor((0.05 * rng.standard_normal((D, N))).astype(np.float32)).cuda()
    p = torch.randn(D, N, device="cuda")
    gr = torch.zeros(D, N, device="cuda")
    lp = torch.zeros(N, dtype=torch.float64, device="cuda")
    steps = torch.full((N,), args.steps, dtype=torch.int32, device="cuda")
    lib = B.lib()
    B.check(lib.smc_k_target(dm.h, th.data_ptr(), N, N, lp.data_ptr(), gr.data_ptr(), prec, s), "smc_k_target")
    ms = _time(torch, lambda: B.check(lib.smc_k_leapfrog(dm.h, th.data_ptr(), p.data_ptr(), gr.data_ptr(),
                                                         lp.data_ptr(), steps.data_ptr(), args.eps, N, N, prec, s),
                                      "smc_k_leapfrog"))
    flops = 2.0 * D * D * N * (args.steps + 1)
    return {"kernel": "dense Gaussian " + ("FP32" if prec == 0 else "warp-MMA"), "D": D, "particles": N,
            "steps": args.steps, "precision": prec, "ms": ms, "tflops_algorithmic": flops / (ms / 1e3) / 1e12}


def run_flow(args):
    torch, workloads, B = _setup()
    s = torch.cuda.current_stream().cuda_stream
    w = workloads.gauss100_cond()
    D, H, L, N = w["D"], args.hidden, args.layers, args.particles
    dm = B.DevModel(B.ModelData.from_workload(w), s)
    rng = np.random.default_rng(1)
    params = workloads.flow_init(D, H, L, seed=5)
    Dh = D // 2
    lsz = H * Dh + H + H * H + H + D * H + D
    for l in range(L):
        o = l * lsz + H * Dh + H + H * H + H
        params[o:o + D * H + D] = 0.1 * rng.standard_normal(D * H + D) / np.sqrt(H)
    par = torch.tensor(params.astype(np.float32)).cuda()
    th = torch.tensor((0.01 * rng.standard_normal((D, N))).astype(np.float32)).cuda()
    p = torch.randn(D, N, device="cuda")
    gr = torch.zeros(D, N, device="cuda")
    lp = torch.zeros(N, dtype=torch.float64, device="cuda")
    steps = torch.full((N,), args.steps, dtype=torch.int32, device="cuda")
    lib = B.lib()
    B.check(lib.smc_k_target(dm.h, th.data_ptr(), N, N, lp.data_ptr(), gr.data_ptr(), 0, s), "smc_k_target")
    prec = B.PREC_FP32 if args.precision is None else args.precision
    ms = _time(torch, lambda: B.check(lib.smc_k_flow_leapfrog(dm.h, H, L, par.data_ptr(), th.data_ptr(), p.data_ptr(),
                                                              gr.data_ptr(), lp.data_ptr(), steps.data_ptr(), args.eps,
                                                              N, N, None, None, None, prec, s), "smc_k_flow_leapfrog"))
    per_grad = L * 4.0 * (Dh * H + H * H + H * D) + 2.0 * D * D
    flops = per_grad * N * (args.steps + 1)
    return {"kernel": "latent-space flow trajectory (" + ("BF16 warp MMA" if prec == B.PREC_BF16 else "FP32 SIMT") + ")",
            "D": D, "hidden": H, "layers": L, "particles": N,
            "steps": args.steps, "ms": ms, "tflops_algorithmic": flops / (ms / 1e3) / 1e12}


def run_flow_train(args):
    """The training gradient of the coupling flow (smc_k_flow_loss_grad: the
    work copies and fragments, the per-CTA gradient kernel, the fixed-order
    reduction) on --particles particles near the 100-d Gaussian's scale, with
    FP32 (--precision 0) or BF16 (2) products."""
    torch, workloads, B = _setup()
    s = torch.cuda.current_stream().cuda_stream
    D, H, L, N = args.dim, args.hidden, args.layers, args.particles
    rng = np.random.default_rng(3)
    params = workloads.flow_init(D, H, L, seed=5)
    Dh = D // 2
    lsz = H * Dh + H + H * H + H + D * H + D
    for l in range(L):
        o = l * lsz + H * Dh + H + H * H + H
        params[o:o + D * H + D] = 0.1 * rng.standard_normal(D * H + D) / np.sqrt(H)
    par = torch.tensor(params.astype(np.float32)).cuda()
    th = torch.tensor(rng.standard_normal((D, N)).astype(np.float32)).cuda()
    W = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    gr = torch.empty(par.numel(), dtype=torch.float32, device="cuda")
    prec = B.PREC_FP32 if args.precision is None else args.precision
    lib = B.lib()
    ms = _time(torch, lambda: B.check(lib.smc_k_flow_loss_grad(D, H, L, par.data_ptr(), th.data_ptr(), W.data_ptr(),
                                                               N, N, gr.data_ptr(), prec, s), "smc_k_flow_loss_grad"))
    # per particle and layer: the conditioner twice (inverse pass, backward
    # recompute), the transposed products and the weight gradients
    flops = 8.0 * L * (Dh * H + H * H + H * D) * N
    return {"kernel": "flow training gradient (" + ("BF16 warp MMA" if prec == B.PREC_BF16 else "FP32 SIMT") + ")",
            "D": D, "hidden": H, "layers": L, "particles": N, "ms": ms,
            "tflops_algorithmic": flops / (ms / 1e3) / 1e12}


def run_latency(args):
    """One SMC run of the 10-d Gaussian workload (256 particles, FP32 thread
    kernel): smc_reset and --iters iterations by graph replay between two
    events, after one untimed run; the time per iteration, best of --reps."""
    torch, workloads, B = _setup()
    import paper_2504_02627_gb300 as g
    s = torch.cuda.current_stream().cuda_stream
    w = workloads.gauss10()
    run = dict(w["run"])
    smp = g.Sampler(g.ModelData.from_workload(w), g.make_config(seed=31, **run), s)
    smp.run(run["n_iters"])
    best = float("inf")
    for r in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        smp.reset(32 + r)
        smp.run(args.iters)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e3 / args.iters)
    smp.close()
    return {"kernel": "SMC iteration latency", "D": w["D"], "particles": run["n_particles"], "iters": args.iters,
            "reps": args.reps, "us_per_iteration": best}


def run_sampler(args):
    """SMC iterations of the centred sampler on a handle (the path the bench
    runs: slot-ordered state, and with --runs > 1 the run-uniform tiles):
    the logistic regression with n observations and --dim coefficients,
    --runs runs of --particles particles each, --iters iterations after one
    untimed iteration; the trajectory stage timed by the library's events."""
    torch, workloads, B = _setup()
    import paper_2504_02627_gb300 as g
    s = torch.cuda.current_stream().cuda_stream
    w = workloads.logistic_large(n=args.n, D=args.dim) if args.dim != 25 else workloads.logistic(n=args.n)
    run = dict(w["run"], n_particles=args.particles, n_iters=args.iters + 1, n_warmup=max(1, args.iters // 2))
    cfgs = [g.make_config(seed=3000 + r, precision=4, **run) for r in range(args.runs)]
    smp = g.Sampler(g.ModelData.from_workload(w), cfgs if args.runs > 1 else cfgs[0], s)
    smp.step(with_stats=False)
    ge0 = sum(x["grad_evals"] for x in smp.summary())
    smp.profile(True)
    for _ in range(args.iters):
        smp.step(with_stats=False)
    torch.cuda.synchronize()
    prof = smp.get_profile()
    ge = sum(x["grad_evals"] for x in smp.summary()) - ge0
    smp.close()
    return {"kernel": "centred sampler", "n": w["n"], "D": w["D"], "runs": args.runs, "particles": args.particles,
            "iters": args.iters, "traj_ms": prof["traj_ms"], "grad_evals": ge,
            "grad_evals_per_traj_s": ge / (prof["traj_ms"] / 1e3)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("which", choices=["stream", "flow", "flow_train", "glm", "gauss", "sampler", "latency"])
    ap.add_argument("--n", type=int, default=20000, help="observations (stream)")
    ap.add_argument("--dim", type=int, default=100, help="coefficients of the streamed regression")
    ap.add_argument("--particles", type=int, default=16384)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--precision", type=int, default=None,
                    help="stream: 2 (BF16), 3 (BF16x2, default) or 4 (centred BF16); glm: 0 (FP32, default), "
                         "1 (BF16x3), 2 (BF16) or 4 (centred BF16); "
                         "flow, flow_train: 0 (FP32, default) or 2 (BF16 products)")
    ap.add_argument("--hidden", type=int, default=128)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--runs", type=int, default=1, help="sampler: runs in the handle")
    ap.add_argument("--iters", type=int, default=3, help="sampler, latency: timed SMC iterations")
    ap.add_argument("--reps", type=int, default=5, help="latency: timed runs (the best is reported)")
    args = ap.parse_args(argv)
    if args.which == "sampler":
        out = run_sampler(args)
    elif args.which == "latency":
        out = run_latency(args)
    elif args.which == "flow":
        out = run_flow(args)
    elif args.which == "flow_train":
        out = run_flow_train(args)
    elif args.which == "gauss":
        out = run_gauss(args)
    else:
        out = run_glm_like(args, streamed=args.which == "stream")
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
