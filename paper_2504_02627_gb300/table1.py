"""The paper's Table 1 study on the GPU (Sec. 4): gradient evaluations per
particle and effective sample size per gradient evaluation of SMC-ChEES on
the synthetic targets of Sec. 4 -- the 5-d Gaussian, the 100-d ill-conditioned
Gaussian (Gamma(0.5, 1) spectrum, Haar rotation) and the 2-d Rosenbrock --
for each jitter scheme of Sec. 3.2.1 built here (N-d Sobol is not), with the
paper's settings: J = 1000 particles, K = 200 iterations of which the first
100 are burn-in, theta_0 ~ N(0, I), L_0 = 5, 10 runs (batched in one handle),
plain FP32 arithmetic.  Also the squared errors of the final weighted
posterior mean and variance against the closed forms.

    python -m paper_2504_02627_gb300.table1 [--targets gauss5,illcond100,banana2] [--schemes 0,1,2] [--runs 10]
                                            [--adam-lr 0.025,0.1]

--adam-lr runs every cell at each listed Adam step size of the ChEES update
(the paper does not state its Adam constants); scheme 11 is the 1-d Halton
sequence with its J x K index matrix read iteration-major.

Metrics, averaged over runs and all K iterations as in the paper's caption:
grad/N = sum_j (S_j + 1) / J (the paper counts one gradient per particle
beyond the S_j leapfrog steps, hence its 501.00 at the 500-step cap), and
ESS/grad = J_eff / sum_j (S_j + 1).  Prints one JSON line per (target,
scheme) and a markdown table.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

SCHEME_NAMES = ["No Jitter", "1-d Halton", "1-d Uniform", "N-d Halton", "N-d Inverse Halton", "N-d Primes",
                "N-d Inverse Primes", "1-d Golden Ratio", "N-d Equidistant", "N-d Offset Equidistant", "1-D Sobol",
                "1-d Halton (iteration-major)"]
# table order of the paper (its NUTS and N-d Sobol rows are not built here)
TABLE_ORDER = [0, 2, 3, 4, 1, 5, 6, 7, 8, 9, 10]


def _setup():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    import workloads
    from . import _binding as B
    return torch, workloads, B


def closed_form(name: str, w: dict):
    """Posterior mean and marginal variances of the Sec. 4 targets."""
    if name == "banana2":
        # theta1 ~ N(0, a) with a the variance (10^2); theta2 | theta1 ~
        # N(b (theta1^2 - a), 1): E theta2 = 0, Var theta2 = 1 + b^2 2 a^2
        a, b = w["a"], w["b"]
        return np.zeros(2), np.array([a, 1.0 + b * b * 2.0 * a * a])
    return np.asarray(w["mu"], dtype=np.float64), np.diag(np.asarray(w["Sigma"], dtype=np.float64)).copy()


def run_one(name: str, scheme: int, n_runs: int, torch, workloads, B, adam_lr: float = 0.025):
    w = {"gauss5": workloads.paper_gauss5, "illcond100": workloads.paper_illcond100,
         "banana2": workloads.paper_banana2}[name]()
    run = w["run"]
    N, K = run["n_particles"], run["n_iters"]
    s = torch.cuda.current_stream().cuda_stream
    cfgs = [B.make_config(seed=sd, jitter=scheme, precision=B.PREC_FP32, adam_lr=adam_lr, **run)
            for sd in workloads.RUN_SEEDS[:n_runs]]
    smp = B.Sampler(B.ModelData.from_workload(w), cfgs, s)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = smp.run(K, with_stats=True)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    grads = np.array([x["grad_evals"] for x in st], dtype=np.float64).reshape(K, n_runs) + N
    ess = np.array([x["ess"] for x in st]).reshape(K, n_runs)
    th, lw = smp.particles()
    smp.close()
    mu_t, var_t = closed_form(name, w)
    se_m, se_v = [], []
    for r in range(n_runs):
        sl = slice(r * N, (r + 1) * N)
        x, l = th[:, sl].astype(np.float64).T, lw[sl]
        wts = np.exp(l - l.max())
        wts /= wts.sum()
        m = wts @ x
        v = wts @ (x - m) ** 2
        se_m.append(np.mean((m - mu_t) ** 2))
        se_v.append(np.mean((v - var_t) ** 2))
    return {"target": name, "scheme": scheme, "scheme_name": SCHEME_NAMES[scheme], "adam_lr": adam_lr,
            "runs": n_runs,
            "particles": N, "iters": K, "grad_per_N": float(np.mean(grads / N)),
            "ess_per_grad": float(np.mean(ess / grads)), "mean_sq_err": float(np.mean(se_m)),
            "var_sq_err": float(np.mean(se_v)), "wall_s": wall}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--targets", default="gauss5,illcond100,banana2")
    ap.add_argument("--schemes", default=",".join(str(i) for i in TABLE_ORDER))
    ap.add_argument("--runs", type=int, default=10)
    ap.add_argument("--adam-lr", default="0.025")
    args = ap.parse_args(argv)
    torch, workloads, B = _setup()
    rows = []
    lrs = [float(x) for x in args.adam_lr.split(",")]
    for lr in lrs:
        for name in args.targets.split(","):
            for sc in (int(x) for x in args.schemes.split(",")):
                r = run_one(name, sc, args.runs, torch, workloads, B, lr)
                rows.append(r)
                print(json.dumps(r), flush=True)
    targets = list(dict.fromkeys(r["target"] for r in rows))
    print("| Adam lr | scheme | " + " | ".join(f"{t} grad/N | {t} ESS/grad | {t} mean SE | {t} var SE"
                                            for t in targets) + " |")
    print("|---|---|" + "---:|" * (4 * len(targets)))
    for lr in lrs:
        for sc in dict.fromkeys(r["scheme"] for r in rows):
            cells = []
            for t in targets:
                r = next(x for x in rows if x["target"] == t and x["scheme"] == sc and x["adam_lr"] == lr)
                cells += [f"{r['grad_per_N']:.2f}", f"{r['ess_per_grad']:.2e}", f"{r['mean_sq_err']:.2e}",
                          f"{r['var_sq_err']:.2e}"]
            print(f"| {lr:g} | {SCHEME_NAMES[sc]} | " + " | ".join(cells) + " |")


if __name__ == "__main__":
    main()
