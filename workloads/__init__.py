"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data (numpy, fixed seeds).  It holds none of the
sampler's arithmetic and is the one module that both the FP64 oracle tests
and the GPU library's tests and benchmark import.

Targets (each returns a dict of float64 numpy arrays plus run settings):

* ``gauss10``   10-d correlated Gaussian N(0, Q diag(lam) Q'), lam log-uniform
                on [1e-2, 1]; q_init N(0, 4I); N=256, K=20.
* ``logistic``  Bayesian logistic regression (Sec. 4, German Credit shape):
                n=1000, D=25 (intercept + 24 N(0,1) features), beta_true ~ N(0,I),
                y ~ Bernoulli(sigmoid(X beta_true)); N=4096, K=50, eps=1e-3.
* ``logistic_large`` n=100000, D=100, equicorrelated (rho=0.3) features;
                N=16384, K=30.
* ``hier``      non-centred hierarchical normal, 50 groups x 20 obs, D=52;
                64 runs with particle counts uniform on 512..8192.
* ``gauss100_cond`` 100-d Gaussian, eigenvalues geometric on [1e-4, 1].
* ``banana50``  50-d banana, pairs x_o ~ N(0,10), x_e ~ N(0.1 (x_o^2 - 10), 1).
* ``paper_gauss5``, ``paper_illcond100``, ``paper_banana2``: Sec. 4 targets.
"""
from __future__ import annotations

import numpy as np

DATA_SEED = 12345
HAAR_SEED = 777
RUN_SEEDS = tuple(range(1000, 1010))
BATCH_SEED = 4242


def haar_orthogonal(D: int, seed: int = HAAR_SEED) -> np.ndarray:
    """Q from the QR factorisation of a seeded Gaussian matrix, columns sign
    fixed by diag(R) so that Q is Haar distributed (Mezzadri 2007)."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((D, D))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def _gauss_from_spectrum(lam: np.ndarray, seed: int) -> dict:
    D = lam.size
    Q = haar_orthogonal(D, seed)
    Sigma = (Q * lam[None, :]) @ Q.T
    P = (Q * (1.0 / lam)[None, :]) @ Q.T
    P = 0.5 * (P + P.T)
    return {"kind": "gauss_dense", "D": D, "mu": np.zeros(D), "P": P, "Sigma": Sigma,
            "eigvals": lam, "c": 0.0}


def gauss10(seed: int = DATA_SEED) -> dict:
    rng = np.random.default_rng(seed)
    lam = 10.0 ** rng.uniform(-2.0, 0.0, size=10)
    t = _gauss_from_spectrum(lam, HAAR_SEED)
    t.update(run=dict(n_particles=256, n_iters=20, n_warmup=10, step_size=0.1,
                      traj_len0=5.0, max_steps=500, init_scale=2.0))
    return t


def logistic(n: int = 1000, d_features: int = 24, seed: int = DATA_SEED) -> dict:
    rng = np.random.default_rng(seed)
    X = np.concatenate([np.ones((n, 1)), rng.standard_normal((n, d_features))], axis=1)
    beta = rng.standard_normal(d_features + 1)
    eta = X @ beta
    y = (rng.uniform(size=n) < 1.0 / (1.0 + np.exp(-eta))).astype(np.float64)
    return {"kind": "logistic", "D": d_features + 1, "n": n, "X": X, "y": y, "tau": 1.0,
            "beta_true": beta,
            "run": dict(n_particles=4096, n_iters=50, n_warmup=25, step_size=1e-3,
                        traj_len0=5.0, max_steps=500, init_scale=1.0)}


def logistic_large(n: int = 100_000, D: int = 100, rho: float = 0.3,
                   seed: int = DATA_SEED) -> dict:
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n, D))
    s = rng.standard_normal((n, 1))
    X = np.sqrt(1.0 - rho) * z + np.sqrt(rho) * s
    beta = rng.standard_normal(D)
    eta = X @ beta
    y = (rng.uniform(size=n) < 1.0 / (1.0 + np.exp(-eta))).astype(np.float64)
    return {"kind": "logistic", "D": D, "n": n, "X": X, "y": y, "tau": 1.0, "beta_true": beta,
            "run": dict(n_particles=16384, n_iters=30, n_warmup=15, step_size=1e-3,
                        traj_len0=5.0, max_steps=500, init_scale=1.0)}


def linear_gauss(n: int = 200, D: int = 6, sigma: float = 0.5, tau: float = 1.0,
                 seed: int = DATA_SEED) -> dict:
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, D))
    beta = rng.standard_normal(D) * tau
    y = X @ beta + sigma * rng.standard_normal(n)
    return {"kind": "linear_gauss", "D": D, "n": n, "X": X, "y": y, "sigma": sigma,
            "tau": tau, "beta_true": beta}


def hier(groups: int = 50, obs: int = 20, sigma: float = 1.0, seed: int = DATA_SEED,
         n_runs: int = 64, n_min: int = 512, n_max: int = 8192) -> dict:
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal()
    tau = np.exp(rng.standard_normal())
    b = mu + tau * rng.standard_normal(groups)
    y = b[:, None] + sigma * rng.standard_normal((groups, obs))
    ybar = y.mean(axis=1)
    ss = ((y - ybar[:, None]) ** 2).sum(axis=1)
    n_g = np.full(groups, float(obs))
    sizes = np.random.default_rng(BATCH_SEED).integers(n_min, n_max + 1, size=n_runs)
    return {"kind": "hier_normal", "D": groups + 2, "n": groups, "ybar": ybar, "n_g": n_g,
            "ss": ss, "sigma": sigma, "y_raw": y, "run_sizes": sizes,
            "run": dict(n_particles=int(sizes.sum()), n_iters=50, n_warmup=25,
                        step_size=0.01, traj_len0=1.0, max_steps=500, init_scale=1.0)}


def gauss100_cond(cond: float = 1e4) -> dict:
    D = 100
    lam = 10.0 ** (-np.log10(cond) * np.arange(D) / (D - 1))
    t = _gauss_from_spectrum(lam, HAAR_SEED)
    t.update(run=dict(n_particles=8192, n_iters=50, n_warmup=25, step_size=0.01,
                      traj_len0=5.0, max_steps=500, init_scale=1.0))
    return t


def banana50() -> dict:
    return {"kind": "banana", "D": 50, "a": 10.0, "b": 0.1,
            "run": dict(n_particles=8192, n_iters=50, n_warmup=25, step_size=0.01,
                        traj_len0=5.0, max_steps=500, init_scale=1.0)}


def paper_gauss5() -> dict:
    """Sec. 4 'Gaussian': D=5, mu=[-4,-2,0,2,4], Sigma=diag(1,1.5,2,2.5,3), eps=0.1."""
    var = np.array([1.0, 1.5, 2.0, 2.5, 3.0])
    return {"kind": "gauss_dense", "D": 5, "mu": np.array([-4.0, -2.0, 0.0, 2.0, 4.0]),
            "P": np.diag(1.0 / var), "Sigma": np.diag(var), "eigvals": var, "c": 0.0,
            "run": dict(n_particles=1000, n_iters=200, n_warmup=100, step_size=0.1,
                        traj_len0=5.0, max_steps=500, init_scale=1.0)}


def paper_illcond100(seed: int = DATA_SEED) -> dict:
    """Sec. 4 'Ill-conditioned Gauss': lam ~ Gamma(shape 0.5, scale 1), Q Haar."""
    rng = np.random.default_rng(seed)
    lam = rng.gamma(0.5, 1.0, size=100)
    t = _gauss_from_spectrum(lam, HAAR_SEED)
    t.update(run=dict(n_particles=1000, n_iters=200, n_warmup=100, step_size=1e-3,
                      traj_len0=5.0, max_steps=500, init_scale=1.0))
    return t


def paper_banana2() -> dict:
    """Sec. 4 'Rosenbrock': theta1 ~ N(0, 10^2), theta2 ~ N(0.03 (theta1^2 - 100), 1)."""
    return {"kind": "banana", "D": 2, "a": 100.0, "b": 0.03,
            "run": dict(n_particles=1000, n_iters=200, n_warmup=100, step_size=0.01,
                        traj_len0=5.0, max_steps=500, init_scale=1.0)}


def flow_init(D: int, H: int = 128, L: int = 4, seed: int = 99) -> np.ndarray:
    """Initial parameters of the affine-coupling flow (layout of the library and
    the oracle: per layer W1 [H x D/2], b1, W2 [H x H], b2, W3 [D x H], b3).
    Hidden weights are normal draws with variance 1 / fan-in (suited to the
    tanh hidden units); the last layer is zero, so the map starts as the
    identity.  A seeded draw shared by both sides."""
    rng = np.random.default_rng(seed)
    Dh = D // 2
    parts = []
    for _ in range(L):
        parts += [rng.standard_normal(H * Dh) * np.sqrt(1.0 / Dh), np.zeros(H),
                  rng.standard_normal(H * H) * np.sqrt(1.0 / H), np.zeros(H),
                  np.zeros(D * H), np.zeros(D)]
    return np.concatenate(parts)

