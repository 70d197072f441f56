"""Helpers shared by the GPU parity tests: device buffers through torch,
raw pointers and streams for the C-ABI, and the FP32-rounded workload copies
that both sides receive as inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2504_02627_gb300 as g  # noqa: E402
import oracle  # noqa: E402


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def ptr(t):
    return t.data_ptr()


def stream():
    return torch.cuda.current_stream().cuda_stream


def f32r(a):
    """The FP32-representable copy of an input, as FP64 (what both sides see)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rounded_workload(w: dict) -> dict:
    """Casts the model data of a workload to FP32 and back, so that the oracle
    and the GPU library start from identical inputs."""
    w = dict(w)
    for k in ("X", "y", "mu", "P", "ybar", "n_g", "ss"):
        if k in w:
            w[k] = f32r(w[k])
    return w


def oracle_target(w: dict):
    k = w["kind"]
    if k == "gauss_dense":
        return oracle.TargetSpec.gauss_dense(w["mu"], w["P"], w.get("c", 0.0))
    if k == "logistic":
        return oracle.TargetSpec.logistic(w["X"], w["y"], w.get("tau", 1.0))
    if k == "linear_gauss":
        return oracle.TargetSpec.linear_gauss(w["X"], w["y"], w["sigma"], w["tau"])
    if k == "hier_normal":
        return oracle.TargetSpec.hier_normal(w["ybar"], w["n_g"], w["ss"], w["sigma"])
    if k == "banana":
        return oracle.TargetSpec.banana(w["D"], w["a"], w["b"])
    raise ValueError(k)
