"""The closed forms the Table 1 study scores its posterior estimates against
(Sec. 4 targets), checked by direct sampling from each target's generative
definition: the 5-d Gaussian's mean and marginal variances, the
ill-conditioned Gaussian's marginal variances (diag of Q diag(lambda) Q'),
and the Rosenbrock target's E theta = 0, Var theta = (100, 1 + 0.03^2 2 10^4
= 19)."""
import numpy as np

import workloads
from paper_2504_02627_gb300.table1 import closed_form


def test_gauss5_closed_form():
    w = workloads.paper_gauss5()
    m, v = closed_form("gauss5", w)
    rng = np.random.default_rng(1)
    x = rng.multivariate_normal(w["mu"], np.linalg.inv(w["P"]), size=400_000)
    assert np.all(np.abs(x.mean(0) - m) < 5 * np.sqrt(v / x.shape[0]))
    assert np.all(np.abs(x.var(0) - v) < 5 * v * np.sqrt(2.0 / x.shape[0]))


def test_illcond100_closed_form_is_the_covariance_diagonal():
    w = workloads.paper_illcond100()
    m, v = closed_form("illcond100", w)
    np.testing.assert_allclose(v, np.diag(np.linalg.inv(w["P"])), rtol=1e-8)
    assert np.all(m == 0.0)


def test_banana2_closed_form_by_sampling():
    w = workloads.paper_banana2()
    m, v = closed_form("banana2", w)
    np.testing.assert_allclose(v, [100.0, 19.0])
    rng = np.random.default_rng(2)
    n = 2_000_000
    x1 = rng.normal(0.0, np.sqrt(w["a"]), n)
    x2 = rng.normal(w["b"] * (x1 * x1 - w["a"]), 1.0)
    x = np.stack([x1, x2], 1)
    assert np.all(np.abs(x.mean(0) - m) < 5 * np.sqrt(v / n))
    # the variance of theta2 has a heavy-ish tail (theta1^4): 5 SE of a kurtotic variance
    assert abs(x[:, 0].var() - v[0]) < 5 * v[0] * np.sqrt(2.0 / n)
    assert abs(x[:, 1].var() - v[1]) < 0.05 * v[1]
