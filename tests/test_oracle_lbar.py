"""Pins for the oracle's trajectory-length bookkeeping (Algorithm 2).

Algorithm 2 keeps a moving average that starts at zero, and in every warm-up
iteration m < M_warmup, after the Adam step on log L, folds in the new
length: Lbar <- 0.9 Lbar + 0.1 L_m.  At m = M_warmup (no Adam step there) the
length is set to Lbar and stays there for the rest of the run.  The jitter of
iteration m scales L_{m-1}, the length left by the previous iteration.

The pins run the oracle one iteration at a time and rebuild every expected
value from the lengths the oracle itself reports, so a slip in the order or
the quantity averaged fails one of them:
* the average of log L instead of L, or of the length before the Adam step;
* the freeze one iteration early (m = M_warmup - 1) or not at all;
* an Adam step or an average update at or after M_warmup;
* the jitter scaling the freshly updated length instead of the previous one.
"""
import ctypes as C

import numpy as np

import oracle


def _trace(n_warmup=6, n_iters=10, seed=1003):
    t = oracle.TargetSpec.gauss_dense(np.zeros(2), np.eye(2))
    cfg = oracle.SMCConfig(n_particles=64, n_iters=n_iters, n_warmup=n_warmup, step_size=0.1,
                           traj_len0=5.0, seed=seed, adam_lr=0.1)
    st = oracle.smc_init(t, cfg)
    st["chees"] = oracle.initial_chees_state(cfg)
    st["eps"] = C.c_double(cfg.step_size)
    L_start = float(np.exp(st["chees"].log_L))
    rows = []
    for k in range(1, n_iters + 1):
        out = oracle.smc_iteration(t, cfg, k, st)
        assert out["status"] == 0
        ch = st["chees"]
        rows.append({"L": float(np.exp(ch.log_L)), "Lbar": ch.Lbar, "t": ch.t,
                     "L_used": out["stats"]["traj_len"]})
    return L_start, rows


def test_lbar_is_the_moving_average_of_the_updated_lengths():
    M = 6
    _, rows = _trace(n_warmup=M)
    Ls = [r["L"] for r in rows]
    # the lengths move under Adam, so the average is not a constant
    assert max(Ls[: M - 1]) - min(Ls[: M - 1]) > 1e-3
    for m in range(1, M):
        expect = sum(0.1 * 0.9 ** (m - i) * Ls[i - 1] for i in range(1, m + 1))
        assert abs(rows[m - 1]["Lbar"] - expect) <= 1e-13 * expect, (m, rows[m - 1]["Lbar"], expect)
        # an average of log L (or of exp of the averaged log) differs at this spread
        logavg = sum(0.1 * 0.9 ** (m - i) * np.log(Ls[i - 1]) for i in range(1, m + 1))
        assert abs(rows[m - 1]["Lbar"] - logavg) > 1e-6
        assert rows[m - 1]["t"] == m                      # one Adam step per warm-up iteration


def test_length_freezes_to_lbar_at_m_warmup_and_stays():
    M = 6
    _, rows = _trace(n_warmup=M)
    Ls = [r["L"] for r in rows]
    lbar_before = sum(0.1 * 0.9 ** (M - 1 - i) * Ls[i - 1] for i in range(1, M))
    # iteration M: no Adam step, no average update, L <- Lbar
    assert rows[M - 1]["t"] == M - 1
    assert rows[M - 1]["Lbar"] == rows[M - 2]["Lbar"]
    assert abs(rows[M - 1]["L"] - lbar_before) <= 1e-13 * lbar_before
    # not frozen one iteration early: iteration M-1 still took its Adam step
    assert rows[M - 2]["t"] == M - 1
    assert rows[M - 2]["L"] != rows[M - 3]["Lbar"]
    # frozen afterwards
    for r in rows[M:]:
        assert r["L"] == rows[M - 1]["L"]
        assert r["Lbar"] == rows[M - 1]["Lbar"]
        assert r["t"] == M - 1


def test_jitter_scales_the_previous_iterations_length():
    M = 6
    L0, rows = _trace(n_warmup=M)
    assert rows[0]["L_used"] == L0
    for k in range(2, len(rows) + 1):
        assert rows[k - 1]["L_used"] == rows[k - 2]["L"], k


def test_freeze_at_first_iteration_keeps_initial_length_when_lbar_is_zero():
    # M_warmup = 1: no warm-up iteration feeds the average, which stays at its
    # initial zero; the oracle keeps L rather than setting a zero length
    L0, rows = _trace(n_warmup=1, n_iters=3)
    assert all(r["t"] == 0 and r["Lbar"] == 0.0 for r in rows)
    assert all(r["L"] == L0 for r in rows)
