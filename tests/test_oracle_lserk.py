"""Pins of the low-storage Runge-Kutta coefficients: classical order
conditions of the equivalent Butcher tableau, stage-time consistency and the
observed convergence order on y' = lambda y."""
import json
import os

import numpy as np

from oracle import lserk

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_coefficients_match_published_decimals():
    with open(os.path.join(GOLDEN, "lserk_ck94.json")) as f:
        g = json.load(f)
    tol = g["decimal_tolerance"]
    assert np.abs(lserk.RK_A - np.array(g["A"])).max() < tol
    assert np.abs(lserk.RK_B - np.array(g["B"])).max() < tol
    assert np.abs(lserk.RK_C - np.array(g["c"])).max() < tol


def test_order_conditions():
    a, b, c = lserk.butcher_tableau()
    # stage times of the recursion are the row sums
    assert np.allclose(c, lserk.RK_C, rtol=0, atol=1e-14)
    assert abs(b.sum() - 1) < 1e-12
    assert abs(b @ c - 1 / 2) < 1e-12
    assert abs(b @ c ** 2 - 1 / 3) < 1e-12
    assert abs(b @ (a @ c) - 1 / 6) < 1e-12
    assert abs(b @ c ** 3 - 1 / 4) < 1e-12
    assert abs(b @ (c * (a @ c)) - 1 / 8) < 1e-12
    assert abs(b @ (a @ c ** 2) - 1 / 12) < 1e-12
    assert abs(b @ (a @ (a @ c)) - 1 / 24) < 1e-12


def test_stage_times_by_integration_of_constant():
    # y' = 1: after stage i the state equals c_{i+1} dt (and dt after stage 5)
    dt = 0.37
    q = {"y": np.zeros(1)}
    res = {"y": np.zeros(1)}
    for i in range(5):
        res["y"] = lserk.RK_A[i] * res["y"] + dt * 1.0
        q["y"] = q["y"] + lserk.RK_B[i] * res["y"]
        nxt = lserk.RK_C[i + 1] if i < 4 else 1.0
        assert abs(q["y"][0] - nxt * dt) < 1e-14


def test_fourth_order_convergence():
    lam = -1.0 + 2.0j
    errs = []
    for n in (10, 20, 40, 80):
        dt = 1.0 / n
        q = {"y": np.array([1.0 + 0j])}
        res = None
        for k in range(n):
            q, res = lserk.step(lambda qq, t: {"y": lam * qq["y"]}, q, k * dt, dt, res)
        errs.append(abs(q["y"][0] - np.exp(lam)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 3.8), slopes


def test_time_dependent_forcing_uses_stage_times():
    # y' = t^3 integrates exactly by a 4th-order method with the right c_i
    dt = 0.25
    q = {"y": np.zeros(1)}
    res = None
    t = 0.0
    for k in range(4):
        q, res = lserk.step(lambda qq, tt: {"y": np.array([tt ** 3])}, q, t, dt, res)
        t += dt
    assert abs(q["y"][0] - t ** 4 / 4) < 1e-13
