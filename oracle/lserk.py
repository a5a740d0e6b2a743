"""Explicit time marching (Section II.B mentions only "explicit time
marching"; the integrator is not named).  Reading: the five-stage,
fourth-order, two-register low-storage Runge-Kutta scheme of Carpenter and
Kennedy (1994), whose published coefficients are written out below.

One step from (q, t) with step dt:
    res <- A_i res + dt * f(q, t + c_i dt);  q <- q + B_i res,  i = 0..4,
with A_0 = 0 so that res carries nothing across steps.
"""
from __future__ import annotations

import numpy as np

RK_A = np.array([0.0,
                 -567301805773.0 / 1357537059087.0,
                 -2404267990393.0 / 2016746695238.0,
                 -3550918686646.0 / 2091501179385.0,
                 -1275806237668.0 / 842570457699.0])
RK_B = np.array([1432997174477.0 / 9575080441755.0,
                 5161836677717.0 / 13612068292357.0,
                 1720146321549.0 / 2090206949498.0,
                 3134564353537.0 / 4481467310338.0,
                 2277821191437.0 / 14882151754819.0])


def _stage_times():
    """c_i = the time at which stage i samples f: apply the recursion to
    y' = 1 from y = 0 with dt = 1; the state before stage i is then c_i.
    (The rational form of c_2 that circulates with these coefficients,
    2526269341429/6820363218741, is off by 4e-8 from this value; the decimal
    table of the original publication, 0.3704009573644, agrees with it.)"""
    c = np.zeros(5)
    y, res = 0.0, 0.0
    for i in range(5):
        c[i] = y
        res = RK_A[i] * res + 1.0
        y = y + RK_B[i] * res
    return c


RK_C = _stage_times()


def butcher_tableau():
    """Equivalent Butcher tableau (a, b, c) of the two-register recursion:
    Y_{i+1} = Y_0 + sum_{j<=i} B_j res_j, res_j = sum_{l<=j} (prod_{m=l+1}^j A_m) dt f_l."""
    s = 5
    a = np.zeros((s + 1, s))
    for i in range(s):              # row i+1 gives stage i+1 (row s = final)
        for l in range(i + 1):
            acc = 0.0
            for j in range(l, i + 1):
                prod = 1.0
                for m in range(l + 1, j + 1):
                    prod *= RK_A[m]
                acc += RK_B[j] * prod
            a[i + 1, l] = acc
    return a[:s], a[s], a[:s].sum(axis=1)


def step(f, q, t, dt, res=None):
    """Advance state q (dict of arrays) by one step; f(q, t) -> dict."""
    if res is None:
        res = {k: np.zeros_like(v) for k, v in q.items()}
    for i in range(5):
        rhs = f(q, t + RK_C[i] * dt)
        for k in q:
            res[k] = RK_A[i] * res[k] + dt * rhs[k]
            q[k] = q[k] + RK_B[i] * res[k]
    return q, res
