"""Stretched-coordinate PML coefficients.

Stretching variable s_u = kappa_u(u) + sigma_u(u)/(j w eps0) (eq. 4), with the
profiles of Section III:
    sigma_u(u) = sigma_max * ((|u| - u0)/L)^p_sigma   for |u| > u0, else 0
    kappa_u(u) = 1 + (kappa_max - 1) * ((|u| - u0)/L)^p_sigma  (else 1).
The time-domain CPML tensors (eq. 9), (u, v, w) cyclic in (x, y, z):
    a_uu = kappa_v kappa_w / kappa_u
    b_uu = (sigma_v kappa_w + sigma_w kappa_v - a_uu sigma_u) / (kappa_u eps0)
    c_uu = sigma_v sigma_w / eps0^2 - b_uu sigma_u / eps0
    d_uu = sigma_u / (kappa_u eps0)
    kappa_uu = kappa_u.
"""
from __future__ import annotations

import numpy as np


def stretch_profiles(prof, x):
    """sigma_u, kappa_u at points x (array with leading axis of size 3)."""
    x = np.asarray(x, dtype=np.float64)
    sig = np.zeros_like(x)
    kap = np.ones_like(x)
    for u in range(3):
        depth = (np.abs(x[u]) - prof.u0) / prof.L
        inside = depth > 0
        g = np.where(inside, np.maximum(depth, 0.0) ** prof.p_sigma, 0.0)
        sig[u] = prof.sigma_max * g
        kap[u] = 1.0 + (prof.kappa_max - 1.0) * g
    return sig, kap


def cpml_tensors(sig, kap, eps0=1.0):
    """Diagonal entries a, b, c, d, kappa (each with a leading axis u=0,1,2)
    of eq. 9."""
    a = np.empty_like(sig)
    b = np.empty_like(sig)
    c = np.empty_like(sig)
    d = np.empty_like(sig)
    for u in range(3):
        v, w = (u + 1) % 3, (u + 2) % 3
        a[u] = kap[v] * kap[w] / kap[u]
        b[u] = (sig[v] * kap[w] + sig[w] * kap[v] - a[u] * sig[u]) / (kap[u] * eps0)
        c[u] = sig[v] * sig[w] / eps0 ** 2 - b[u] * sig[u] / eps0
        d[u] = sig[u] / (kap[u] * eps0)
    return a, b, c, d, kap.copy()
