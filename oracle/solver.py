"""Time loop of the DGTD solver: sources, probes, objective (FP64 oracle).

Probe readout: E, H at a point x_p = l(r_p)^T q_{k_p} after every full step;
the objective is J = sum over probes and steps of |E(x_p)|^2 in FP64.
Point location takes the lowest-index element whose barycentric coordinates
are all >= -1e-12.

Source time function (Section III prints G(t) = e^{(t-t0)^2/4 tau^2}, which
lacks the minus sign).  Reading: G(t) = exp(-(t-t0)^2 / (4 tau^2)); a point
dipole of moment amplitude*G(t) along `dir` radiates the current
J = amplitude*G'(t)*dir*delta(x - x_s).

Stable step: dt = cfl * 2 / ((N+1)^2 * max_{k,f} Fscale_{k,f}), i.e.
cfl * min(altitude)/(N+1)^2 since 1/Fscale is half the element altitude over
that face.
"""
from __future__ import annotations

import numpy as np

from . import lserk
from .geometry import Geometry
from .maxwell import Discretization
from .refelem import RefElement, ref_element

FIELDS = ("E", "H", "PE", "PH")


def dipole_current(src, t):
    tau = src.width
    g = np.exp(-(t - src.t0) ** 2 / (4.0 * tau * tau))
    return src.amplitude * (-(t - src.t0) / (2.0 * tau * tau)) * g


class Simulation:
    def __init__(self, N, vxyz, etov, profile=None, eps=None, mu=None,
                 sources=(), probes=(), n_batch=1, scheme="waa", alpha=1.0,
                 stored_quad_points=None, vcanon=None, volume_rule=None):
        self.ref = ref_element(N) if volume_rule is None else RefElement(
            N, volume_rule=volume_rule)
        self.geom = Geometry(self.ref, vxyz, etov, vcanon)
        self.disc = Discretization(self.ref, self.geom, eps, mu, profile,
                                   alpha, stored_quad_points)
        self.N, self.K, self.Np = N, self.geom.K, self.ref.Np
        self.n_batch = n_batch
        self.scheme = scheme
        self.sources = []
        for s in sources:
            k, rst = self.geom.locate(np.array(s.x))
            ell = self.ref.lagrange_at(*rst)[0]
            w = (self.ref.Minv @ ell) / self.geom.J[k]        # M_k^{-1} l(r_s)
            self.sources.append((s, k, w))
        self.probes = []
        for p in probes:
            k, rst = self.geom.locate(np.array(p))
            self.probes.append((k, self.ref.lagrange_at(*rst)[0]))

    def zero_state(self):
        return [{f: np.zeros((3, self.K, self.Np)) for f in FIELDS}
                for _ in range(self.n_batch)]

    def stable_dt(self, cfl=1.0):
        return cfl * 2.0 / ((self.N + 1) ** 2 * self.geom.Fscale.max())

    def rhs(self, q, t, batch=0):
        CE, CH = self.disc.curl_operators(q["E"], q["H"])
        for (s, k, w) in self.sources:
            if s.batch != batch:
                continue
            jt = dipole_current(s, t)
            for u in range(3):
                CH[u, k] -= jt * s.dir[u] * w
        if self.scheme == "waa":
            return self.disc.rhs_waa(q, CE, CH)
        if self.scheme == "stored":
            return self.disc.rhs_stored(q, CE, CH)
        raise ValueError(self.scheme)

    def probe_values(self, q):
        """(nprobe, 6) array of (Ex,Ey,Ez,Hx,Hy,Hz) at the probes."""
        out = np.zeros((len(self.probes), 6))
        for i, (k, ell) in enumerate(self.probes):
            for u in range(3):
                out[i, u] = ell @ q["E"][u, k]
                out[i, 3 + u] = ell @ q["H"][u, k]
        return out

    def run(self, states, nsteps, dt, t=0.0, record=True):
        """Advance every excitation by nsteps; returns (states, t, probes,
        objective) with probes shaped [nsteps][nprobe][6][n_batch]."""
        nb = self.n_batch
        rec = np.zeros((nsteps, len(self.probes), 6, nb)) if record else None
        J = 0.0
        for b in range(nb):
            f = lambda qq, tt, b=b: self.rhs(qq, tt, b)
            tb = t
            res = None
            for n in range(nsteps):
                states[b], res = lserk.step(f, states[b], tb, dt, res)
                tb = t + (n + 1) * dt
                if record and self.probes:
                    pv = self.probe_values(states[b])
                    rec[n, :, :, b] = pv
                    J += float(np.sum(pv[:, :3] ** 2))
        return states, t + nsteps * dt, rec, J

    def energy(self, q):
        return self.disc.energy(q)
