"""Discrete adjoint of the oracle's solver (FP64), for the gradient of the
probe objective J = sum over steps and probes of |E(x_p)|^2 with respect to
the per-element relative permittivity eps_k and the PML profile parameters
(sigma_max, p_sigma).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The right-hand side of ``maxwell.Discretization`` (curl operator with upwind
flux, WAA terms of eqs. 26-29, dipole source) is restated here operation by
operation with PyTorch FP64 CPU tensors, and the LSERK recursion of
``lserk.step`` is replayed on it; reverse-mode differentiation of that replay
is the exact discrete adjoint of the oracle's time stepping (adjoint of the
recursion res <- A res + dt f, q <- q + B res, and of every linear operator in
f).  Constant data (reference operators, geometry, connectivity, quadrature
points) comes from the NumPy oracle objects; the parameters enter as leaf
tensors:

    eps_k           -> 1/eps_k in eqs. 10, 11 and the flux impedances
                       Z = sqrt(mu/eps) of both sides of every face
    sigma_max, p_s  -> sigma_u(x_q) = sigma_max * d^p_s, d = max(0, (|u|-u0)/L),
                       then eq. 9 (kappa = 1)
"""
from __future__ import annotations

import numpy as np
import torch

from . import lserk
from .solver import dipole_current

DT = torch.float64


def _t(a):
    return torch.as_tensor(np.asarray(a), dtype=DT)


class TorchRHS:
    """The oracle RHS as a differentiable function of (eps, sigma_max, p_sigma)."""

    def __init__(self, sim):
        ref, g, d = sim.ref, sim.geom, sim.disc
        if sim.disc.profile is None:
            raise ValueError("needs a PML profile")
        self.prof = sim.disc.profile
        if self.prof.kappa_max != 1.0:
            raise ValueError("the adjoint is written for kappa = 1")
        self.sim = sim
        self.K, self.Np = sim.K, sim.Np
        self.Dr, self.Ds, self.Dt = _t(ref.Dr), _t(ref.Ds), _t(ref.Dt)
        self.LIFT, self.Vq, self.Pq = _t(ref.LIFT), _t(ref.Vq), _t(ref.Pq)
        self.rx, self.ry, self.rz = _t(g.rx), _t(g.ry), _t(g.rz)
        self.sx, self.sy, self.sz = _t(g.sx), _t(g.sy), _t(g.sz)
        self.tx, self.ty, self.tz = _t(g.tx), _t(g.ty), _t(g.tz)
        self.vmapM = torch.as_tensor(g.vmapM.reshape(-1))
        self.vmapP = torch.as_tensor(g.vmapP.reshape(-1))
        self.kP = torch.as_tensor((g.vmapP // sim.Np))
        self.n = _t(d.n)
        self.Fsc = _t(d.Fsc)
        self.bnd = torch.as_tensor(d.bnd)
        self.mu = _t(d.mu)
        self.alpha = d.alpha
        self.xq = _t(d.xq)                      # (3, K, Nq)
        self.sources = sim.sources
        self.probes = sim.probes

    # ---------------------------------------------------------------- parts
    def grad(self, u):
        ur, us, ut = u @ self.Dr.T, u @ self.Ds.T, u @ self.Dt.T
        ux = self.rx[:, None] * ur + self.sx[:, None] * us + self.tx[:, None] * ut
        uy = self.ry[:, None] * ur + self.sy[:, None] * us + self.ty[:, None] * ut
        uz = self.rz[:, None] * ur + self.sz[:, None] * us + self.tz[:, None] * ut
        return ux, uy, uz

    def curl(self, F):
        dx = [self.grad(F[c]) for c in range(3)]
        return torch.stack([dx[2][1] - dx[1][2], dx[0][2] - dx[2][0], dx[1][0] - dx[0][1]])

    @staticmethod
    def cross(n, a):
        return torch.stack([n[1] * a[2] - n[2] * a[1], n[2] * a[0] - n[0] * a[2],
                            n[0] * a[1] - n[1] * a[0]])

    def curl_operators(self, E, H, eps):
        K, Np = self.K, self.Np
        n = self.n
        Ef, Hf = E.reshape(3, -1), H.reshape(3, -1)
        EM, EP = Ef[:, self.vmapM].reshape(3, K, -1), Ef[:, self.vmapP].reshape(3, K, -1)
        HM, HP = Hf[:, self.vmapM].reshape(3, K, -1), Hf[:, self.vmapP].reshape(3, K, -1)
        EP = torch.where(self.bnd[None], -EM, EP)
        HP = torch.where(self.bnd[None], HM, HP)
        dE, dH = EP - EM, HP - HM
        Z = torch.sqrt(self.mu / eps)
        ZM = Z[:, None].expand(K, self.kP.shape[1])
        ZP = Z[self.kP]
        YM, YP = 1.0 / ZM, 1.0 / ZP
        al = self.alpha
        fluxH = (ZP * self.cross(n, dH) - al * self.cross(n, self.cross(n, dE))) / (ZM + ZP)
        fluxE = (YP * self.cross(n, dE) + al * self.cross(n, self.cross(n, dH))) / (YM + YP)
        L = self.LIFT
        CE = self.curl(E) + torch.stack([(self.Fsc * fluxE[c]) @ L.T for c in range(3)])
        CH = self.curl(H) + torch.stack([(self.Fsc * fluxH[c]) @ L.T for c in range(3)])
        return CE, CH

    def coefficients(self, sigma_max, p_sigma):
        pr = self.prof
        sig = []
        for u in range(3):
            depth = (torch.abs(self.xq[u]) - pr.u0) / pr.L
            pos = depth > 0
            safe = torch.where(pos, depth, torch.ones_like(depth))
            sig.append(torch.where(pos, sigma_max * safe ** p_sigma, torch.zeros_like(depth)))
        eps0 = pr.eps0
        b, c, d = [], [], []
        for u in range(3):
            v, w = (u + 1) % 3, (u + 2) % 3
            bu = (sig[v] + sig[w] - sig[u]) / eps0          # eq. 9 with kappa = 1
            b.append(bu)
            c.append(sig[v] * sig[w] / eps0 ** 2 - bu * sig[u] / eps0)
            d.append(sig[u] / eps0)
        return b, c, d

    def rhs(self, q, t, batch, eps, coef):
        E, H, PE, PH = q
        CE, CH = self.curl_operators(E, H, eps)
        CH = CH.clone()
        for (s, k, w) in self.sources:
            if s.batch != batch:
                continue
            jt = dipole_current(s, t)
            for u in range(3):
                CH[u, k] = CH[u, k] - jt * s.dir[u] * _t(w)
        b, c, d = coef
        vq = lambda f: f @ self.Vq.T
        pq = lambda f: f @ self.Pq.T
        mu, ep = self.mu[:, None], eps[:, None]
        oE, oH, oPE, oPH = [], [], [], []
        for u in range(3):
            vH, vPH, vE, vPE = vq(H[u]), vq(PH[u]), vq(E[u]), vq(PE[u])
            # eqs. 26-29 with a = 1 (P_q a^{-1} V_q written out, as in the NumPy oracle)
            oH.append(-pq(vq(pq(b[u] * vH + c[u] * vPH) + CE[u] / mu)))
            oE.append(-pq(vq(pq(b[u] * vE + c[u] * vPE) - CH[u] / ep)))
            oPH.append(pq(vH - d[u] * vPH))
            oPE.append(pq(vE - d[u] * vPE))
        return torch.stack(oE), torch.stack(oH), torch.stack(oPE), torch.stack(oPH)

    # --------------------------------------------------------------- driver
    def objective(self, eps, sigma_max, p_sigma, nsteps, dt, batch=0):
        """J over nsteps LSERK steps from a zero state (FP64, differentiable)."""
        K, Np = self.K, self.Np
        coef = self.coefficients(sigma_max, p_sigma)
        q = [torch.zeros(3, K, Np, dtype=DT) for _ in range(4)]
        res = [torch.zeros(3, K, Np, dtype=DT) for _ in range(4)]
        J = torch.zeros((), dtype=DT)
        ells = [(k, _t(ell)) for (k, ell) in self.probes]
        for n in range(nsteps):
            t = n * dt
            for i in range(5):
                f = self.rhs(q, t + lserk.RK_C[i] * dt, batch, eps, coef)
                res = [lserk.RK_A[i] * r + dt * fi for r, fi in zip(res, f)]
                q = [qi + lserk.RK_B[i] * r for qi, r in zip(q, res)]
            for (k, ell) in ells:
                for u in range(3):
                    J = J + (ell @ q[0][u, k]) ** 2
        return J


def gradient(sim, eps, sigma_max, p_sigma, nsteps, dt, batch=0):
    """(J, dJ/deps [K], dJ/dsigma_max, dJ/dp_sigma) by reverse-mode
    differentiation of the replayed time stepping."""
    tr = TorchRHS(sim)
    e = torch.tensor(np.asarray(eps, np.float64), requires_grad=True)
    sm = torch.tensor(float(sigma_max), dtype=DT, requires_grad=True)
    ps = torch.tensor(float(p_sigma), dtype=DT, requires_grad=True)
    J = tr.objective(e, sm, ps, nsteps, dt, batch)
    J.backward()
    return float(J.detach()), e.grad.numpy().copy(), float(sm.grad), float(ps.grad)
