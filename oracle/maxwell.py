"""Semi-discrete SC-PML Maxwell system, both PML schemes (Section II.A).

State: dict of arrays of shape (3, K, Np) -- the nodal values of E, H, P^E,
P^H per Cartesian component.  The oracle carries P^E and P^H on every element
(outside the PML their coefficient c vanishes, so they never feed back).

Curl operator with numerical flux (the unnumbered equation after eq. 15),
in strong form with M_k^{-1} applied (this is the bar-C of eqs. 26, 27):
    Cbar_k(f, f', g, g') = curl f + LIFT (Fscale * flux),
the flux being the upwind (Riemann) flux for isotropic media; the paper leaves
the flux unspecified ("in general involves unknowns from ... k and ...
k'").  Reading: with D = exterior - interior, impedances Z = sqrt(mu/eps),
Y = 1/Z and alpha = 1 (alpha = 0 gives the central flux),
    flux for f = H (drives E):  (Z+ n x DH - alpha n x (n x DE)) / (Z- + Z+)
    flux for f = E (drives H):  (Y+ n x DE + alpha n x (n x DH)) / (Y- + Y+)
so that eps dE/dt = Cbar(H, ...) and mu dH/dt = -Cbar(E, ...) without PML.
Perfect electric conductor faces use the mirror state E+ = -E-, H+ = H-.

Sign reading of eqs. 26, 27: Cbar enters eq. 26 as +mu^{-1} Cbar(E) inside
-P_q a^{-1} V_q[...] and eq. 27 as -eps^{-1} Cbar(H), matching eqs. 5, 6.
Reading of the c-term of eq. 6: c . eps P^E (the text prints mu; eq. 11 and
the frequency-domain derivation need eps; the two agree at eps = mu = 1).

Point dipole source: eps dE/dt = curl H - J with J = p'(t) dir delta(x - x_s);
projected with M_k^{-1} it subtracts p'(t) dir J_k^{-1} M^{-1} l(r_s) from
Cbar(H) in the source element.
"""
from __future__ import annotations

import numpy as np

from .pml import cpml_tensors, stretch_profiles
from .refelem import stroud_rule, tet_basis


def cross(n, a):
    return np.stack([n[1] * a[2] - n[2] * a[1],
                     n[2] * a[0] - n[0] * a[2],
                     n[0] * a[1] - n[1] * a[0]])


class Discretization:
    def __init__(self, ref, geom, eps=None, mu=None, profile=None,
                 alpha=1.0, stored_quad_points=None):
        self.ref, self.geom = ref, geom
        K, Np, Nfp = geom.K, ref.Np, ref.Nfp
        self.K = K
        self.eps = np.ones(K) if eps is None else np.asarray(eps, np.float64)
        self.mu = np.ones(K) if mu is None else np.asarray(mu, np.float64)
        self.alpha = alpha
        g = geom
        # per-trace-node face quantities, shape (K, 4 Nfp)
        rep = lambda a: np.repeat(a, Nfp, axis=1)
        self.n = np.stack([rep(g.nx), rep(g.ny), rep(g.nz)])
        self.Fsc = rep(g.Fscale)
        self.bnd = rep(g.boundary)
        Z = np.sqrt(self.mu / self.eps)
        kP = g.vmapP // Np
        self.ZM = np.repeat(Z[:, None], 4 * Nfp, axis=1)
        self.ZP = Z[kP]
        self.profile = profile
        self.set_profile(profile)
        self.stored_quad_points = stored_quad_points or (ref.N + 6)
        self._stored = None

    # ------------------------------------------------------------ PML data
    def set_profile(self, profile, element_constant_at=None):
        """Coefficient samples a^{-1}, b, c, d, kappa^{-1} at the quadrature
        nodes of every element (eq. 20 samples alpha_k(r_q)).

        element_constant_at: optional (3, K) points; when given, the profile
        is evaluated once per element at that point (test hook for the
        element-constant identity of eq. 18)."""
        self.profile = profile
        ref, g = self.ref, self.geom
        xq = g.map_points(ref.rq, ref.sq, ref.tq)            # (3, K, Nq)
        self.xq = xq
        if profile is None:
            shape = xq.shape
            sig, kap = np.zeros(shape), np.ones(shape)
        elif element_constant_at is not None:
            s1, k1 = stretch_profiles(profile, element_constant_at[:, :, None])
            sig = np.broadcast_to(s1, xq.shape).copy()
            kap = np.broadcast_to(k1, xq.shape).copy()
        else:
            sig, kap = stretch_profiles(profile, xq)
        eps0 = 1.0 if profile is None else profile.eps0
        a, b, c, d, k = cpml_tensors(sig, kap, eps0)
        self.qa_inv, self.qb, self.qc, self.qd = 1.0 / a, b, c, d
        self.qk_inv = 1.0 / k
        self.element_constant_at = element_constant_at
        self._stored = None

    # --------------------------------------------------------------- curl
    def grad(self, u):
        """Physical gradient of nodal fields u (K, Np)."""
        ref, g = self.ref, self.geom
        ur, us, ut = u @ ref.Dr.T, u @ ref.Ds.T, u @ ref.Dt.T
        ux = g.rx[:, None] * ur + g.sx[:, None] * us + g.tx[:, None] * ut
        uy = g.ry[:, None] * ur + g.sy[:, None] * us + g.ty[:, None] * ut
        uz = g.rz[:, None] * ur + g.sz[:, None] * us + g.tz[:, None] * ut
        return ux, uy, uz

    def curl(self, F):
        dx = [self.grad(F[c]) for c in range(3)]       # dx[c][d] = dF_c/dx_d
        return np.stack([dx[2][1] - dx[1][2],
                         dx[0][2] - dx[2][0],
                         dx[1][0] - dx[0][1]])

    def traces(self, F):
        g = self.geom
        Ff = F.reshape(3, -1)
        return Ff[:, g.vmapM], Ff[:, g.vmapP]

    def curl_operators(self, E, H):
        """(Cbar(E, E', H, H'), Cbar(H, H', E, E')) for all elements."""
        n = self.n
        EM, EP = self.traces(E)
        HM, HP = self.traces(H)
        # perfect electric conductor: E+ = -E-, H+ = H-
        EP = np.where(self.bnd[None], -EM, EP)
        HP = np.where(self.bnd[None], HM, HP)
        dE, dH = EP - EM, HP - HM
        ZM, ZP = self.ZM, self.ZP
        YM, YP = 1.0 / ZM, 1.0 / ZP
        al = self.alpha
        fluxH = (ZP * cross(n, dH) - al * cross(n, cross(n, dE))) / (ZM + ZP)
        fluxE = (YP * cross(n, dE) + al * cross(n, cross(n, dH))) / (YM + YP)
        L = self.ref.LIFT
        CE = self.curl(E) + np.stack([(self.Fsc * fluxE[c]) @ L.T for c in range(3)])
        CH = self.curl(H) + np.stack([(self.Fsc * fluxH[c]) @ L.T for c in range(3)])
        return CE, CH

    # -------------------------------------------------------- WAA scheme
    def rhs_waa(self, q, CE, CH):
        """Eqs. 26-29, per component u, with the general a != 1 path."""
        ref = self.ref
        Vq, Pq = ref.Vq, ref.Pq
        vq = lambda f: f @ Vq.T
        pq = lambda f: f @ Pq.T
        mu, eps = self.mu[:, None], self.eps[:, None]
        out = {k: np.empty_like(q["E"]) for k in ("E", "H", "PE", "PH")}
        for u in range(3):
            ai, b, c = self.qa_inv[u], self.qb[u], self.qc[u]
            d, ki = self.qd[u], self.qk_inv[u]
            vH, vPH = vq(q["H"][u]), vq(q["PH"][u])
            vE, vPE = vq(q["E"][u]), vq(q["PE"][u])
            # eq. 26
            out["H"][u] = -pq(ai * vq(pq(b * vH + c * vPH) + CE[u] / mu))
            # eq. 27
            out["E"][u] = -pq(ai * vq(pq(b * vE + c * vPE) - CH[u] / eps))
            # eqs. 28, 29
            out["PH"][u] = pq(ki * vH - d * vPH)
            out["PE"][u] = pq(ki * vE - d * vPE)
        return out

    # ----------------------------------------------------- stored scheme
    def stored_matrices(self):
        """Per-element weighted mass matrices M_k^{alpha,u} (eq. 15) for
        alpha in {a, b, c, d, 1/kappa}, by a high-degree quadrature.  The paper
        writes J_k * integral over Omega_k (eq. 19); reading: J_k times the
        reference-element integral."""
        if self._stored is not None:
            return self._stored
        ref, g = self.ref, self.geom
        rh, sh, th, wh = stroud_rule(self.stored_quad_points)
        Vh = tet_basis(ref.N, rh, sh, th) @ ref.Vinv          # (Nh, Np)
        if self.element_constant_at is not None:
            x = np.broadcast_to(self.element_constant_at[:, :, None],
                                (3, g.K, rh.size))
        else:
            x = g.map_points(rh, sh, th)                       # (3, K, Nh)
        if self.profile is None:
            sig, kap = np.zeros(x.shape), np.ones(x.shape)
        else:
            sig, kap = stretch_profiles(self.profile, x)
        eps0 = 1.0 if self.profile is None else self.profile.eps0
        a, b, c, d, k = cpml_tensors(sig, kap, eps0)
        J = g.J[:, None, None]
        mats = {}
        for name, coef in (("a", a), ("b", b), ("c", c), ("d", d), ("kinv", 1.0 / k)):
            mats[name] = np.stack([
                J * np.einsum("qi,kq,qj->kij", Vh, coef[u] * wh[None, :], Vh)
                for u in range(3)])                            # (3, K, Np, Np)
        mats["Mk"] = J * ref.M[None]                           # (K, Np, Np)
        self._stored = mats
        return mats

    def rhs_stored(self, q, CE, CH):
        """Eqs. 10-13 with the stored per-element matrices."""
        S = self.stored_matrices()
        mv = lambda A, x: np.einsum("kij,kj->ki", A, x)
        solve = lambda A, x: np.linalg.solve(A, x[:, :, None])[:, :, 0]
        mu, eps = self.mu[:, None], self.eps[:, None]
        Mk = S["Mk"]
        out = {k: np.empty_like(q["E"]) for k in ("E", "H", "PE", "PH")}
        for u in range(3):
            Ma, Mb, Mc = S["a"][u], S["b"][u], S["c"][u]
            Md, Mki = S["d"][u], S["kinv"][u]
            out["H"][u] = -solve(Ma, mv(Mb, q["H"][u]) + mv(Mc, q["PH"][u])
                                 + mv(Mk, CE[u]) / mu)
            out["E"][u] = -solve(Ma, mv(Mb, q["E"][u]) + mv(Mc, q["PE"][u])
                                 - mv(Mk, CH[u]) / eps)
            out["PH"][u] = solve(Mk, mv(Mki, q["H"][u]) - mv(Md, q["PH"][u]))
            out["PE"][u] = solve(Mk, mv(Mki, q["E"][u]) - mv(Md, q["PE"][u]))
        return out

    # ----------------------------------------------------------- energy
    def energy(self, q):
        """(1/2) sum_k (eps E^T M_k E + mu H^T M_k H)."""
        M, J = self.ref.M, self.geom.J
        e = 0.0
        for u in range(3):
            E, H = q["E"][u], q["H"][u]
            e += np.sum(self.eps * J * np.einsum("ki,ij,kj->k", E, M, E))
            e += np.sum(self.mu * J * np.einsum("ki,ij,kj->k", H, M, H))
        return 0.5 * e
