"""Reference tetrahedron for nodal DG of order N (Section II.A).

Reference element: vertices v1=(-1,-1,-1), v2=(1,-1,-1), v3=(-1,1,-1),
v4=(-1,-1,1), volume 4/3.

* Orthonormal polynomial basis phi_i (the "i-th orthonormal polynomial basis"
  used to define the generalized Vandermonde matrices of eq. 20): the
  collapsed-coordinate (Koornwinder/Dubiner) products of normalised Jacobi
  polynomials.
* Interpolation nodes: the paper only says "nodal DG".  Reading: equispaced
  nodes r = -1 + 2(i, j, k)/N, i+j+k <= N, enumerated with k outermost, then
  j, then i.
* M = (V V^T)^{-1} (eq. 14 on the reference element), Dr/Ds/Dt = V_r V^{-1}
  (so that M Dr is the stiffness matrix of eq. 16), LIFT = M^{-1} E with E the
  face mass matrices (eq. 17), so that M^{-1} F = LIFT.
* Quadrature: a rule of degree 2N+1 (eq. 19).  Reading: the conical-product
  Gauss-Jacobi (Stroud) rule with N+1 points per collapsed direction, which
  has positive weights and degree 2N+1.
* V_q = V_I V^{-1} and P_q = M^{-1} V_q^T W (eqs. 20, 21).
"""
from __future__ import annotations

import functools
import math

import numpy as np
import scipy.special as sps


# ---------------------------------------------------------------- 1-D Jacobi

def jacobi_normalized(x, alpha, beta, n):
    """Jacobi polynomial P_n^(alpha,beta)(x) scaled to unit norm under the
    weight (1-x)^alpha (1+x)^beta on [-1, 1]."""
    x = np.asarray(x, dtype=np.float64)
    h = (2.0 ** (alpha + beta + 1) / (2 * n + alpha + beta + 1)
         * math.gamma(n + alpha + 1) * math.gamma(n + beta + 1)
         / (math.gamma(n + alpha + beta + 1) * math.factorial(n)))
    return sps.eval_jacobi(n, alpha, beta, x) / math.sqrt(h)


def jacobi_normalized_deriv(x, alpha, beta, n):
    """d/dx of jacobi_normalized, from d/dx P_n^(a,b) = (n+a+b+1)/2 P_{n-1}^(a+1,b+1)."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    h = (2.0 ** (alpha + beta + 1) / (2 * n + alpha + beta + 1)
         * math.gamma(n + alpha + 1) * math.gamma(n + beta + 1)
         / (math.gamma(n + alpha + beta + 1) * math.factorial(n)))
    return (0.5 * (n + alpha + beta + 1)
            * sps.eval_jacobi(n - 1, alpha + 1, beta + 1, x) / math.sqrt(h))


# -------------------------------------------------------------- basis on tet

def n_nodes(N):
    return (N + 1) * (N + 2) * (N + 3) // 6


def n_face_nodes(N):
    return (N + 1) * (N + 2) // 2


def mode_indices(N):
    return [(i, j, k) for i in range(N + 1) for j in range(N + 1 - i)
            for k in range(N + 1 - i - j)]


def _collapse(r, s, t):
    """(r,s,t) -> collapsed (a,b,c); the singular edges take a=-1 / b=-1."""
    r, s, t = (np.asarray(v, dtype=np.float64) for v in (r, s, t))
    a = np.full_like(r, -1.0)
    den = -(s + t)
    ok = np.abs(den) > 1e-14
    a[ok] = 2.0 * (1.0 + r[ok]) / den[ok] - 1.0
    b = np.full_like(r, -1.0)
    ok = np.abs(1.0 - t) > 1e-14
    b[ok] = 2.0 * (1.0 + s[ok]) / (1.0 - t[ok]) - 1.0
    return a, b, t.copy()


def tet_basis(N, r, s, t):
    """Vandermonde V[p, m] = phi_m(r_p) of the orthonormal basis
    phi_ijk = 2 sqrt(2) P_i(a) (1-b)^i P_j^(2i+1,0)(b) (1-c)^(i+j) P_k^(2i+2j+2,0)(c)."""
    a, b, c = _collapse(r, s, t)
    cols = []
    for (i, j, k) in mode_indices(N):
        cols.append(2.0 * math.sqrt(2.0)
                    * jacobi_normalized(a, 0, 0, i)
                    * jacobi_normalized(b, 2 * i + 1, 0, j) * (1.0 - b) ** i
                    * jacobi_normalized(c, 2 * i + 2 * j + 2, 0, k)
                    * (1.0 - c) ** (i + j))
    return np.stack(cols, axis=1)


def tet_basis_grad(N, r, s, t):
    """(V_r, V_s, V_t): partial derivatives of the basis by the chain rule
    through the collapsed coordinates, written with the reduced powers of
    (1-b), (1-c) so that the values at the collapsed edges are the limits."""
    a, b, c = _collapse(r, s, t)
    C = 2.0 * math.sqrt(2.0)
    Vr, Vs, Vt = [], [], []
    for (i, j, k) in mode_indices(N):
        fa = jacobi_normalized(a, 0, 0, i)
        dfa = jacobi_normalized_deriv(a, 0, 0, i)
        gb = jacobi_normalized(b, 2 * i + 1, 0, j)
        dgb = jacobi_normalized_deriv(b, 2 * i + 1, 0, j)
        hc = jacobi_normalized(c, 2 * i + 2 * j + 2, 0, k)
        dhc = jacobi_normalized_deriv(c, 2 * i + 2 * j + 2, 0, k)

        def pw(x, e):
            return x ** e if e >= 0 else np.zeros_like(x)

        # d/dr: only through a, da/dr = 4 / ((1-b)(1-c))
        dr = 4.0 * dfa * gb * pw(1 - b, i - 1) * hc * pw(1 - c, i + j - 1)
        if i == 0:
            dr = np.zeros_like(a)
        # d/ds: through a (da/ds = 2(1+a)/((1-b)(1-c))) and b (db/ds = 2/(1-c))
        ds_a = 2.0 * (1 + a) * dfa * gb * pw(1 - b, i - 1) * hc * pw(1 - c, i + j - 1)
        if i == 0:
            ds_a = np.zeros_like(a)
        # d/db of gb (1-b)^i
        dg_full = dgb * pw(1 - b, i) - (i * gb * pw(1 - b, i - 1) if i > 0 else 0.0)
        ds_b = 2.0 * fa * dg_full * hc * pw(1 - c, i + j - 1)
        if i + j == 0:
            ds_b = np.zeros_like(a)
        ds = ds_a + ds_b
        # d/dt: a (same as for s), b (db/dt = (1+b)/(1-c)), c (dc/dt = 1)
        dt_b = fa * dg_full * (1 + b) * hc * pw(1 - c, i + j - 1)
        if i + j == 0:
            dt_b = np.zeros_like(a)
        dh_full = dhc * pw(1 - c, i + j) - ((i + j) * hc * pw(1 - c, i + j - 1)
                                           if i + j > 0 else 0.0)
        dt_c = fa * gb * pw(1 - b, i) * dh_full
        dt = ds_a + dt_b + dt_c
        Vr.append(C * dr)
        Vs.append(C * ds)
        Vt.append(C * dt)
    return (np.stack(Vr, axis=1), np.stack(Vs, axis=1), np.stack(Vt, axis=1))


def tri_basis(N, r, s):
    """Orthonormal basis on the reference triangle (-1,-1),(1,-1),(-1,1):
    psi_ij = sqrt(2) P_i(a) (1-b)^i P_j^(2i+1,0)(b), a = 2(1+r)/(1-s)-1, b = s."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    a = np.full_like(r, -1.0)
    ok = np.abs(1.0 - s) > 1e-14
    a[ok] = 2.0 * (1.0 + r[ok]) / (1.0 - s[ok]) - 1.0
    b = s
    cols = []
    for i in range(N + 1):
        for j in range(N + 1 - i):
            cols.append(math.sqrt(2.0) * jacobi_normalized(a, 0, 0, i)
                        * jacobi_normalized(b, 2 * i + 1, 0, j) * (1 - b) ** i)
    return np.stack(cols, axis=1)


# -------------------------------------------------------------------- nodes

def equispaced_nodes(N):
    """Equispaced nodes; node (i,j,k) at r=-1+2i/N, s=-1+2j/N, t=-1+2k/N,
    enumerated k outermost, then j, then i (i fastest)."""
    pts = []
    for k in range(N + 1):
        for j in range(N + 1 - k):
            for i in range(N + 1 - k - j):
                pts.append((-1 + 2 * i / N, -1 + 2 * j / N, -1 + 2 * k / N))
    p = np.array(pts, dtype=np.float64)
    return p[:, 0], p[:, 1], p[:, 2]


# --------------------------------------------------------------- quadrature

def stroud_rule(n):
    """Conical-product rule with n points per collapsed direction:
    a ~ Gauss-Jacobi(0,0), b ~ Gauss-Jacobi(1,0), c ~ Gauss-Jacobi(2,0);
    r=(1+a)(1-b)(1-c)/4-1, s=(1+b)(1-c)/2-1, t=c, w=w_a w_b w_c/8.
    Exact for polynomials of total degree 2n-1 on the reference tet."""
    xa, wa = sps.roots_jacobi(n, 0, 0)
    xb, wb = sps.roots_jacobi(n, 1, 0)
    xc, wc = sps.roots_jacobi(n, 2, 0)
    A, B, Cc = np.meshgrid(xa, xb, xc, indexing="ij")
    WA, WB, WC = np.meshgrid(wa, wb, wc, indexing="ij")
    r = (1 + A) * (1 - B) * (1 - Cc) / 4 - 1
    s = (1 + B) * (1 - Cc) / 2 - 1
    t = Cc
    w = WA * WB * WC / 8
    return r.ravel(), s.ravel(), t.ravel(), w.ravel()


# ------------------------------------------------------------ the element

# Faces: 1: t=-1, 2: s=-1, 3: r+s+t=-1, 4: r=-1 (reference outward normals
# (0,0,-1), (0,-1,0), (1,1,1)/sqrt3, (-1,0,0)).  Face-local 2-D coordinates:
# (r,s), (r,t), (r,s), (s,t).
FACE_VERTS = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))


class RefElement:
    """volume_rule: optional (nq, 4) array of points (r, s, t) and weights on
    the reference tetrahedron to use for the weight-adjusted terms instead
    of the conical-product rule (Section III uses rules of degree 2p with
    fewer points); it must integrate degree 2N exactly for P_q V_q = I."""

    def __init__(self, N, quad_points_per_dir=None, volume_rule=None):
        if N < 1:
            raise ValueError("N >= 1")
        self.N = N
        self.Np = n_nodes(N)
        self.Nfp = n_face_nodes(N)
        r, s, t = equispaced_nodes(N)
        self.r, self.s, self.t = r, s, t
        V = tet_basis(N, r, s, t)
        self.V = V
        self.Vinv = np.linalg.inv(V)
        self.Minv = V @ V.T
        self.M = np.linalg.inv(self.Minv)
        Vr, Vs, Vt = tet_basis_grad(N, r, s, t)
        self.Dr = Vr @ self.Vinv
        self.Ds = Vs @ self.Vinv
        self.Dt = Vt @ self.Vinv
        # face node lists (ascending node index)
        tol = 1e-10
        self.Fmask = [np.where(np.abs(1 + t) < tol)[0],
                      np.where(np.abs(1 + s) < tol)[0],
                      np.where(np.abs(1 + r + s + t) < tol)[0],
                      np.where(np.abs(1 + r) < tol)[0]]
        face2d = [(r, s), (r, t), (r, s), (s, t)]
        E = np.zeros((self.Np, 4 * self.Nfp))
        for f in range(4):
            fm = self.Fmask[f]
            u, v = face2d[f]
            Vf = tri_basis(N, u[fm], v[fm])
            Mf = np.linalg.inv(Vf @ Vf.T)
            E[np.ix_(fm, np.arange(f * self.Nfp, (f + 1) * self.Nfp))] = Mf
        self.Emat = E
        self.LIFT = self.Minv @ E
        # quadrature of degree 2N+1 (eq. 19), or the caller's rule; V_q, P_q
        # (eqs. 20, 21)
        if volume_rule is not None:
            rule = np.asarray(volume_rule, dtype=np.float64).reshape(-1, 4)
            rq, sq, tq, wq = (rule[:, i].copy() for i in range(4))
        else:
            nq = quad_points_per_dir or (N + 1)
            rq, sq, tq, wq = stroud_rule(nq)
        self.rq, self.sq, self.tq, self.wq = rq, sq, tq, wq
        self.Nq = rq.size
        VI = tet_basis(N, rq, sq, tq)
        self.Vq = VI @ self.Vinv
        self.Pq = self.Minv @ self.Vq.T @ np.diag(wq)

    def lagrange_at(self, r, s, t):
        """Row vector(s) l_i(r) of the nodal basis at reference points."""
        phi = tet_basis(self.N, np.atleast_1d(r), np.atleast_1d(s),
                        np.atleast_1d(t))
        return phi @ self.Vinv

    def interp_matrix(self, r, s, t):
        return self.lagrange_at(r, s, t)


@functools.lru_cache(maxsize=None)
def ref_element(N):
    return RefElement(N)
