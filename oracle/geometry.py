"""Affine element geometry and face connectivity (nodal DG setting of
Section II.A: straight-sided tetrahedra, M_k = J_k M, M_k^{-1} = J_k^{-1} M^{-1}).

x(r,s,t) = -(1+r+s+t)/2 v1 + (1+r)/2 v2 + (1+s)/2 v3 + (1+t)/2 v4.
J_k = det(dx/dr); (r_x, r_y, ...) the rows of the inverse Jacobian matrix.
Outward unit normals and surface Jacobians sJ follow from the gradient of the
face's defining reference coordinate (face 1: -grad t, face 2: -grad s,
face 3: grad(r+s+t), face 4: -grad r), sJ = |that gradient| * J_k, and the
face-to-volume scaling is Fscale = sJ / J_k.

Face connectivity is found by matching the vertex triples of faces; the
exterior trace node of each face node is the node of the neighbouring element
at the same physical position.  Faces with no neighbour are the outer wall of
the PML and carry the perfect-electric-conductor condition (Section III).
"""
from __future__ import annotations

import numpy as np

from .refelem import FACE_VERTS


class Geometry:
    def __init__(self, ref, vxyz, etov, vcanon=None):
        """vcanon: optional [nv] periodic identification of the vertices (two
        faces whose vertices have the same representatives are neighbours,
        their nodes matched up to the translation between the two faces)."""
        vxyz = np.asarray(vxyz, dtype=np.float64)
        etov = np.asarray(etov, dtype=np.int64)
        self.ref = ref
        self.K = K = etov.shape[0]
        Np, Nfp = ref.Np, ref.Nfp
        v = vxyz[etov]                       # (K, 4, 3)
        self.verts = v
        # physical node coordinates
        r, s, t = ref.r, ref.s, ref.t
        self.x = self.map_points(r, s, t)    # (3, K, Np)
        # dx/dr = (v2 - v1)/2 etc.
        xr = 0.5 * (v[:, 1] - v[:, 0])
        xs = 0.5 * (v[:, 2] - v[:, 0])
        xt = 0.5 * (v[:, 3] - v[:, 0])
        Jm = np.stack([xr, xs, xt], axis=2)  # (K, 3 xyz, 3 rst)
        self.J = np.linalg.det(Jm)
        if np.any(self.J <= 0):
            raise ValueError("non-positive element Jacobian")
        inv = np.linalg.inv(Jm)              # (K, 3 rst, 3 xyz)
        self.rx, self.ry, self.rz = inv[:, 0, 0], inv[:, 0, 1], inv[:, 0, 2]
        self.sx, self.sy, self.sz = inv[:, 1, 0], inv[:, 1, 1], inv[:, 1, 2]
        self.tx, self.ty, self.tz = inv[:, 2, 0], inv[:, 2, 1], inv[:, 2, 2]
        gr = inv[:, 0, :]
        gs = inv[:, 1, :]
        gt = inv[:, 2, :]
        fn = [-gt, -gs, gr + gs + gt, -gr]   # un-normalised outward normals
        self.nx = np.zeros((K, 4))
        self.ny = np.zeros((K, 4))
        self.nz = np.zeros((K, 4))
        self.sJ = np.zeros((K, 4))
        for f in range(4):
            mag = np.linalg.norm(fn[f], axis=1)
            self.nx[:, f] = fn[f][:, 0] / mag
            self.ny[:, f] = fn[f][:, 1] / mag
            self.nz[:, f] = fn[f][:, 2] / mag
            self.sJ[:, f] = mag * self.J
        self.Fscale = self.sJ / self.J[:, None]
        self._connect(etov, None if vcanon is None else np.asarray(vcanon, np.int64))

    def map_points(self, r, s, t):
        v = self.verts
        r, s, t = (np.asarray(a, dtype=np.float64) for a in (r, s, t))
        l1 = -(1 + r + s + t) / 2
        l2 = (1 + r) / 2
        l3 = (1 + s) / 2
        l4 = (1 + t) / 2
        return np.stack([np.outer(v[:, 0, d], l1) + np.outer(v[:, 1, d], l2)
                         + np.outer(v[:, 2, d], l3) + np.outer(v[:, 3, d], l4)
                         for d in range(3)])

    def _connect(self, etov, vcanon=None):
        ref = self.ref
        K, Np, Nfp = self.K, ref.Np, ref.Nfp
        # faces sharing the same sorted vertex triple (of periodic
        # representatives, when given) are neighbours
        ids = etov if vcanon is None else vcanon[etov]
        keys = np.sort(ids[:, np.array(FACE_VERTS)], axis=2).reshape(-1, 3)
        order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
        ks = keys[order]
        same = np.all(ks[1:] == ks[:-1], axis=1)
        a, b = order[:-1][same], order[1:][same]
        self.EToE = np.tile(np.arange(K)[:, None], (1, 4))
        self.EToF = np.tile(np.arange(4)[None, :], (K, 1))
        eflat, fflat = self.EToE.reshape(-1), self.EToF.reshape(-1)
        eflat[a], fflat[a] = b // 4, b % 4
        eflat[b], fflat[b] = a // 4, a % 4
        self.boundary = self.EToE == np.arange(K)[:, None]   # (K, 4) PEC faces
        # vmapM / vmapP: global node index (k*Np + i) of interior and exterior
        # traces, ordered [k][face][face node]
        fm = np.stack(ref.Fmask)                             # (4, Nfp)
        self.vmapM = (np.arange(K)[:, None] * Np
                      + fm.reshape(1, -1)).astype(np.int64)
        vP = self.vmapM.reshape(K, 4, Nfp).copy()
        X = self.x.reshape(3, -1)
        h = np.cbrt(self.J.min())
        tol = 1e-7 * h
        kk, ff = np.nonzero(~self.boundary)
        for lo in range(0, kk.size, 65536):
            k1, f1 = kk[lo:lo + 65536], ff[lo:lo + 65536]
            k2, f2 = self.EToE[k1, f1], self.EToF[k1, f1]
            idM = k1[:, None] * Np + fm[f1]
            idP = k2[:, None] * Np + fm[f2]
            # translation between the two faces (zero unless periodic)
            fv = np.array(FACE_VERTS)
            shift = (self.verts[k1[:, None], fv[f1]].mean(axis=1)
                     - self.verts[k2[:, None], fv[f2]].mean(axis=1))      # (n, 3)
            d = np.zeros((k1.size, Nfp, Nfp))
            for c in range(3):
                d += (X[c][idM][:, :, None] - shift[:, c, None, None]
                      - X[c][idP][:, None, :]) ** 2
            match = np.argmin(d, axis=2)
            best = np.take_along_axis(d, match[:, :, None], axis=2)
            if np.any(np.sqrt(best) > tol):
                raise ValueError("face node matching failed")
            vP[k1, f1] = np.take_along_axis(idP, match, axis=1)
        self.vmapP = vP.reshape(K, 4 * Nfp)

    def locate(self, x, tol=1e-12):
        """Lowest-index element containing point x (all barycentric coordinates
        >= -tol) and the point's reference coordinates there."""
        x = np.asarray(x, dtype=np.float64)
        v = self.verts
        T = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]],
                     axis=2)
        lam = np.linalg.solve(T, (x[None, :] - v[:, 0])[:, :, None])[:, :, 0]
        lam0 = 1 - lam.sum(axis=1)
        inside = np.all(lam >= -tol, axis=1) & (lam0 >= -tol)
        idx = np.nonzero(inside)[0]
        if idx.size == 0:
            raise ValueError(f"point {x} is outside the mesh")
        k = int(idx[0])
        r, s, t = -1 + 2 * lam[k]
        return k, (r, s, t)
