"""Jittered structured tetrahedral meshes of the cube [-1, 1]^3.

Each of the n^3 hexahedra is split into six tetrahedra that share the
diagonal from the hexahedron's lowest corner to its highest corner (the
Kuhn/Freudenthal split).  Every square face is then cut along the same
diagonal from both sides, so the mesh is conforming.  Interior vertices are
moved by independent uniform offsets in [-j*h, j*h] per coordinate; a
coordinate that lies on the cube boundary is not moved, so boundary vertices
stay on their faces.  The paper's meshes are not available; these stand in for
them (Section III uses paved tetrahedral meshes that do not conform to the PML
interface, which is what a jittered Kuhn mesh with a PML shell of arbitrary
thickness gives).
"""
from __future__ import annotations

import itertools

import numpy as np

# The six permutations of the axes; the tetrahedron for permutation p walks
# from corner 000 along axis p[0], then p[1], then p[2] to corner 111.
_PERMS = list(itertools.permutations(range(3)))


def _perm_sign(p):
    s = 1
    p = list(p)
    for i in range(3):
        for j in range(i + 1, 3):
            if p[i] > p[j]:
                s = -s
    return s


def cube_tet_mesh(n: int, jitter: float = 0.0, seed: int = 0):
    """Return (vxyz [nv,3] float64, etov [6 n^3, 4] int64).

    Vertex (i, j, k) of the (n+1)^3 lattice has index i + (n+1)(j + (n+1)k)
    and unjittered position -1 + 2(i, j, k)/n.  Tetrahedra are listed hex by
    hex (hex index ix + n(iy + n iz)), six per hex in the order of
    itertools.permutations(range(3)); every tetrahedron is positively
    oriented, det[v1-v0, v2-v0, v3-v0] > 0.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 2.0 / n
    m = n + 1
    g = np.arange(m)
    kk, jj, ii = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)  # index order
    vxyz = -1.0 + h * lat.astype(np.float64)
    if jitter:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=vxyz.shape)
        on_bdry = (lat == 0) | (lat == n)
        d[on_bdry] = 0.0
        vxyz = vxyz + d

    def vid(i, j, k):
        return i + m * (j + m * k)

    tets = []
    hx, hy, hz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n),
                             indexing="ij")
    # hex order: ix fastest
    order = np.lexsort((hx.ravel(), hy.ravel(), hz.ravel()))
    hxs, hys, hzs = hx.ravel()[order], hy.ravel()[order], hz.ravel()[order]
    corners = []
    for p in _PERMS:
        c = [(0, 0, 0)]
        cur = [0, 0, 0]
        for ax in p:
            cur[ax] = 1
            c.append(tuple(cur))
        if _perm_sign(p) < 0:
            c[1], c[2] = c[2], c[1]
        corners.append(c)
    etov = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for t, c in enumerate(corners):
        for a, (dx, dy, dz) in enumerate(c):
            etov[:, t, a] = vid(hxs + dx, hys + dy, hzs + dz)
    etov = etov.reshape(-1, 4)
    vol6 = _signed_vol6(vxyz, etov)
    if not np.all(vol6 > 0):
        bad = int(np.argmin(vol6))
        raise ValueError(f"jitter inverted tetrahedron {bad} "
                         f"(6*volume {vol6[bad]:.3e}); lower the jitter")
    return vxyz, etov


def box_tet_mesh(n, lo, hi, jitter: float = 0.0, seed: int = 0, periodic=(False, False, False)):
    """Kuhn-split box [lo, hi] with n = (nx, ny, nz) hexahedra per axis.

    Returns (vxyz, etov, vcanon).  Vertex (i, j, k) has index
    i + (nx+1)(j + (ny+1)k) and unjittered position lo + (hi-lo)(i/nx, j/ny,
    k/nz); tetrahedra are listed as in cube_tet_mesh.  On a periodic axis the
    lattice planes 0 and n are identified: vcanon maps every vertex to the
    vertex of index 0 on that axis that it is a translate of (the identity on
    non-periodic axes), and the jitter is drawn per periodic class, so that the
    two boundary surfaces stay exact translates of each other.  On a
    non-periodic axis the boundary coordinate is not jittered.  vcanon is None
    when no axis is periodic.
    """
    n = np.asarray(n, dtype=np.int64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    per = np.asarray(periodic, dtype=bool)
    if np.any(n < 1) or np.any(hi <= lo):
        raise ValueError("bad box")
    if np.any(per & (n < 3)):
        # with two hexahedra a diagonal face and a different face can share
        # their vertex classes; three keep every face's class triple unique
        raise ValueError("a periodic axis needs at least 3 hexahedra")
    h = (hi - lo) / n
    m = n + 1
    kk, jj, ii = np.meshgrid(np.arange(m[2]), np.arange(m[1]), np.arange(m[0]), indexing="ij")
    lat = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
    canon_lat = np.where(per[None, :], lat % n[None, :], lat)
    vid = lambda l: l[..., 0] + m[0] * (l[..., 1] + m[1] * l[..., 2])
    vxyz = lo + h * lat.astype(np.float64)
    if jitter:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-1.0, 1.0, size=vxyz.shape) * (jitter * h)
        d = d[vid(canon_lat)]                     # one draw per periodic class
        on_bdry = ((lat == 0) | (lat == n[None, :])) & ~per[None, :]
        d[on_bdry] = 0.0
        vxyz = vxyz + d
    hx, hy, hz = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    order = np.lexsort((hx.ravel(), hy.ravel(), hz.ravel()))
    hxs, hys, hzs = hx.ravel()[order], hy.ravel()[order], hz.ravel()[order]
    corners = []
    for p in _PERMS:
        c = [(0, 0, 0)]
        cur = [0, 0, 0]
        for ax in p:
            cur[ax] = 1
            c.append(tuple(cur))
        if _perm_sign(p) < 0:
            c[1], c[2] = c[2], c[1]
        corners.append(c)
    nh = int(n[0] * n[1] * n[2])
    etov = np.empty((nh, 6, 4), dtype=np.int64)
    for t, c in enumerate(corners):
        for a, (dx, dy, dz) in enumerate(c):
            etov[:, t, a] = (hxs + dx) + m[0] * ((hys + dy) + m[1] * (hzs + dz))
    etov = etov.reshape(-1, 4)
    vol6 = _signed_vol6(vxyz, etov)
    if not np.all(vol6 > 0):
        raise ValueError("jitter inverted a tetrahedron; lower the jitter")
    vcanon = vid(canon_lat).astype(np.int64) if per.any() else None
    return vxyz, etov, vcanon


def _signed_vol6(vxyz, etov):
    v = vxyz[etov]
    a = v[:, 1] - v[:, 0]
    b = v[:, 2] - v[:, 0]
    c = v[:, 3] - v[:, 0]
    return np.einsum("ij,ij->i", a, np.cross(b, c))
