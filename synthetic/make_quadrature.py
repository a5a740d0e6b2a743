"""Generate fully symmetric volume quadrature rules on the tetrahedron.

Writes ``synthetic/quadrature_rules.json``: for N = 1..5 a rule of degree 2N
(exact for every polynomial of total degree <= 2N) with positive weights and
every point strictly inside the tetrahedron.  Degree 2N is what the weight-
adjusted scheme needs: with it the projection P_q = M^-1 V_q^T W inverts the
interpolation V_q on the degree-N space, and the mass matrix it implies is
exact (Section II.A: rules of degree 2p, with far fewer points than the
conical-product rule of (N+1)^3 points).

The rules are inputs to the method, like the mesh: the paper takes tabulated
rules from the literature, which are not available here, so this script
finds rules of its own.  Nothing of the DGTD method is computed here.

Construction.  A fully symmetric rule is a union of orbits of the group of
vertex permutations acting on barycentric coordinates:
  S4    (1/4, 1/4, 1/4, 1/4)                 1 point,   0 parameters
  S31   (a, a, a, 1 - 3a)                    4 points,  1 parameter
  S22   (a, a, 1/2 - a, 1/2 - a)             6 points,  1 parameter
  S211  (a, a, b, 1 - 2a - b)               12 points,  2 parameters
  S1111 (a, b, c, 1 - a - b - c)            24 points,  3 parameters
each with one weight.  Such a rule is exact for every polynomial of degree
<= d exactly when it is exact for the monomials lambda^alpha whose exponent
vectors alpha are partitions of k <= d into at most four parts (one per
orbit of exponent vectors), whose integrals over the simplex of volume 1 are
3! prod(alpha_i!) / (|alpha| + 3)!.  For each degree the script tries orbit
structures in order of increasing point count, solves the moment equations
by bounded nonlinear least squares from seeded random starts, and keeps the
first solution whose relative moment residuals are below 1e-14.

Run: python synthetic/make_quadrature.py  (a few minutes; deterministic)
"""
from __future__ import annotations

import itertools
import json
import math
import os
import sys

import numpy as np
from scipy.optimize import least_squares

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "quadrature_rules.json")

# reference tetrahedron of the library and the oracle
VERTS = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
REF_VOLUME = 4.0 / 3.0

ORBIT_POINTS = {"S4": 1, "S31": 4, "S22": 6, "S211": 12, "S1111": 24}
ORBIT_PARAMS = {"S4": 0, "S31": 1, "S22": 1, "S211": 2, "S1111": 3}


def partitions(k, parts=4):
    """Exponent vectors: partitions of k into at most `parts` parts, padded."""
    out = []

    def rec(rem, maxp, acc):
        if len(acc) == parts:
            if rem == 0:
                out.append(tuple(acc))
            return
        for p in range(min(rem, maxp), -1, -1):
            rec(rem - p, p, acc + [p])
    rec(k, k, [])
    return out


def exponents(d):
    return [a for k in range(d + 1) for a in partitions(k)]


def simplex_moment(alpha):
    """Integral of prod lambda_i^alpha_i over the simplex of volume 1."""
    return 6.0 * math.prod(math.factorial(a) for a in alpha) / math.factorial(sum(alpha) + 3)


def orbit_bary(kind, u):
    """Barycentric generator of an orbit from unconstrained-in-box params u."""
    if kind == "S4":
        return (0.25, 0.25, 0.25, 0.25)
    if kind == "S31":
        a = u[0] / 3.0                       # u in (0, 1)
        return (a, a, a, 1.0 - 3.0 * a)
    if kind == "S22":
        a = u[0] / 4.0                       # u in (0, 1): a in (0, 1/4)
        return (a, a, 0.5 - a, 0.5 - a)
    if kind == "S211":
        a = u[0] / 2.0
        b = u[1] * (1.0 - 2.0 * a)
        return (a, a, b, 1.0 - 2.0 * a - b)
    if kind == "S1111":
        a = u[0]
        b = u[1] * (1.0 - a)
        c = u[2] * (1.0 - a - b)
        return (a, b, c, 1.0 - a - b - c)
    raise ValueError(kind)


def orbit_points(lam):
    """Distinct permutations of a barycentric 4-tuple."""
    pts = sorted(set(itertools.permutations(lam)))
    return np.array(pts)


def unpack(structure, x):
    """x = [orbit params..., weights...] -> list of [kind, params, weight]."""
    out = []
    i = 0
    for kind in structure:
        n = ORBIT_PARAMS[kind]
        out.append([kind, x[i:i + n]])
        i += n
    for o in out:
        o.append(x[i])
        i += 1
    return out


# index patterns of the distinct permutations of each orbit's generator
# (generators with the repeated entries first, as orbit_bary returns them)
PERMS = {k: np.array(sorted(set(itertools.permutations(pat))))
         for k, pat in (("S4", (0, 0, 0, 0)), ("S31", (0, 0, 0, 3)), ("S22", (0, 0, 2, 2)),
                        ("S211", (0, 0, 2, 3)), ("S1111", (0, 1, 2, 3)))}


def orbit_matrix(structure, u, alphas):
    """A[j, o] = sum over the points of orbit o of lambda^alpha_j."""
    A = np.empty((len(alphas), len(structure)))
    i = 0
    for o, kind in enumerate(structure):
        n = ORBIT_PARAMS[kind]
        g = np.array(orbit_bary(kind, u[i:i + n]))
        i += n
        P = g[PERMS[kind]]                                   # points x 4
        A[:, o] = np.prod(P[:, None, :] ** alphas[None, :, :], axis=2).sum(axis=0)
    return A


def weights_for(structure, u, alphas, target):
    """Weights of least moment residual for fixed orbit positions (the
    moment equations are linear in the weights)."""
    A = orbit_matrix(structure, u, alphas) / target[:, None]
    w = np.linalg.lstsq(A, np.ones(len(target)), rcond=None)[0]
    return w, A


def projected_residual(u, structure, alphas, target):
    w, A = weights_for(structure, u, alphas, target)
    return A @ w - 1.0


def full_residual(x, structure, alphas, target):
    npar = len(x) - len(structure)
    A = orbit_matrix(structure, x[:npar], alphas) / target[:, None]
    return A @ x[npar:] - 1.0


def structures(d, max_points):
    """Orbit structures with at least as many unknowns as independent moment
    equations, ordered by point count (then by fewer large orbits).  On the
    simplex sum(lambda) = 1, so a symmetric polynomial of lower degree times
    a power of sum(lambda) is one of degree d: the independent equations are
    those of the partitions of d itself."""
    neq = len(partitions(d))
    out = []
    for n4 in (0, 1):
        for n31 in range(0, 7):
            for n22 in range(0, 4):
                for n211 in range(0, 6):
                    for n1111 in range(0, 4):
                        unknowns = n4 + 2 * n31 + 2 * n22 + 3 * n211 + 4 * n1111
                        pts = n4 + 4 * n31 + 6 * n22 + 12 * n211 + 24 * n1111
                        nor = n4 + n31 + n22 + n211 + n1111
                        if unknowns >= neq and pts <= max_points and nor <= neq:
                            out.append((pts, n1111, n211, n4, n31, n22))
    out.sort()
    return [(["S4"] * o[3] + ["S31"] * o[4] + ["S22"] * o[5] + ["S211"] * o[2] +
             ["S1111"] * o[1], o[0]) for o in out]


def distinct_orbits(parts, tol=1e-6):
    """Reject solutions whose orbits collapse onto each other or onto a
    smaller orbit (the point count would not be what the structure says)."""
    pts = np.concatenate([orbit_points(np.array(orbit_bary(k, u))) if k != "S4"
                          else np.array([[0.25] * 4]) for k, u, _ in parts])
    expected = sum(ORBIT_POINTS[k] for k, _, _ in parts)
    if len(pts) != expected:
        return False
    dmin = min(np.linalg.norm(pts[i] - pts[j]) for i in range(len(pts)) for j in range(i))
    return dmin > tol


def solve(d, structure, starts, seed):
    """Orbit positions by variable projection from seeded random starts, then
    a Gauss-Newton polish of positions and weights together."""
    rng = np.random.default_rng(seed)
    # homogeneous degree-d exponent vectors (independent equations) plus all
    # lower degrees (consistent, and they keep the problem well scaled)
    alphas = np.array(exponents(d), dtype=float)
    target = np.array([simplex_moment(tuple(int(v) for v in a)) for a in alphas])
    npar = sum(ORBIT_PARAMS[k] for k in structure)
    lo, hi = np.full(max(npar, 1), 1e-4), np.full(max(npar, 1), 1 - 1e-4)
    for _ in range(starts):
        if npar:
            u0 = rng.uniform(0.05, 0.95, npar)
            try:
                sol = least_squares(projected_residual, u0, bounds=(lo, hi),
                                    args=(structure, alphas, target), xtol=1e-14,
                                    ftol=1e-14, gtol=1e-14, max_nfev=200 * npar)
            except ValueError:
                continue
            if np.max(np.abs(sol.fun)) > 1e-9:
                continue
            u = sol.x
        else:
            u = np.zeros(0)
        w, _ = weights_for(structure, u, alphas, target)
        if np.any(w <= 0):
            continue
        x = np.r_[u, w]
        for _ in range(30):
            r = full_residual(x, structure, alphas, target)
            J = np.empty((len(r), len(x)))
            for j in range(len(x)):
                h = 1e-7 * max(1.0, abs(x[j]))
                xp, xm = x.copy(), x.copy()
                xp[j] += h
                xm[j] -= h
                J[:, j] = (full_residual(xp, structure, alphas, target) -
                           full_residual(xm, structure, alphas, target)) / (2 * h)
            dx = np.linalg.lstsq(J, -r, rcond=None)[0]
            x = x + dx
            if np.max(np.abs(dx)) < 1e-16:
                break
        res = float(np.max(np.abs(full_residual(x, structure, alphas, target))))
        parts = unpack(structure, x)
        ok = res < 1e-14 and all(w > 0 for _, _, w in parts)
        ok = ok and all(np.all((np.array(u) > 0) & (np.array(u) < 1)) for _, u, _ in parts)
        if ok and distinct_orbits(parts):
            return parts, res
    return None, None


def expand(parts):
    """(r, s, t, w) of every point, w scaled to the reference volume 4/3."""
    rows = []
    for kind, u, w in parts:
        lam = np.array(orbit_bary(kind, u))
        P = orbit_points(lam) if kind != "S4" else np.array([lam])
        for p in P:
            x = p @ VERTS
            rows.append([float(x[0]), float(x[1]), float(x[2]), float(w * REF_VOLUME)])
    return rows


def _try(args):
    d, structure, pts, starts, seed = args
    parts, res = solve(d, structure, starts, seed)
    return structure, pts, parts, res


def main():
    import multiprocessing as mp
    rules = {}
    limits = {1: 4, 2: 14, 3: 31, 4: 60, 5: 100}
    starts = {1: 20, 2: 40, 3: 60, 4: 60, 5: 60}
    ctx = mp.get_context("spawn")
    for N in range(1, 6):
        d = 2 * N
        found = None
        cands = structures(d, limits[N])
        # structures in order of point count, a batch at a time in parallel;
        # the first batch holding a solution decides (fewest points first)
        with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
            for i0 in range(0, len(cands), 8):
                batch = [(d, st, pts, starts[N], 1000 * N + i0 + j)
                         for j, (st, pts) in enumerate(cands[i0:i0 + 8])]
                res_b = pool.map(_try, batch)
                ok = [r for r in res_b if r[2] is not None]
                for st, pts, parts, res in res_b:
                    print(f"N={N} degree {d}: {pts} points {st}: "
                          f"{'found' if parts is not None else 'none'}", file=sys.stderr, flush=True)
                if ok:
                    ok.sort(key=lambda r: r[1])
                    found = ok[0]
                    break
        if found is None:
            raise SystemExit(f"no rule found for degree {d}")
        structure, pts, parts, res = found
        print(f"N={N} degree {d}: {pts} points {structure} residual {res:.1e}", file=sys.stderr)
        rules[str(N)] = {
            "degree": d,
            "points": pts,
            "orbits": [{"kind": k, "bary": [float(v) for v in orbit_bary(k, u)],
                        "weight_unit_volume": float(w)} for k, u, w in parts],
            "rstw": expand(parts),
        }
    doc = {"about": "fully symmetric positive interior tetrahedron rules of degree 2N "
                    "on the reference tetrahedron (-1,-1,-1),(1,-1,-1),(-1,1,-1),(-1,-1,1); "
                    "rstw rows are r, s, t, weight (weights sum to 4/3); written by "
                    "synthetic/make_quadrature.py",
           "rules": rules}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print(OUT)


if __name__ == "__main__":
    main()
