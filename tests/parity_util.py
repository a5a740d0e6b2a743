"""Shared helpers of the GPU parity tests: set up the same workload on the
library (through the C ABI) and on the oracle, convert state layouts, and
compare.  The oracle side never sees a value produced by the library."""
from __future__ import annotations

import numpy as np

from oracle.solver import Simulation
from synthetic import cube_tet_mesh

FIELDS = ("E", "H", "PE", "PH")


def pml_mask(vxyz, etov, prof):
    """Elements the library carries P^E, P^H for: a vertex beyond u0 on an
    active axis (the classing rule stated in include/wadg.h)."""
    if prof is None:
        return np.zeros(etov.shape[0], bool)
    v = vxyz[etov]                                   # (K, 4, 3)
    active = (prof.sigma_max > 0) or (prof.kappa_max != 1.0)
    if not active:
        return np.zeros(etov.shape[0], bool)
    return np.any(np.abs(v) > prof.u0, axis=(1, 2))


def to_lib(states):
    """oracle states (list over batch of dicts (3,K,Np)) -> [nb][K][12][Np]"""
    out = []
    for st in states:
        out.append(np.concatenate([np.transpose(st[f], (1, 0, 2)) for f in FIELDS], axis=1))
    return np.ascontiguousarray(np.stack(out))


def from_lib(q):
    states = []
    for b in range(q.shape[0]):
        states.append({f: np.ascontiguousarray(np.transpose(q[b][:, 3 * i:3 * i + 3], (1, 0, 2)))
                       for i, f in enumerate(FIELDS)})
    return states


def random_states(K, Np, n_batch, seed, mask=None):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_batch):
        st = {f: rng.normal(size=(3, K, Np)) for f in FIELDS}
        if mask is not None:
            for f in ("PE", "PH"):
                st[f][:, ~mask] = 0.0
        out.append(st)
    return out


def rel_err(q_lib, states_ref, mask):
    """Relative L2 error over E, H of all elements and P of PML elements."""
    ref = to_lib(states_ref)
    sel = np.ones(ref.shape[:3], bool)
    sel[:, ~mask, 6:] = False
    d = (q_lib - ref)[sel]
    return float(np.linalg.norm(d) / max(np.linalg.norm(ref[sel]), 1e-300))


def increment_err(q_lib, states_ref, q0, mask):
    """Relative L2 error of the stage increment: |q_lib - q_ref| / |q_ref - q0|
    over E, H of all elements and P of PML elements.  One stage changes the
    state by a fraction of its size (dt |f(q)| against |q|), so dividing by the
    increment, not by the state, keeps the bound on the part the kernel
    computes."""
    ref = to_lib(states_ref)
    sel = np.ones(ref.shape[:3], bool)
    sel[:, ~mask, 6:] = False
    inc = (ref - q0)[sel]
    return float(np.linalg.norm((q_lib - ref)[sel]) / max(np.linalg.norm(inc), 1e-300))


def round_states(states, precision):
    """Inputs of a non-FP64 comparison rounded to FP32 on both sides, so that
    the error measured is that of the stage and not of storing its input."""
    if precision == "fp64":
        return states
    return [{f: st[f].astype(np.float32).astype(np.float64) for f in st} for st in states]


def make_pair(N, n_hex, jitter, seed, prof, precision="fp64", sources=(), probes=(),
              eps=None, mu=None, n_batch=1, scheme="waa", mesh=None, volume_rule=None):
    """scheme: "waa", "stored" (eqs. 10-13) or "ec" (the weight-adjusted
    scheme with the profile evaluated at each element's centroid).  mesh:
    (vertices, elements) to use instead of the jittered cube.  volume_rule:
    (nq, 4) points and weights given to both sides instead of the default."""
    from paper_2006_02551_gb300 import Solver
    v, e = cube_tet_mesh(n_hex, jitter, seed) if mesh is None else mesh
    sim = Simulation(N, v, e, profile=prof, eps=eps, mu=mu, sources=sources,
                     probes=probes, n_batch=n_batch,
                     scheme="stored" if scheme == "stored" else "waa",
                     volume_rule=volume_rule)
    if scheme == "ec" and prof is not None:
        sim.disc.set_profile(prof, element_constant_at=sim.geom.verts.mean(axis=1).T)
    s = Solver(N, precision, n_batch=n_batch)
    if volume_rule is not None:
        s.set_quadrature(volume_rule)
    s.set_mesh(v, e)
    if eps is not None or mu is not None:
        s.set_materials(eps, mu)
    s.set_pml(prof, scheme)
    if sources:
        s.set_sources(sources)
    if probes:
        s.set_probes(probes)
    return s, sim, pml_mask(v, e, prof)
