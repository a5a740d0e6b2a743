"""Workload definitions: mesh recipe, order, PML profile, sources, probes.

The five workloads mirror the method's intended use: a small FP64 case the
CPU oracle finishes in seconds, a production-size N=4 case, an N=5 precision
case, a batched-excitation case and a differentiation case.  They are plain
parameter records; nothing here evaluates a profile, a source waveform or a
basis function.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np


@dataclass(frozen=True)
class PmlProfile:
    """Parameters of sigma_u(u) = sigma_max * s^p, kappa_u = 1 + (kappa_max-1) s^p,
    s = max(0, (|u| - u0)/L), the profile family of Section III (same u0, L,
    sigma_max, exponent and kappa_max on all three axes)."""
    u0: float = 0.75
    L: float = 0.25
    sigma_max: float = 20.0
    p_sigma: float = 3.0
    kappa_max: float = 1.0
    eps0: float = 1.0


@dataclass(frozen=True)
class Dipole:
    """Point electric dipole: moment G(t) = amplitude*exp(-(t-t0)^2/(4 width^2))
    along the unit vector `dir`, located at `x`, driving excitation `batch`."""
    x: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    dir: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    t0: float = 1.0
    width: float = 0.25
    amplitude: float = 1.0
    batch: int = 0


PROBES8 = tuple((sx * 0.5, sy * 0.5, sz * 0.5)
                for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1))


@dataclass(frozen=True)
class Workload:
    name: str
    n_hex: int                 # hexahedra per cube edge (K = 6 n^3)
    jitter: float              # vertex jitter as a fraction of h = 2/n
    mesh_seed: int
    N: int                     # polynomial order
    pml: PmlProfile
    sources: Tuple[Dipole, ...] = (Dipole(),)
    probes: Tuple[Tuple[float, float, float], ...] = PROBES8
    steps: int = 200
    n_batch: int = 1
    precision: str = "fp64"
    eps_seed: Optional[int] = None   # per-element eps_r ~ U[1,4] when set

    @property
    def K(self) -> int:
        return 6 * self.n_hex ** 3


_PML_SMALL = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0)
_PML_LARGE = PmlProfile(u0=0.8, L=0.2, sigma_max=40.0, p_sigma=3.0)


def random_dipoles(n: int, seed: int) -> Tuple[Dipole, ...]:
    """n dipoles, one per excitation: positions uniform in the ball |x| < 0.5,
    uniformly random unit orientations, pulse widths uniform in [0.15, 0.4],
    pulse centre t0 = 4 * width."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n):
        while True:
            x = rng.uniform(-0.5, 0.5, 3)
            if np.dot(x, x) < 0.25:
                break
        d = rng.normal(size=3)
        d = d / np.linalg.norm(d)
        w = rng.uniform(0.15, 0.4)
        out.append(Dipole(x=tuple(float(v) for v in x),
                          dir=tuple(float(v) for v in d),
                          t0=4.0 * w, width=w, amplitude=1.0, batch=b))
    return tuple(out)


WORKLOADS = {
    # 4^3 x 6 = 384 tets, N=3, sigma_max=20 cubic shell of thickness 0.25
    "cube4_n3": Workload("cube4_n3", 4, 0.15, 0, 3, _PML_SMALL, steps=200),
    # the same with kappa_max = 2 (exercises a != 1)
    "cube4_n3_kappa2": Workload("cube4_n3_kappa2", 4, 0.15, 0, 3,
                                replace(_PML_SMALL, kappa_max=2.0), steps=200),
    # 40^3 x 6 = 384k tets, N=4, sigma_max=40 cubic shell of thickness 0.2
    "cube40_n4": Workload("cube40_n4", 40, 0.2, 1, 4, _PML_LARGE, steps=1000,
                          precision="fp32"),
    # 64^3 x 6 = 1.57M tets, N=5
    "cube64_n5": Workload("cube64_n5", 64, 0.2, 2, 5, _PML_LARGE, steps=500,
                          precision="tf32"),
    # 30^3 x 6 = 162k tets, N=3, 64 independent excitations
    "cube30_n3_batch64": Workload("cube30_n3_batch64", 30, 0.2, 3, 3,
                                  _PML_LARGE, sources=random_dipoles(64, 3),
                                  steps=800, n_batch=64, precision="fp32"),
    # 24^3 x 6 = 83k tets, N=3, eps_r ~ U[1,4]
    "cube24_n3_grad": Workload("cube24_n3_grad", 24, 0.2, 4, 3, _PML_LARGE,
                               steps=2000, precision="fp32", eps_seed=5),
}


def workload(name: str, **overrides) -> Workload:
    w = WORKLOADS[name]
    return replace(w, **overrides) if overrides else w


def eps_r(w: Workload) -> Optional[np.ndarray]:
    """Per-element relative permittivity for workloads that vary it."""
    if w.eps_seed is None:
        return None
    return np.random.default_rng(w.eps_seed).uniform(1.0, 4.0, w.K)
