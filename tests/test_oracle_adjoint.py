"""Pins of the oracle adjoint (exact reverse-mode derivative of the replayed
FP64 time stepping): its right-hand side equals the NumPy oracle's, its
objective equals the NumPy run's, and its gradient matches central finite
differences of the NumPy oracle forward in random directions."""
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle.adjoint import TorchRHS, gradient
from oracle.solver import Simulation
from synthetic import Dipole, PmlProfile, cube_tet_mesh

PROF = PmlProfile(u0=0.5, L=0.5, sigma_max=15.0, p_sigma=2.0)
SRC = [Dipole(x=(0.1, 0.05, -0.1), t0=0.4, width=0.15)]
PROBES = [(0.3, 0.2, 0.1), (-0.4, 0.3, 0.2)]


@pytest.fixture(scope="module")
def case():
    v, e = cube_tet_mesh(2, 0.15, 4)
    K = e.shape[0]
    eps = np.random.default_rng(5).uniform(1, 4, K)
    sim = Simulation(2, v, e, profile=PROF, eps=eps, sources=SRC, probes=PROBES)
    return v, e, eps, sim


def test_torch_rhs_equals_numpy_rhs(case):
    v, e, eps, sim = case
    rng = np.random.default_rng(1)
    st = {f: rng.normal(size=(3, sim.K, sim.Np)) for f in ("E", "H", "PE", "PH")}
    r = sim.rhs(st, 0.3, 0)
    tr = TorchRHS(sim)
    coef = tr.coefficients(torch.tensor(PROF.sigma_max, dtype=torch.float64),
                           torch.tensor(PROF.p_sigma, dtype=torch.float64))
    rt = tr.rhs([torch.tensor(st[f]) for f in ("E", "H", "PE", "PH")], 0.3, 0,
                torch.tensor(eps), coef)
    for i, f in enumerate(("E", "H", "PE", "PH")):
        assert np.abs(rt[i].numpy() - r[f]).max() < 1e-13 * np.abs(r[f]).max()


def test_gradient_matches_central_differences(case):
    v, e, eps, sim = case
    dt = sim.stable_dt(1.0)
    nsteps = 20
    J, gE, gS, gP = gradient(sim, eps, PROF.sigma_max, PROF.p_sigma, nsteps, dt)
    z = sim.zero_state()
    _, _, _, Jn = sim.run(z, nsteps, dt)
    assert abs(J - Jn) < 1e-13 * abs(Jn)

    def Jfun(eps_, sm, ps):
        s2 = Simulation(2, v, e, profile=replace(PROF, sigma_max=sm, p_sigma=ps), eps=eps_,
                        sources=SRC, probes=PROBES)
        _, _, _, Jv = s2.run(s2.zero_state(), nsteps, dt)
        return Jv

    h = 1e-5
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.normal(size=eps.size)
        fd = (Jfun(eps + h * d, PROF.sigma_max, PROF.p_sigma)
              - Jfun(eps - h * d, PROF.sigma_max, PROF.p_sigma)) / (2 * h)
        assert abs(fd - gE @ d) < 1e-7 * abs(fd)
    fd = (Jfun(eps, PROF.sigma_max + h, PROF.p_sigma)
          - Jfun(eps, PROF.sigma_max - h, PROF.p_sigma)) / (2 * h)
    assert abs(fd - gS) < 1e-7 * abs(fd)
    fd = (Jfun(eps, PROF.sigma_max, PROF.p_sigma + h)
          - Jfun(eps, PROF.sigma_max, PROF.p_sigma - h)) / (2 * h)
    assert abs(fd - gP) < 1e-7 * abs(fd)
