"""GPU discrete adjoint against the oracle adjoint (exact reverse-mode
derivative of the FP64 oracle) and against central differences of the GPU
forward; checkpoint spacing must not change the gradient."""
import numpy as np
import pytest
import torch

from oracle.adjoint import gradient
from oracle.solver import Simulation
from synthetic import Dipole, PmlProfile, cube_tet_mesh

pytestmark = pytest.mark.gpu

PROF = PmlProfile(u0=0.5, L=0.5, sigma_max=15.0, p_sigma=2.0)
SRC = [Dipole(x=(0.1, 0.05, -0.1), t0=0.4, width=0.15)]
PROBES = [(0.3, 0.2, 0.1), (-0.4, 0.3, 0.2)]
NSTEPS = 20


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def case():
    v, e = cube_tet_mesh(2, 0.15, 4)
    eps = np.random.default_rng(5).uniform(1, 4, e.shape[0])
    sim = Simulation(2, v, e, profile=PROF, eps=eps, sources=SRC, probes=PROBES)
    dt = sim.stable_dt(1.0)
    ref = gradient(sim, eps, PROF.sigma_max, PROF.p_sigma, NSTEPS, dt)
    return v, e, eps, dt, ref


def gpu_solver(v, e, eps, prec, prof=PROF):
    from paper_2006_02551_gb300 import Solver
    s = Solver(2, prec)
    s.set_mesh(v, e)
    s.set_materials(eps)
    s.set_pml(prof)
    s.set_sources(SRC)
    s.set_probes(PROBES)
    s.set_state(None, 0.0)
    return s


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
def test_adjoint_matches_oracle(case, prec, tol):
    v, e, eps, dt, (J, gE, gS, gP) = case
    s = gpu_solver(v, e, eps, prec)
    Jg, ge, gs, gp = s.adjoint(NSTEPS, dt, ckpt_every=7)
    s.close()
    # the three axes share sigma_max and p_sigma in the oracle
    errs = (abs(Jg[0] - J) / abs(J), np.linalg.norm(ge[0] - gE) / np.linalg.norm(gE),
            abs(gs[0].sum() - gS) / abs(gS), abs(gp[0].sum() - gP) / abs(gP))
    print(f"{prec} adjoint vs oracle (J, eps, sigma_max, p_sigma):", ["%.2e" % x for x in errs])
    assert max(errs) < tol, errs


def test_checkpoint_spacing_does_not_change_gradient(case):
    v, e, eps, dt, _ = case
    out = []
    for ck in (1, 6, NSTEPS):
        s = gpu_solver(v, e, eps, "fp64")
        out.append(s.adjoint(NSTEPS, dt, ckpt_every=ck))
        s.close()
    # equal up to the summation order of the atomically accumulated sums
    for o in out[1:]:
        for a, b in zip(out[0], o):
            assert np.allclose(a, b, rtol=1e-12, atol=1e-15 * np.abs(a).max())


def test_adjoint_matches_central_differences_of_gpu_forward(case):
    """20 random directions in (eps_r, sigma_max, p_sigma): the adjoint's
    directional derivative against the central difference (h = 1e-4) of the
    GPU forward objective; sigma_max and p_sigma move all three axes."""
    v, e, eps, dt, _ = case
    s = gpu_solver(v, e, eps, "fp64")
    J, ge, gs, gp = s.adjoint(NSTEPS, dt, ckpt_every=5)

    def Jf(eps_, sm, ps):
        s.set_materials(eps_)
        s.set_pml(PmlProfile(u0=PROF.u0, L=PROF.L, sigma_max=sm, p_sigma=ps))
        s.set_sources(SRC)
        s.set_probes(PROBES)
        s.set_state(None, 0.0)
        s.run_steps(NSTEPS, dt)
        return s.objective()[0]

    rng = np.random.default_rng(11)
    h = 1e-4
    worst = 0.0
    for _ in range(20):
        d = rng.normal(size=eps.size)
        dsm, dps = rng.normal(size=2)
        fd = (Jf(eps + h * d, PROF.sigma_max + h * dsm, PROF.p_sigma + h * dps) -
              Jf(eps - h * d, PROF.sigma_max - h * dsm, PROF.p_sigma - h * dps)) / (2 * h)
        ad = ge[0] @ d + gs[0].sum() * dsm + gp[0].sum() * dps
        worst = max(worst, abs(fd - ad) / abs(fd))
    print(f"adjoint vs central differences, 20 directions: worst relative error {worst:.2e}")
    assert worst < 1e-6
    s.close()


def test_autograd_function(case):
    from paper_2006_02551_gb300.autograd import probe_objective
    from paper_2006_02551_gb300 import Solver
    v, e, eps, dt, (J, gE, gS, gP) = case
    s = Solver(2, "fp64")
    s.set_mesh(v, e)
    s.set_sources(SRC)
    s.set_probes(PROBES)
    er = torch.tensor(eps, requires_grad=True)
    sm = torch.tensor(PROF.sigma_max, dtype=torch.float64, requires_grad=True)
    ps = torch.tensor(PROF.p_sigma, dtype=torch.float64, requires_grad=True)
    out = probe_objective(s, er, sm, ps, PROF, NSTEPS, dt, ckpt_every=10)
    (2.0 * out).backward()
    s.close()
    assert abs(out.item() - J) < 1e-10 * abs(J)
    assert np.linalg.norm(er.grad.numpy() - 2 * gE) < 1e-9 * np.linalg.norm(gE)
    assert abs(sm.grad.item() - 2 * gS) < 1e-9 * abs(gS)
    assert abs(ps.grad.item() - 2 * gP) < 1e-9 * abs(gP)
