"""The differentiation workload at full size: 24^3 x 6 = 82,944 jittered tets
(seed 4), N = 3, relative permittivity U[1, 4] (seed 5), the benchmark PML,
objective J = sum over probes and steps of |E|^2.  The FP64 runs these checks
need are too slow for the workload's 2000 steps, so the dipole fires earlier
(t0 = 0.15, width 0.06) and 8 probes sit 0.12-0.2 from it, which puts the
signal at the probes inside the shortened windows (J is then of order one
instead of 1e-35).  The 2000-step FP32 gradient is timed by bench.py.

* The FP32 adjoint (checkpoints every 45 steps) against the FP64 adjoint over
  the same 250 steps: J, dJ/deps_r, dJ/dsigma_max and dJ/dp_sigma agree to
  1e-5 (relative L2; measured 2e-6 to 4e-6; the FP64 adjoint itself matches
  the oracle's reverse-mode derivative to 1e-10 in tests/test_gpu_adjoint.py).
* The FP64 adjoint against central differences (h = 1e-4) of the FP64 forward
  along 3 random directions of eps_r, 250 steps: relative error 1e-6.  (In
  250 steps no wave reaches the PML and returns to the probes, so J does not
  depend on sigma_max or p_sigma here; tests/test_gpu_adjoint.py checks those
  derivatives along 20 random directions on a case where they matter.)
"""
import numpy as np
import pytest

from synthetic import Dipole, cube_tet_mesh, workload
from synthetic.workloads import eps_r

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def setup():
    w = workload("cube24_n3_grad")
    v, e = cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed)
    return w, v, e, eps_r(w)


SOURCE = [Dipole(x=(0.02, -0.01, 0.015), dir=(0.0, 0.0, 1.0), t0=0.15, width=0.06)]
PROBES = [(0.12 * sx, 0.13 * sy, 0.14 * sz) for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]


def solver(w, v, e, eps, prec):
    from paper_2006_02551_gb300 import Solver
    s = Solver(w.N, prec)
    s.set_mesh(v, e)
    s.set_materials(eps)
    s.set_pml(w.pml)
    s.set_sources(SOURCE)
    s.set_probes(PROBES)
    s.set_state(None, 0.0)
    return s


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def test_fp32_adjoint_matches_fp64_at_full_size(setup):
    w, v, e, eps = setup
    nst = 250
    out = {}
    for prec in ("fp64", "fp32"):
        s = solver(w, v, e, eps, prec)
        dt = s.stable_dt(1.0)
        out[prec] = s.adjoint(nst, dt, ckpt_every=45)
        s.close()
    J64, ge64, gs64, gp64 = out["fp64"]
    J32, ge32, gs32, gp32 = out["fp32"]
    errs = (abs(J32[0] - J64[0]) / J64[0], rel(ge32, ge64), rel(gs32, gs64), rel(gp32, gp64))
    print(f"J = {J64[0]:.4e}; FP32 vs FP64 adjoint (J, eps, sigma_max, p_sigma):",
          ["%.2e" % x for x in errs])
    assert max(errs) < 1e-5, errs


def test_fp64_adjoint_matches_central_differences_at_full_size(setup):
    w, v, e, eps = setup
    nst = 250
    s = solver(w, v, e, eps, "fp64")
    dt = s.stable_dt(1.0)
    J, ge, gs, gp = s.adjoint(nst, dt, ckpt_every=45)
    print(f"J = {J[0]:.6e}")

    def Jf(x):
        s.set_materials(x)
        s.set_pml(w.pml)
        s.set_sources(SOURCE)
        s.set_probes(PROBES)
        s.set_state(None, 0.0)
        s.run_steps(nst, dt)
        return s.objective()[0]

    rng = np.random.default_rng(12)
    h = 1e-4
    for _ in range(3):
        d = rng.normal(size=eps.size)
        fd = (Jf(eps + h * d) - Jf(eps - h * d)) / (2 * h)
        print(f"directional derivative: adjoint {ge[0] @ d:.10e}  central difference {fd:.10e}")
        assert abs(fd - ge[0] @ d) < 1e-6 * abs(fd)
    s.close()

