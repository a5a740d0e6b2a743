"""Normal-incidence plane-wave box (the geometry type of the paper's first
experiment, Section III): periodic in x and y, PML at both ends in z.

* Parity: the library on a jittered periodic box with the z-PML against the
  FP64 oracle (one stage from a random state; 40 steps of a plane-wave pulse
  through run_steps), FP64 1e-12 and FP32 1e-5.
* Plane-wave order: on a fully periodic box E_x = H_y = sin(2 pi (z - t)/2)
  is exact; the GPU FP64 error decays at rate >= N + 0.8.
* Reflection at normal incidence: a Gaussian pulse E_x = H_y = exp(-(z/w)^2)
  travels in +z into the PML (u0 = 1.5, L = 0.5, two element layers, cubic
  profile) on a jittered (paved, not layer-aligned) lattice; the probe signal
  at z = 1 is compared with the extended box |z| <= 6 without PML (its PEC
  echo arrives after the window).  The smoothly varying profile's error has
  an interior minimum over the sigma_max scan and its best value is below the
  element-constant one's.
"""
import numpy as np
import pytest

from oracle import lserk
from oracle.solver import Simulation
from synthetic import PmlProfile, box_tet_mesh
from tests.parity_util import (increment_err, pml_mask, random_states, rel_err,
                                 round_states, to_lib)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
PMLZ = PmlProfile(u0=0.6, L=0.4, sigma_max=15.0, p_sigma=3.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def solver(N, prec, v, e, c, prof=None, scheme="waa"):
    from paper_2006_02551_gb300 import Solver
    s = Solver(N, prec)
    s.set_mesh(v, e, c)
    if prof is not None:
        s.set_pml(prof, scheme)
    return s


def pulse_state(sim, w=0.2, z0=0.0):
    st = sim.zero_state()
    z = sim.geom.x[2]
    g = np.exp(-((z - z0) / w) ** 2)
    st[0]["E"][0] = g
    st[0]["H"][1] = g
    return st


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_periodic_box_parity(prec):
    N = 3
    v, e, c = box_tet_mesh((3, 3, 6), (-0.5, -0.5, -1.0), (0.5, 0.5, 1.0), 0.15, 5,
                           (True, True, False))
    sim = Simulation(N, v, e, profile=PMLZ, vcanon=c)
    mask = pml_mask(v, e, PMLZ)
    assert mask.any() and not mask.all()
    # one stage from a random state
    s = solver(N, prec, v, e, c, PMLZ)
    st = round_states(random_states(sim.K, sim.Np, 1, 9, mask), prec)
    q0 = to_lib(st)
    s.set_state(q0, 0.0)
    dt, t, stage = 0.01, 0.3, 3
    s.rk_stage(stage, t, dt)
    q, _ = s.get_state()
    rhs = sim.rhs(st[0], t + lserk.RK_C[stage] * dt, 0)
    for f in st[0]:
        st[0][f] = st[0][f] + lserk.RK_B[stage] * dt * rhs[f]
    assert increment_err(q, st, q0, mask) < TOL[prec]
    # 40 steps of a plane-wave pulse
    st = pulse_state(sim)
    s.set_state(to_lib(st), 0.0)
    dt = sim.stable_dt(1.0)
    s.run_steps(40, dt, record=False)
    q, _ = s.get_state()
    st, _, _, _ = sim.run(st, 40, dt, record=False)
    err = rel_err(q, st, mask)
    s.close()
    assert err < TOL[prec], err


def test_plane_wave_order_fully_periodic():
    N, T, k = 2, 0.25, np.pi
    errs = []
    for nz in (4, 8):
        v, e, c = box_tet_mesh((3, 3, nz), (-0.5, -0.5, -1.0), (0.5, 0.5, 1.0), 0.1, 11,
                               (True, True, True))
        sim = Simulation(N, v, e, vcanon=c)   # node coordinates and mass matrix only
        x = sim.geom.x
        st = sim.zero_state()
        st[0]["E"][0] = np.sin(k * x[2])
        st[0]["H"][1] = np.sin(k * x[2])
        s = solver(N, "fp64", v, e, c)
        s.set_state(to_lib(st), 0.0)
        nst = int(np.ceil(T / s.stable_dt(0.5)))
        s.run_steps(nst, T / nst, record=False)
        q, _ = s.get_state()
        s.close()
        ex = np.sin(k * (x[2] - T))
        M, J = sim.ref.M, sim.geom.J
        d = [q[0][:, 0, :] - ex, q[0][:, 4, :] - ex]   # E_x, H_y  [K][Np]
        err2 = sum(np.sum(J * np.einsum("ki,ij,kj->k", dd, M, dd)) for dd in d)
        for comp in (1, 2, 3, 5):
            dd = q[0][:, comp, :]
            err2 += np.sum(J * np.einsum("ki,ij,kj->k", dd, M, dd))
        errs.append(np.sqrt(err2))
    slope = np.log2(errs[0] / errs[1])
    assert slope >= N + 0.8, (errs, slope)


SIGMAS = (2.0, 5.0, 10.0, 20.0, 40.0, 80.0, 160.0, 320.0)


def test_normal_incidence_reflection_scan():
    """Jittered (paved) lattice, h = 1/4, N = 3, FP64.  The computational box
    is the middle third (|z| <= 2) of the extended box |z| <= 6, cut out hex
    layer by hex layer, so both runs share their interior elements exactly."""
    N = 3
    vb, eb, cb = box_tet_mesh((4, 4, 48), (-0.5, -0.5, -6.0), (0.5, 0.5, 6.0), 0.2, 21,
                              (True, True, False))
    per_layer = 6 * 4 * 4
    es = eb[16 * per_layer:32 * per_layer]          # hex layers 16..31: |z| <= 2
    probe = [(0.1, -0.05, 1.0)]
    sim_s = Simulation(N, vb, es, vcanon=cb)
    sim_b = Simulation(N, vb, eb, vcanon=cb)
    q0s, q0b = to_lib(pulse_state(sim_s)), to_lib(pulse_state(sim_b))
    s = solver(N, "fp64", vb, eb, cb)
    dt = 0.9 * s.stable_dt(1.0)
    s.close()
    nsteps = int(np.ceil(3.5 / dt))

    def run(e, q0, prof, scheme):
        s = solver(N, "fp64", vb, e, cb, prof, scheme)
        s.set_probes(probe)
        s.set_state(q0, 0.0)
        rec = s.run_steps(nsteps, dt)
        s.close()
        return rec[:, 0, 0, 0]                                   # E_x at the probe

    ref = run(eb, q0b, None, "waa")
    scale = np.abs(ref).max()
    err = {}
    for scheme in ("waa", "ec"):
        for sm in SIGMAS:
            prof = PmlProfile(u0=1.5, L=0.5, sigma_max=sm, p_sigma=3.0)
            err[scheme, sm] = float(np.abs(run(es, q0s, prof, scheme) - ref).max() / scale)
    print("\nsigma_max " + " ".join(f"{sm:>9g}" for sm in SIGMAS))
    for scheme in ("waa", "ec"):
        print(f"{scheme:9s} " + " ".join(f"{err[scheme, sm]:9.2e}" for sm in SIGMAS))
    waa = [err["waa", sm] for sm in SIGMAS]
    ec = [err["ec", sm] for sm in SIGMAS]
    k = int(np.argmin(waa))
    assert 0 < k < len(SIGMAS) - 1, waa
    assert min(waa) < min(ec), (waa, ec)
