"""PML reflection against an extended-domain reference (the paper's way of
measuring it, Section III): a sigma_max scan for the smoothly varying
coefficients sampled at the quadrature nodes (the weight-adjusted scheme)
and for element-constant coefficients (the profile at each centroid).

Set-up (synthetic stand-in for the paper's experiment): a z-dipole near the
centre of [-1, 1]^3 on the structured Kuhn lattice with h = 1/8 (N = 3),
PML shell u0 = 0.75, L = 0.25 (two element layers) with the cubic profile,
PEC behind it; probes 0.5-0.6 from the source.  Reference: the same lattice
extended to [-3, 3]^3 without PML, whose boundary echo reaches the probes only
after the recorded window (t <= 3.5).  The interior discretisation of both
runs is identical (same elements, N and time step), so the difference of the
probe signals is the boundary's reflection.  Error = max over probes, steps
and components of |E - E_ref| / max |E_ref|.

Checked: the weight-adjusted scan has its minimum at an interior sigma_max
(too weak a layer lets the PEC echo through, too strong a one reflects at
its discretised gradient), and its best value is below the element-constant
variant's best value."""
import numpy as np
import pytest

from synthetic import Dipole, PmlProfile, cube_tet_mesh

pytestmark = pytest.mark.gpu

SIGMAS = (2.5, 5.0, 10.0, 20.0, 40.0, 80.0, 160.0, 320.0)
SOURCE = Dipole(x=(0.0313, 0.0217, 0.0411), dir=(0.0, 0.0, 1.0), t0=1.0, width=0.25)
PROBES = [(0.55, 0.02, 0.03), (0.03, 0.56, -0.02), (-0.02, 0.04, 0.57),
          (0.33, 0.31, 0.32), (-0.41, -0.38, 0.05)]
T_END = 3.5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def run(v, e, prof, scheme, dt, nsteps):
    from paper_2006_02551_gb300 import Solver
    s = Solver(3, "fp32")
    s.set_mesh(v, e)
    if prof is not None:
        s.set_pml(prof, scheme)
    s.set_sources([SOURCE])
    s.set_probes(PROBES)
    s.set_state(None, 0.0)
    rec = s.run_steps(nsteps, dt)
    dtl = s.stable_dt(1.0)
    s.close()
    return rec[:, :, :3, 0], dtl


def test_reflection_scan():
    from paper_2006_02551_gb300 import Solver
    vs, es = cube_tet_mesh(16, 0.0, 0)
    vb, eb = cube_tet_mesh(48, 0.0, 0)
    vb = vb * 3.0
    probe = Solver(3, "fp32")
    probe.set_mesh(vs, es)
    dt = 0.9 * probe.stable_dt(1.0)
    probe.close()
    nsteps = int(np.ceil(T_END / dt))
    ref, dtb = run(vb, eb, None, "waa", dt, nsteps)
    assert dt <= dtb   # same lattice spacing: the reference is stable at dt
    scale = np.abs(ref).max()
    err = {}
    for scheme in ("waa", "ec"):
        for sm in SIGMAS:
            prof = PmlProfile(u0=0.75, L=0.25, sigma_max=sm, p_sigma=3.0)
            rec, _ = run(vs, es, prof, scheme, dt, nsteps)
            err[scheme, sm] = float(np.abs(rec - ref).max() / scale)
    print("\nsigma_max " + " ".join(f"{sm:>9g}" for sm in SIGMAS))
    for scheme in ("waa", "ec"):
        print(f"{scheme:9s} " + " ".join(f"{err[scheme, sm]:9.2e}" for sm in SIGMAS))
    waa = [err["waa", sm] for sm in SIGMAS]
    ec = [err["ec", sm] for sm in SIGMAS]
    k = int(np.argmin(waa))
    assert 0 < k < len(SIGMAS) - 1, waa          # interior minimum
    assert min(waa) < min(ec), (waa, ec)
