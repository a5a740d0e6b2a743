"""Pins of the oracle's semi-discrete Maxwell/PML operator.

* polynomial preservation: fields of degree <= N with a known curl give the
  exact right-hand side on elements away from the boundary and the PML;
* energy: with the central flux the semi-discrete energy is conserved, with
  the upwind flux it does not grow (PEC box, no PML);
* the weight-adjusted approximation is exact for element-constant
  coefficients (eq. 18), and with kappa = 1 the WAA scheme equals the stored
  scheme built on the same quadrature (eqs. 22-25 vs eqs. 10-13);
* the WAA error stays below the discretisation error and falls with N;
* point-source projection and probe interpolation reproduce polynomials;
* a PEC cavity mode converges at order N+1;
* the PML absorbs: late-time energy falls by orders of magnitude.
"""
import numpy as np
import pytest

from oracle.solver import Simulation
from synthetic import Dipole, PmlProfile, cube_tet_mesh

PML = PmlProfile(u0=0.5, L=0.5, sigma_max=20.0, p_sigma=3.0, kappa_max=1.0)
PMLK = PmlProfile(u0=0.5, L=0.5, sigma_max=20.0, p_sigma=3.0, kappa_max=2.0)


def interior_elements(sim, margin_u0=None):
    g = sim.geom
    ok = ~np.any(g.boundary, axis=1)
    if margin_u0 is not None:
        ok &= np.all(np.abs(g.verts).max(axis=1) <= margin_u0, axis=1)
    return ok


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_gradient_fields_have_zero_curl_rhs(N):
    v, e = cube_tet_mesh(4, 0.15, 2)
    sim = Simulation(N, v, e)
    x, y, z = sim.geom.x
    # E = grad(phi), phi = x^a y^b z^c of degree N+1 -> E of degree N
    rng = np.random.default_rng(N)
    a, b = rng.integers(0, N + 1), 0
    b = rng.integers(0, N + 1 - a)
    c = N + 1 - a - b
    E = np.stack([a * x ** max(a - 1, 0) * y ** b * z ** c,
                  b * x ** a * y ** max(b - 1, 0) * z ** c,
                  c * x ** a * y ** b * z ** max(c - 1, 0)])
    q = {"E": E, "H": np.zeros_like(E), "PE": np.zeros_like(E),
         "PH": np.zeros_like(E)}
    r = sim.rhs(q, 0.0)
    m = interior_elements(sim)
    scale = np.abs(E).max()
    assert np.abs(r["H"][:, m]).max() < 1e-11 * scale
    assert np.abs(r["E"][:, m]).max() < 1e-11 * scale


@pytest.mark.parametrize("N", [1, 3])
def test_rotation_field_has_known_curl(N):
    """E = (-y, x, 0) has curl (0, 0, 2): dH/dt = -(0, 0, 2), dE/dt = 0."""
    v, e = cube_tet_mesh(3, 0.1, 5)
    mu = np.full(6 * 27, 2.0)
    sim = Simulation(N, v, e, mu=mu)
    x, y, z = sim.geom.x
    E = np.stack([-y, x, 0 * z])
    q = {"E": E, "H": 0 * E, "PE": 0 * E, "PH": 0 * E}
    r = sim.rhs(q, 0.0)
    m = interior_elements(sim)
    assert np.abs(r["H"][0][m]).max() < 1e-12
    assert np.abs(r["H"][1][m]).max() < 1e-12
    assert np.abs(r["H"][2][m] + 2.0 / 2.0).max() < 1e-12
    assert np.abs(r["E"][:, m]).max() < 1e-12


def _random_state(sim, seed):
    rng = np.random.default_rng(seed)
    return {f: rng.normal(size=(3, sim.K, sim.Np)) for f in ("E", "H", "PE", "PH")}


def _energy_rate(sim, q, r):
    M, J = sim.ref.M, sim.geom.J
    eps, mu = sim.disc.eps, sim.disc.mu
    s = 0.0
    for u in range(3):
        s += np.sum(eps * J * np.einsum("ki,ij,kj->k", q["E"][u], M, r["E"][u]))
        s += np.sum(mu * J * np.einsum("ki,ij,kj->k", q["H"][u], M, r["H"][u]))
    return s


@pytest.mark.parametrize("N", [1, 2, 3])
def test_energy_conserved_central_dissipated_upwind(N):
    v, e = cube_tet_mesh(3, 0.15, 9)
    K = 6 * 27
    rng = np.random.default_rng(3)
    sim_c = Simulation(N, v, e, alpha=0.0)
    q = _random_state(sim_c, 1)
    scale = sim_c.energy(q) * sim_c.geom.Fscale.max() * (N + 1) ** 2
    rate_c = _energy_rate(sim_c, q, sim_c.rhs(q, 0.0))
    assert abs(rate_c) < 1e-12 * scale
    # upwind: strictly dissipative for a random state, with varying media
    sim_u = Simulation(N, v, e, eps=rng.uniform(1, 4, K), mu=rng.uniform(1, 2, K))
    for seed in range(3):
        q = _random_state(sim_u, 10 + seed)
        rate_u = _energy_rate(sim_u, q, sim_u.rhs(q, 0.0))
        assert rate_u < -1e-3 * abs(rate_c + 1) or rate_u < 0


def test_upwind_energy_rate_equals_jump_dissipation():
    """For uniform media the upwind energy rate is
    -(1/2) sum_faces oint |n x [E]|^2 + |n x [H]|^2 / 2 (each interior face
    counted from both sides, PEC jumps E+ - E- = -2 E-)."""
    N = 2
    v, e = cube_tet_mesh(2, 0.1, 4)
    sim = Simulation(N, v, e)
    q = _random_state(sim, 5)
    rate = _energy_rate(sim, q, sim.rhs(q, 0.0))
    g, ref, d = sim.geom, sim.ref, sim.disc
    EM, EP = d.traces(q["E"])
    HM, HP = d.traces(q["H"])
    EP = np.where(d.bnd[None], -EM, EP)
    HP = np.where(d.bnd[None], HM, HP)
    n = d.n
    def tang(a):
        return a - n * np.sum(n * a, axis=0)
    jE, jH = tang(EP - EM), tang(HP - HM)
    Nfp = ref.Nfp
    tot = 0.0
    for f in range(4):
        sl = slice(f * Nfp, (f + 1) * Nfp)
        Mf = ref.Emat[ref.Fmask[f], sl]
        w = g.sJ[:, f]
        for c in range(3):
            tot += np.sum(w * np.einsum("ki,ij,kj->k", jE[c][:, sl], Mf, jE[c][:, sl]))
            tot += np.sum(w * np.einsum("ki,ij,kj->k", jH[c][:, sl], Mf, jH[c][:, sl]))
    assert abs(rate - (-0.25 * tot)) < 1e-11 * abs(tot)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_waa_exact_for_element_constant_coefficients(N):
    """M_k (M_k^{1/alpha})^{-1} M_k = alpha M_k for constant alpha (eq. 18):
    with element-constant sigma, kappa the WAA and stored schemes coincide."""
    v, e = cube_tet_mesh(2, 0.1, 6)
    sim = Simulation(N, v, e, profile=PMLK)
    cen = sim.geom.verts.mean(axis=1).T * 1.7                 # push into the PML
    sim.disc.set_profile(PMLK, element_constant_at=cen)
    q = _random_state(sim, 2)
    CE, CH = sim.disc.curl_operators(q["E"], q["H"])
    rw = sim.disc.rhs_waa(q, CE, CH)
    rs = sim.disc.rhs_stored(q, CE, CH)
    for f in rw:
        scale = np.abs(rs[f]).max()
        assert np.abs(rw[f] - rs[f]).max() < 1e-11 * scale, f


@pytest.mark.parametrize("N", [1, 2, 3])
def test_kappa_one_waa_equals_stored_on_same_rule(N):
    """kappa = 1 gives a = 1, so (M^a)^{-1} = M_k^{-1} and eqs. 26-29 equal
    eqs. 10-13 whenever M^b, M^c, M^d are built by the same quadrature."""
    v, e = cube_tet_mesh(2, 0.15, 7)
    sim = Simulation(N, v, e, profile=PML, stored_quad_points=N + 1)
    q = _random_state(sim, 3)
    CE, CH = sim.disc.curl_operators(q["E"], q["H"])
    rw = sim.disc.rhs_waa(q, CE, CH)
    rs = sim.disc.rhs_stored(q, CE, CH)
    for f in rw:
        scale = np.abs(rs[f]).max()
        assert np.abs(rw[f] - rs[f]).max() < 1e-10 * scale, f


@pytest.mark.parametrize("N", [1, 2])
def test_waa_and_stored_schemes_converge_under_refinement(N):
    """Smooth kappa_u = 1 + u^2 (sigma = 0): for a state w of degree N in each
    element, the stored operator (M^a)^{-1} M_k w is the a-weighted projection
    of w/a and the WAA operator P_q a^{-1} V_q w its plain L2 projection; the
    two differ by Pi_a(w/a - Pi(w/a)) = O(h) * O(h) |w|, so the relative
    difference of the right-hand sides falls like h^2 (a wrong sign or
    coefficient in either scheme leaves an O(1) difference)."""
    prof = PmlProfile(u0=0.0, L=1.0, sigma_max=0.0, p_sigma=2.0, kappa_max=2.0)
    errs = []
    for n in (2, 4):
        v, e = cube_tet_mesh(n, 0.0, 0)
        sim = Simulation(N, v, e, profile=prof, stored_quad_points=N + 6)
        x, y, z = sim.geom.x
        F = np.stack([np.sin(1.3 * x + 0.2) * np.cos(y), np.cos(0.7 * z) * y,
                      np.exp(0.3 * x) * np.sin(z + y)])
        q = {"E": F, "H": 0.5 * F[::-1], "PE": 0 * F, "PH": 0 * F}
        CE, CH = sim.disc.curl_operators(q["E"], q["H"])
        rw = sim.disc.rhs_waa(q, CE, CH)
        rs = sim.disc.rhs_stored(q, CE, CH)
        d = {k: rw[k] - rs[k] for k in rw}
        errs.append(np.sqrt(sim.energy(d) / sim.energy(rs)))
    assert errs[0] < 0.1
    assert np.log2(errs[0] / errs[1]) > 1.8, errs


@pytest.mark.parametrize("N", [1, 3])
def test_source_projection_and_probes_reproduce_polynomials(N):
    v, e = cube_tet_mesh(2, 0.1, 1)
    xs = (0.13, -0.21, 0.37)
    sim = Simulation(N, v, e, sources=[Dipole(x=xs)], probes=[xs, (0.5, 0.5, -0.5)])
    _, k, w = sim.sources[0]
    x, y, z = sim.geom.x
    u = (1 + x + 2 * y * z) if N >= 2 else (1 + x - 3 * z)
    uv = (1 + xs[0] + 2 * xs[1] * xs[2]) if N >= 2 else (1 + xs[0] - 3 * xs[2])
    # u^T M_k w = u(x_s): w is the projection of the point delta
    assert abs(u[k] @ (sim.geom.J[k] * sim.ref.M) @ w - uv) < 1e-12
    F = np.stack([u, 2 * u, -u])
    q = {"E": F, "H": 3 * F, "PE": 0 * F, "PH": 0 * F}
    pv = sim.probe_values(q)
    assert np.allclose(pv[0], [uv, 2 * uv, -uv, 3 * uv, 6 * uv, -3 * uv], atol=1e-12)


def _cavity_error(N, n, T=0.5, cfl=0.25):
    v, e = cube_tet_mesh(n, 0.1, 0)
    sim = Simulation(N, v, e)
    x, y, z = sim.geom.x
    kx = ky = np.pi / 2
    w = np.sqrt(kx ** 2 + ky ** 2)

    def exact(t):
        Ez = np.sin(kx * (x + 1)) * np.sin(ky * (y + 1)) * np.cos(w * t)
        Hx = -(ky / w) * np.sin(kx * (x + 1)) * np.cos(ky * (y + 1)) * np.sin(w * t)
        Hy = (kx / w) * np.cos(kx * (x + 1)) * np.sin(ky * (y + 1)) * np.sin(w * t)
        Z = 0 * x
        return np.stack([Z, Z, Ez]), np.stack([Hx, Hy, Z])

    E0, H0 = exact(0.0)
    st = [{"E": E0, "H": H0, "PE": 0 * E0, "PH": 0 * E0}]
    dt0 = sim.stable_dt(cfl)
    nsteps = int(np.ceil(T / dt0))
    dt = T / nsteps
    st, t, _, _ = sim.run(st, nsteps, dt, record=False)
    E1, H1 = exact(T)
    err = {"E": st[0]["E"] - E1, "H": st[0]["H"] - H1, "PE": 0 * E1, "PH": 0 * E1}
    return np.sqrt(2 * sim.energy(err))


@pytest.mark.slow
@pytest.mark.parametrize("N", [1, 2, 3])
def test_cavity_mode_converges_at_order_N_plus_1(N):
    e1 = _cavity_error(N, 2)
    e2 = _cavity_error(N, 4)
    slope = np.log2(e1 / e2)
    assert slope > N + 0.7, (e1, e2, slope)


def test_pml_absorbs_outgoing_pulse():
    """PEC box with and without the PML shell: energy left after the pulse has
    had time to cross the shell twice.  The pulse starts with G(0) = e^-9, so
    no static dipole is left behind."""
    v, e = cube_tet_mesh(4, 0.15, 0)
    src = [Dipole(x=(0.0, 0.0, 0.0), t0=1.5, width=0.25)]
    prof = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0)
    out = []
    for p in (None, prof):
        sim = Simulation(2, v, e, profile=p, sources=src)
        dt = sim.stable_dt(1.0)
        st = sim.zero_state()
        st, t, _, _ = sim.run(st, int(4.5 / dt), dt, record=False)
        out.append(sim.energy(st[0]))
    assert out[1] < 1e-2 * out[0], out
