"""Pins of the oracle's PML coefficients (eqs. 4, 9) and element geometry."""
import numpy as np
import pytest

from oracle.geometry import Geometry
from oracle.pml import cpml_tensors, stretch_profiles
from oracle.refelem import ref_element
from synthetic import PmlProfile, cube_tet_mesh


def test_cpml_tensors_reproduce_stretched_coordinates():
    """Frequency domain: the E-update of eqs. 6, 8 is
    eps E [jw a + b + c/(jw kappa_u + sigma_u/eps0)] = curl H (P = E/(jw kappa_u + sigma_u)),
    and must equal the stretched-coordinate form jw eps (s_v s_w / s_u) E of
    eqs. 1-4.  Complex arithmetic on both sides, random coefficients."""
    rng = np.random.default_rng(7)
    for eps0 in (1.0, 8.854e-12):
        sig = rng.uniform(0, 50, (3, 200)) * eps0
        kap = rng.uniform(1, 3, (3, 200))
        w = rng.uniform(0.1, 30, 200)
        a, b, c, d, k = cpml_tensors(sig, kap, eps0)
        jw = 1j * w
        s = kap + sig / (jw * eps0)
        for u in range(3):
            v, ww = (u + 1) % 3, (u + 2) % 3
            lhs = jw * a[u] + b[u] + c[u] / (jw * kap[u] + sig[u] / eps0)
            rhs = jw * s[v] * s[ww] / s[u]
            assert np.allclose(lhs, rhs, rtol=1e-12, atol=0)
            # the P-update: jw P = E/kappa_u - d P  <=> P = E / (jw kappa_u + sigma_u/eps0)
            assert np.allclose(1.0 / (jw + d[u]) / k[u],
                               1.0 / (jw * kap[u] + sig[u] / eps0), rtol=1e-12)


def test_tensors_without_pml_are_trivial():
    sig = np.zeros((3, 5))
    kap = np.ones((3, 5))
    a, b, c, d, k = cpml_tensors(sig, kap)
    assert np.all(a == 1) and np.all(b == 0) and np.all(c == 0) and np.all(d == 0)


def test_profile_shape():
    p = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0, kappa_max=2.0)
    x = np.array([[0.0, 0.75, -0.75, 0.875, -1.0, 1.0]] * 3)
    sig, kap = stretch_profiles(p, x)
    assert np.allclose(sig[0], [0, 0, 0, 20 * 0.5 ** 3, 20, 20])
    assert np.allclose(kap[0], [1, 1, 1, 1 + 0.5 ** 3, 2, 2])


@pytest.mark.parametrize("N", [1, 3])
def test_geometry_closed_forms(N):
    ref = ref_element(N)
    v, e = cube_tet_mesh(3, 0.15, 11)
    g = Geometry(ref, v, e)
    # volume of the cube: J_k times reference volume 4/3
    assert abs(g.J.sum() * 4 / 3 - 8.0) < 1e-12
    # boundary area: sJ is physical area / 2
    assert abs((2 * g.sJ[g.boundary]).sum() - 24.0) < 1e-12
    # closed surface per element: sum_f area_f n_f = 0
    for comp in (g.nx, g.ny, g.nz):
        assert np.abs((g.sJ * comp).sum(axis=1)).max() < 1e-13
    # neighbouring faces: opposite normals, same area, coincident nodes,
    # exterior of the exterior is the interior
    k, f = np.nonzero(~g.boundary)
    k2, f2 = g.EToE[k, f], g.EToF[k, f]
    assert np.allclose(g.nx[k, f], -g.nx[k2, f2], atol=1e-13)
    assert np.allclose(g.sJ[k, f], g.sJ[k2, f2], rtol=1e-12)
    X = g.x.reshape(3, -1)
    assert np.abs(X[:, g.vmapM] - X[:, g.vmapP]).max() < 1e-13
    Nfp = ref.Nfp
    for kk, ff in list(zip(k, f))[:300]:
        k2_, f2_ = g.EToE[kk, ff], g.EToF[kk, ff]
        mine = g.vmapM[kk, ff * Nfp:(ff + 1) * Nfp]
        ext = g.vmapP[kk, ff * Nfp:(ff + 1) * Nfp]
        back_m = g.vmapM[k2_, f2_ * Nfp:(f2_ + 1) * Nfp]
        back_p = g.vmapP[k2_, f2_ * Nfp:(f2_ + 1) * Nfp]
        for a in range(Nfp):
            slot = int(np.nonzero(back_m == ext[a])[0][0])
            assert back_p[slot] == mine[a]
    # nodes on boundary faces lie on the cube surface
    b = g.vmapM[np.repeat(g.boundary, ref.Nfp, axis=1)]
    assert np.allclose(np.abs(X[:, b]).max(axis=0), 1.0, atol=1e-13)


def test_metric_terms_invert_map():
    ref = ref_element(2)
    v, e = cube_tet_mesh(2, 0.2, 3)
    g = Geometry(ref, v, e)
    # x = map(r): finite difference of the map against (rx ...)^{-1}
    h = 1e-6
    x0 = g.map_points([0.1], [-0.3], [-0.2])
    xr = (g.map_points([0.1 + h], [-0.3], [-0.2]) - x0) / h
    for k in range(g.K):
        J = np.array([[g.rx[k], g.ry[k], g.rz[k]],
                      [g.sx[k], g.sy[k], g.sz[k]],
                      [g.tx[k], g.ty[k], g.tz[k]]])
        col = xr[:, k, 0]
        assert np.allclose(J @ col, [1, 0, 0], atol=1e-8)
