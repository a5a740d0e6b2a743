"""Pins of the oracle's reference element against closed forms.

Each check is independent of the code path it tests: simplex monomial
integrals in closed form, exact derivatives of monomials, integration by
parts on the reference tetrahedron, and the paper's own node counts.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle.refelem import RefElement, stroud_rule, ref_element

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def simplex_bary_integral(exps, volume):
    """int over a d-simplex of prod lambda_i^{e_i} = d! V prod e_i! / (d + sum e)!"""
    d = len(exps) - 1
    num = math.factorial(d) * volume
    for e in exps:
        num *= math.factorial(e)
    return num / math.factorial(d + sum(exps))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_stroud_rule_exact_to_degree_2n_minus_1(n):
    r, s, t, w = stroud_rule(n)
    assert np.all(w > 0)
    l1, l2, l3 = (1 + r) / 2, (1 + s) / 2, (1 + t) / 2
    l0 = 1 - l1 - l2 - l3
    deg = 2 * n - 1
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                for d in range(deg + 1 - a - b - c):
                    q = np.sum(w * l0 ** d * l1 ** a * l2 ** b * l3 ** c)
                    ex = simplex_bary_integral((d, a, b, c), 4.0 / 3.0)
                    assert abs(q - ex) < 1e-14 * max(1.0, abs(ex)) + 1e-16


def test_node_counts_match_paper():
    # Section III: p in {1..5} gives N_p in {4, 10, 20, 35, 56}
    with open(os.path.join(GOLDEN, "paper_table1.json")) as f:
        g = json.load(f)
    for row in g["rows"]:
        assert ref_element(row["p"]).Np == row["N_p"]


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_basis_orthonormal_and_mass(N):
    re = RefElement(N)
    # orthonormality of phi under an exact rule (degree 2N+1 >= 2N)
    VI = re.Vq @ re.V
    G = VI.T @ np.diag(re.wq) @ VI
    assert np.abs(G - np.eye(re.Np)).max() < 1e-12
    # M = (V V^T)^{-1} equals the Lagrange mass matrix by quadrature
    Mq = re.Vq.T @ np.diag(re.wq) @ re.Vq
    assert np.abs(Mq - re.M).max() < 1e-13
    assert abs(re.M.sum() - 4.0 / 3.0) < 1e-13
    assert np.all(np.linalg.eigvalsh(re.M) > 0)
    # Lagrange property at the nodes
    L = re.lagrange_at(re.r, re.s, re.t)
    assert np.abs(L - np.eye(re.Np)).max() < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_differentiation_exact_on_monomials(N):
    re = RefElement(N)
    r, s, t = re.r, re.s, re.t
    for a in range(N + 1):
        for b in range(N + 1 - a):
            for c in range(N + 1 - a - b):
                f = r ** a * s ** b * t ** c
                fr = a * r ** max(a - 1, 0) * s ** b * t ** c
                fs = b * r ** a * s ** max(b - 1, 0) * t ** c
                ft = c * r ** a * s ** b * t ** max(c - 1, 0)
                assert np.abs(re.Dr @ f - fr).max() < 1e-12
                assert np.abs(re.Ds @ f - fs).max() < 1e-12
                assert np.abs(re.Dt @ f - ft).max() < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_face_mass_matches_triangle_closed_form(N):
    """u^T E_f v = int_face u v for face-restricted barycentric monomials,
    face parametrised with reference area 2 (eq. 17)."""
    re = RefElement(N)
    r, s, t = re.r, re.s, re.t
    bary = [-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2]
    face_verts = [(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)]
    Nfp = re.Nfp
    rng = np.random.default_rng(1)
    for f in range(4):
        fm = re.Fmask[f]
        Ef = re.Emat[:, f * Nfp:(f + 1) * Nfp]
        assert np.abs(np.delete(Ef, fm, axis=0)).max() == 0.0
        Mf = Ef[fm]
        lv = [bary[v][fm] for v in face_verts[f]]
        for _ in range(12):
            e1 = rng.multinomial(rng.integers(0, N + 1), [1 / 3] * 3)
            e2 = rng.multinomial(rng.integers(0, N + 1), [1 / 3] * 3)
            u = lv[0] ** e1[0] * lv[1] ** e1[1] * lv[2] ** e1[2]
            v = lv[0] ** e2[0] * lv[1] ** e2[1] * lv[2] ** e2[2]
            ex = simplex_bary_integral(tuple(e1 + e2), 2.0)
            assert abs(u @ Mf @ v - ex) < 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_integration_by_parts(N):
    """M Dr + (M Dr)^T = oint n_r l_i l_j: face 3 (n_r sJ = 1) minus face 4."""
    re = RefElement(N)
    Nfp = re.Nfp
    Ef = [re.Emat[:, f * Nfp:(f + 1) * Nfp][:, :] for f in range(4)]
    full = []
    for f in range(4):
        A = np.zeros((re.Np, re.Np))
        A[:, re.Fmask[f]] = Ef[f]
        full.append(A)
    nr = [0, 0, 1, -1]
    ns = [0, -1, 1, 0]
    nt = [-1, 0, 1, 0]
    for D, nn in ((re.Dr, nr), (re.Ds, ns), (re.Dt, nt)):
        S = re.M @ D
        rhs = sum(nn[f] * full[f] for f in range(4))
        assert np.abs(S + S.T - rhs).max() < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_projection_of_interpolation_is_identity(N):
    # P_q V_q = M^{-1} V_q^T W V_q = I for a rule exact to degree 2N (eq. 21)
    re = RefElement(N)
    assert np.abs(re.Pq @ re.Vq - np.eye(re.Np)).max() < 5e-13
    assert re.Nq == (N + 1) ** 3
