"""Oracle pins of the periodic connectivity used by the plane-wave box.

* On a fully periodic jittered box no face is a boundary face and the trace
  map is an involution (every exterior trace's exterior trace is the interior
  trace), with the face nodes matched up to the period translation.
* A plane wave E_x = H_y = sin(2 pi (z - t) / L_z) (eps = mu = 1) is an exact
  solution of Maxwell's equations on a box periodic in all three directions;
  the L2 error of the discrete solution after a fixed time decays at the
  optimal rate (observed slope >= N + 0.8 over two refinements), which fails
  if a periodic face pair is matched with the wrong node order or shift.
"""
import numpy as np
import pytest

from oracle.solver import Simulation
from synthetic import box_tet_mesh


def test_fully_periodic_box_has_no_boundary_and_involutive_traces():
    v, e, c = box_tet_mesh((3, 3, 3), (-0.5, -0.5, -1.0), (0.5, 0.5, 1.0), 0.15, 7,
                           (True, True, True))
    sim = Simulation(3, v, e, vcanon=c)
    g = sim.geom
    assert not g.boundary.any()
    vM, vP = g.vmapM.reshape(-1), g.vmapP.reshape(-1)
    inv = np.empty(vM.size, np.int64)
    inv[np.argsort(vM)] = np.arange(vM.size)  # position of each interior trace node
    # vmapM lists each face node once per face it lies on: compare through
    # (element, face, node) slots instead of node ids
    K, Nfp = sim.K, sim.ref.Nfp
    slot_of = {}
    for k in range(K):
        for f in range(4):
            for m in range(Nfp):
                slot_of[(k, f, int(vP.reshape(K, 4, Nfp)[k, f, m]))] = m
    EToE, EToF = g.EToE, g.EToF
    X = g.x.reshape(3, -1)
    fv = np.array([[0, 1, 2], [0, 1, 3], [1, 2, 3], [0, 2, 3]])
    for k in range(0, K, 7):
        for f in range(4):
            k2, f2 = EToE[k, f], EToF[k, f]
            assert EToE[k2, f2] == k and EToF[k2, f2] == f
            shift = g.verts[k, fv[f]].mean(axis=0) - g.verts[k2, fv[f2]].mean(axis=0)
            idM = g.vmapM.reshape(K, 4, Nfp)[k, f]
            idP = g.vmapP.reshape(K, 4, Nfp)[k, f]
            assert np.allclose(X[:, idM] - shift[:, None], X[:, idP], atol=1e-12)
            # the shift is a period vector
            assert np.allclose(np.abs(shift), [0, 0, 0], atol=1e-12) or \
                np.isclose(np.abs(shift).max(), 1.0) or np.isclose(np.abs(shift).max(), 2.0)


def _plane_wave_error(N, nz, T=0.25):
    Lz = 2.0
    v, e, c = box_tet_mesh((3, 3, nz), (-0.5, -0.5, -1.0), (0.5, 0.5, 1.0), 0.1, 11,
                           (True, True, True))
    sim = Simulation(N, v, e, vcanon=c)
    x = sim.geom.x
    k = 2.0 * np.pi / Lz
    st = sim.zero_state()
    st[0]["E"][0] = np.sin(k * x[2])
    st[0]["H"][1] = np.sin(k * x[2])
    dt0 = sim.stable_dt(0.5)
    nst = int(np.ceil(T / dt0))
    dt = T / nst
    st, t, _, _ = sim.run(st, nst, dt, record=False)
    exact = np.sin(k * (x[2] - T))
    M, J = sim.ref.M, sim.geom.J
    err2 = 0.0
    for (fld, comp) in (("E", 0), ("H", 1)):
        d = st[0][fld][comp] - exact
        err2 += np.sum(J * np.einsum("ki,ij,kj->k", d, M, d))
    for (fld, comps) in (("E", (1, 2)), ("H", (0, 2))):
        for cc in comps:
            d = st[0][fld][cc]
            err2 += np.sum(J * np.einsum("ki,ij,kj->k", d, M, d))
    return np.sqrt(err2)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_plane_wave_convergence_on_periodic_box(N):
    nzs = (4, 8, 16) if N == 1 else (4, 8)
    errs = [_plane_wave_error(N, nz) for nz in nzs]
    slopes = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(slopes) >= N + 0.8, (errs, slopes)
