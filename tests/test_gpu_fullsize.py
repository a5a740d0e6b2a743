"""GPU checks at the full workload sizes, in the launch configuration the
benchmark uses.

* One Runge-Kutta stage of the 40^3 x 6 = 384,000-tet N=4 workload from a
  seeded random state, FP32 and TF32, against the FP64 oracle evaluated on the
  whole mesh (every output compared).
* Batched excitations on the 30^3 x 6 = 162,000-tet N=3 mesh: each excitation
  of a batched run equals the run of that excitation alone, bit for bit
  (the batch only selects which state block a tile reads and writes).
"""
import numpy as np
import pytest

from oracle import lserk
from synthetic import Dipole, workload
from tests.parity_util import increment_err, pml_mask, to_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def big_stage():
    from oracle.solver import Simulation
    from synthetic import cube_tet_mesh
    w = workload("cube40_n4")
    v, e = cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed)
    sim = Simulation(w.N, v, e, profile=w.pml, sources=w.sources)
    mask = pml_mask(v, e, w.pml)
    rng = np.random.default_rng(77)
    st = {f: rng.normal(size=(3, sim.K, sim.Np)).astype(np.float32).astype(np.float64)
          for f in ("E", "H", "PE", "PH")}
    for f in ("PE", "PH"):
        st[f][:, ~mask] = 0.0
    q0 = to_lib([st])
    dt, t, stage = 0.004, 0.9, 2
    rhs = sim.rhs(st, t + lserk.RK_C[stage] * dt)
    ref = {f: st[f] + lserk.RK_B[stage] * dt * rhs[f] for f in st}
    return w, v, e, mask, q0, ref, (dt, t, stage)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("tf32", 1e-2)])
def test_full_size_one_stage(big_stage, prec, tol):
    from paper_2006_02551_gb300 import Solver
    w, v, e, mask, q0, ref, (dt, t, stage) = big_stage
    s = Solver(w.N, prec)
    s.set_mesh(v, e)
    s.set_pml(w.pml)
    s.set_sources(list(w.sources))
    s.set_state(q0, 0.0)
    s.rk_stage(stage, t, dt)
    q, _ = s.get_state()
    s.close()
    # error of the stage increment (the input is FP32-exact on both sides)
    err = increment_err(q, [ref], q0, mask)
    print(f"{prec} full-size stage error {err:.3e}")
    assert err < tol, err


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_batched_excitations_equal_single_runs(prec):
    from paper_2006_02551_gb300 import Solver
    from synthetic import cube_tet_mesh
    w = workload("cube30_n3_batch64")
    v, e = cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed)
    src = list(w.sources[:4])
    nb = len(src)

    def run(sources, n_batch):
        s = Solver(w.N, prec, n_batch=n_batch)
        s.set_mesh(v, e)
        s.set_pml(w.pml)
        s.set_sources(sources)
        s.set_probes(list(w.probes))
        s.set_state(None, 0.0)
        dt = s.stable_dt(1.0)
        rec = s.run_steps(3, dt)
        q, _ = s.get_state()
        J = s.objective()
        s.close()
        return q, rec, J

    qb, recb, Jb = run(src, nb)
    for b in range(nb):
        d = src[b]
        single = Dipole(x=d.x, dir=d.dir, t0=d.t0, width=d.width, amplitude=d.amplitude, batch=0)
        q1, rec1, J1 = run([single], 1)
        assert np.array_equal(qb[b], q1[0])
        assert np.array_equal(recb[..., b], rec1[..., 0])
        assert Jb[b] == J1[0]
