"""The allocation-free stepping entry point (wadg_run_steps_noalloc), for
callers that cannot allocate device memory while they step, must give the
same probe records, state and objective as wadg_run_steps, on two calls in a
row (the second call finds the scratch array holding the first call's
contents).  Collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from synthetic import workload

pytestmark = pytest.mark.gpu

TOL = 1e-12   # FP64 path (the probe objective sums in a different order)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def make(w):
    from paper_2006_02551_gb300 import Solver
    from synthetic import cube_tet_mesh
    v, e = cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed)
    s = Solver(w.N, "fp64")
    s.set_mesh(v, e)
    s.set_pml(w.pml)
    s.set_sources(list(w.sources))
    s.set_probes(list(w.probes))
    s.set_state(None, 0.0)
    return s


def test_noalloc_steps_match_run_steps_twice():
    w = workload("cube4_n3")
    a, b = make(w), make(w)
    dt = a.stable_dt(1.0)
    for n in (23, 17):   # two calls in a row on each path
        ra = a.run_steps(n, dt)
        rb = b.run_steps_noalloc(n, dt)
        assert np.abs(ra - rb).max() <= TOL * np.abs(ra).max()
        qa, ta = a.get_state()
        qb, tb = b.get_state()
        assert ta == tb
        assert np.abs(qa - qb).max() <= TOL * np.abs(qa).max()
        Ja, Jb = a.objective()[0], b.objective()[0]
        assert abs(Ja - Jb) <= TOL * abs(Ja)
    a.close()
    b.close()


def test_noalloc_rejects_oversized_step_records():
    from paper_2006_02551_gb300 import Solver, WadgError, wadg
    from synthetic import cube_tet_mesh
    v, e = cube_tet_mesh(1, 0.0, 0)
    # 3 probes x 6 values x 120000 excitations x 8 bytes > 16 MiB
    s = Solver(1, "fp32", n_batch=120000)
    s.set_mesh(v, e)
    s.set_probes([(0.1, 0.1, 0.1), (-0.2, 0.3, 0.1), (0.5, -0.5, 0.2)])
    s.set_state(None, 0.0)
    with pytest.raises(WadgError) as err:
        s.run_steps_noalloc(1, 0.01, record=False)
    assert err.value.status == wadg.WADG_EINVAL
    s.close()
