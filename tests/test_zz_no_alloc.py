"""The allocation-free stepping entry point (wadg_run_steps_noalloc), for
callers that cannot allocate device memory while they step, must give the
same probe records, state and objective as wadg_run_steps, on two calls in a
row (the second call finds the scratch array holding the first call's
contents).  Collected last so that a run stopping at the first failure has
already run every other test.

Both entry points launch the same stage, probe and clock kernels on the same
data (one replays a captured graph, the other launches them directly), so
the results agree to rounding-order level: the bounds below are far above
what a same-kernel comparison can differ by, and far below any real error."""
import numpy as np
import pytest

from synthetic import Dipole, cube_tet_mesh, workload

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6, "tf32": 1e-6, "bf16": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def make(w, precision="fp64", scheme="waa", rule="default"):
    from paper_2006_02551_gb300 import Solver
    from synthetic import compact_rule
    v, e = cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed)
    s = Solver(w.N, precision)
    if rule == "compact":
        s.set_quadrature(compact_rule(w.N))
    s.set_mesh(v, e)
    s.set_pml(w.pml, scheme)
    s.set_sources(list(w.sources))
    s.set_probes(list(w.probes))
    s.set_state(None, 0.0)
    return s


def close_to(a, b, tol):
    return np.abs(a - b).max() <= tol * max(np.abs(a).max(), 1e-300)


@pytest.mark.parametrize("precision,scheme,rule", [
    ("fp64", "waa", "default"), ("fp32", "waa", "default"), ("fp32", "stored", "default"),
    ("fp32", "ec", "default"), ("tf32", "waa", "default"), ("bf16", "waa", "default"),
    ("tf32", "stored", "default"), ("tf32", "waa", "compact"), ("bf16", "waa", "compact")])
def test_noalloc_steps_match_run_steps_twice(precision, scheme, rule):
    w = workload("cube4_n3")
    a, b = make(w, precision, scheme, rule), make(w, precision, scheme, rule)
    dt = a.stable_dt(1.0)
    tol = TOL[precision]
    for n in (23, 17):   # two calls in a row on each path
        ra = a.run_steps(n, dt)
        rb = b.run_steps_noalloc(n, dt)
        assert close_to(ra, rb, tol)
        qa, ta = a.get_state()
        qb, tb = b.get_state()
        assert ta == tb
        assert close_to(qa, qb, tol)
        Ja, Jb = a.objective()[0], b.objective()[0]
        assert abs(Ja - Jb) <= tol * abs(Ja)
    a.close()
    b.close()


def test_noalloc_records_span_several_chunks():
    """Records of one step that fill more than half of the scratch array:
    every step is its own chunk, with the counters set again for each."""
    from paper_2006_02551_gb300 import Solver
    v, e = cube_tet_mesh(2, 0.1, 7)
    nb = 512
    rng = np.random.default_rng(3)
    probes = rng.uniform(-0.9, 0.9, (400, 3))      # 400 x 6 x 512 doubles per step
    srcs = [Dipole(x=tuple(rng.uniform(-0.5, 0.5, 3)), t0=0.3, width=0.15, batch=b)
            for b in range(0, nb, 37)]

    def solver():
        s = Solver(1, "fp32", n_batch=nb)
        s.set_mesh(v, e)
        s.set_sources(srcs)
        s.set_probes(probes)
        s.set_state(None, 0.0)
        return s

    a, b = solver(), solver()
    dt = a.stable_dt(1.0)
    for n in (3, 2):
        ra = a.run_steps(n, dt)
        rb = b.run_steps_noalloc(n, dt)
        assert np.abs(ra).max() > 0
        assert close_to(ra, rb, TOL["fp32"])
        qa, _ = a.get_state()
        qb, _ = b.get_state()
        assert close_to(qa, qb, TOL["fp32"])
    a.close()
    b.close()


def test_noalloc_allocates_nothing():
    """Capped at the bytes it holds, a fresh context with probes cannot run
    wadg_run_steps (its first run allocates the device copy of the probe
    records), while wadg_run_steps_noalloc runs and gives the same records."""
    from paper_2006_02551_gb300.wadg import WADG_ENOMEM, WadgError
    w = workload("cube4_n3")
    ref = make(w, "fp32")
    dt = ref.stable_dt(1.0)
    r_ref = ref.run_steps(11, dt)
    q_ref, _ = ref.get_state()
    ref.close()

    s = make(w, "fp32")
    held = s.set_memory_limit(0)
    s.set_memory_limit(held)
    with pytest.raises(WadgError) as err:
        s.run_steps(11, dt)
    assert err.value.status == WADG_ENOMEM
    s.set_state(None, 0.0)
    r = s.run_steps_noalloc(11, dt)
    assert s.set_memory_limit(held) == held
    q, _ = s.get_state()
    assert close_to(r_ref, r, TOL["fp32"])
    assert close_to(q_ref, q, TOL["fp32"])
    s.close()


def test_noalloc_rejects_oversized_step_records():
    from paper_2006_02551_gb300 import Solver, WadgError, wadg
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
