"""Failure detection on the GPU without a fault.

The tensor-core stage kernels hand work between one issuing thread and the
compute warps through mbarriers, and every wait on them gives up after about a
second.  wadg_arm_wait_timeout makes one block of a later launch issue a flux
product without its completion signal, so one of those waits runs out.  These
tests check that the stepping call then reports WADG_ETIMEOUT within seconds,
that the flag does not outlive the call, and that the context steps exactly as
before afterwards.  Nothing here faults, traps or waits without a limit."""
import time

import numpy as np
import pytest

from synthetic import PmlProfile
from tests.parity_util import make_pair, random_states, to_lib

pytestmark = pytest.mark.gpu

PML3 = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def _status_of(call):
    from paper_2006_02551_gb300 import WadgError
    try:
        call()
    except WadgError as e:
        return e.status
    return 0


@pytest.mark.parametrize("rule", ["default", "compact"])
@pytest.mark.parametrize("precision", ["tf32", "bf16"])
@pytest.mark.parametrize("prof", [PML3, None], ids=["pml", "nopml"])
def test_withheld_signal_reports_timeout_and_context_recovers(precision, prof, rule):
    """Both tensor-core PML kernels (the (N+1)^3-rule kernel and the
    row-owned kernel of compact rules) and the non-PML kernel."""
    from paper_2006_02551_gb300.wadg import WADG_ETIMEOUT
    from synthetic import compact_rule
    if rule == "compact" and prof is None:
        pytest.skip("the rule only concerns the PML class")
    s, sim, mask = make_pair(3, 4, 0.15, 5, prof, precision,
                             volume_rule=compact_rule(3) if rule == "compact" else None)
    q0 = to_lib(random_states(sim.K, sim.Np, 1, 17, mask))
    dt = s.stable_dt(0.5)

    s.set_state(q0, 0.0)
    s.run_steps(3, dt)
    clean, _ = s.get_state()

    s.set_state(q0, 0.0)
    s.arm_wait_timeout()
    t0 = time.perf_counter()
    st = _status_of(lambda: s.run_steps(3, dt))
    elapsed = time.perf_counter() - t0
    assert st == WADG_ETIMEOUT
    # one withheld signal: the compute warps' wait and the issuing thread's
    # wait for the next operands each end after about a second
    assert elapsed < 20.0, elapsed
    hit, _ = s.get_state()
    assert np.all(np.isfinite(hit))

    # the request was taken and the flag cleared: the context steps as before
    s.set_state(q0, 0.0)
    s.run_steps(3, dt)
    again, _ = s.get_state()
    assert np.array_equal(again, clean)

    # the single-stage entry point reports it the same way
    s.set_state(q0, 0.0)
    s.arm_wait_timeout()
    assert _status_of(lambda: s.rk_stage(0, 0.0, dt)) == WADG_ETIMEOUT
    s.set_state(q0, 0.0)
    s.rk_stage(0, 0.0, dt)

    # and so does the allocation-free stepping entry point, whose next call
    # then steps as before (the flag was read and cleared)
    s.set_state(q0, 0.0)
    s.arm_wait_timeout()
    assert _status_of(lambda: s.run_steps_noalloc(3, dt)) == WADG_ETIMEOUT
    s.set_state(q0, 0.0)
    s.run_steps_noalloc(3, dt)
    again, _ = s.get_state()
    assert np.array_equal(again, clean)
    s.close()


def test_cuda_core_contexts_have_no_waits_to_arm():
    from paper_2006_02551_gb300.wadg import WADG_EUNSUPPORTED
    for precision in ("fp32", "fp64"):
        s, _, _ = make_pair(2, 2, 0.1, 1, PML3, precision)
        assert _status_of(s.arm_wait_timeout) == WADG_EUNSUPPORTED
        s.close()


def assert_refused(s, dt):
    """Every call that launches kernels or touches the device state returns
    ESTATE (before any launch) after a set-up call failed part-way."""
    from paper_2006_02551_gb300.wadg import WADG_ESTATE
    for call in (lambda: s.run_steps(1, dt), lambda: s.run_steps_noalloc(1, dt),
                 lambda: s.rk_stage(0, 0.0, dt), lambda: s.set_state(None, 0.0),
                 lambda: s.get_state(), lambda: s.profile_stage(1, dt),
                 lambda: s.adjoint(2, dt, 1)):
        assert _status_of(call) == WADG_ESTATE


def test_memory_limit_reports_enomem_and_context_recovers():
    """An allocation past the context's cap fails as an exhausted device
    would (ENOMEM, no device call made), and the context then completes the
    same work once the cap is raised, bit for bit as a context never capped."""
    from paper_2006_02551_gb300 import Solver
    from paper_2006_02551_gb300.wadg import WADG_ENOMEM
    from synthetic import cube_tet_mesh

    v, e = cube_tet_mesh(3, 0.1, 2)

    def setup(s):
        s.set_mesh(v, e)
        s.set_pml(PML3)
        s.set_state(None, 0.0)

    ref = Solver(2, "fp32")
    setup(ref)
    ref.set_probes([(0.1, 0.2, 0.3)])
    dt = ref.stable_dt(0.5)
    rec_ref = ref.run_steps(4, dt)
    q_ref, _ = ref.get_state()
    ref.close()

    s = Solver(2, "fp32")
    held0 = s.set_memory_limit(0)
    assert held0 > 0                                   # operators, counters
    s.set_memory_limit(held0 + 1024)
    assert _status_of(lambda: s.set_mesh(v, e)) == WADG_ENOMEM
    # nothing steps or touches the state on a half-built context
    assert_refused(s, dt)
    s.set_memory_limit(0)
    setup(s)
    held1 = s.set_memory_limit(0)
    assert held1 > held0
    # a profile whose fields and samples do not fit leaves the tables
    # incomplete (capped at what the context holds without a PML)
    s.set_pml(None)
    s.set_memory_limit(s.set_memory_limit(0))
    assert _status_of(lambda: s.set_pml(PML3)) == WADG_ENOMEM
    assert_refused(s, dt)
    s.set_memory_limit(0)
    s.set_pml(PML3)
    s.set_state(None, 0.0)
    s.set_memory_limit(held1)                          # cap at what is held
    # probe records are allocated by the first run: refuse them, then allow
    assert _status_of(lambda: s.set_probes([(0.1, 0.2, 0.3)])) == WADG_ENOMEM
    assert_refused(s, dt)
    s.set_memory_limit(0)
    s.set_probes([(0.1, 0.2, 0.3)])
    s.set_memory_limit(s.set_memory_limit(0))          # cap at what is held
    assert _status_of(lambda: s.run_steps(4, dt)) == WADG_ENOMEM
    s.set_memory_limit(0)
    s.set_state(None, 0.0)
    rec = s.run_steps(4, dt)
    q, _ = s.get_state()
    assert np.array_equal(q, q_ref)
    assert np.array_equal(rec, rec_ref)
    # the adjoint's buffers count too
    s.set_memory_limit(s.set_memory_limit(0))
    assert _status_of(lambda: s.adjoint(4, dt)) == WADG_ENOMEM
    s.set_memory_limit(0)
    s.set_state(None, 0.0)
    J, *_ = s.adjoint(4, dt)
    assert np.all(np.isfinite(J))
    s.close()


def test_malformed_input_is_rejected():
    from paper_2006_02551_gb300 import Solver
    from paper_2006_02551_gb300.wadg import WADG_EINVAL
    from synthetic import Dipole

    s = Solver(1, "fp64")
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, -1], [0, 0, 2.0]])
    # three positively oriented tetrahedra on one face: not a manifold mesh
    bad = np.array([[0, 1, 2, 3], [0, 2, 1, 4], [0, 1, 2, 5]])
    assert _status_of(lambda: s.set_mesh(v, bad)) == WADG_EINVAL
    assert _status_of(lambda: s.set_mesh(v, np.array([[0, 1, 2, 6]]))) == WADG_EINVAL
    s.set_mesh(v, bad[:2])                      # two elements, one shared face
    assert _status_of(lambda: s.set_materials(np.array([1.0, -1.0]), None)) == WADG_EINVAL
    src = Dipole(x=(0.1, 0.1, 0.1), dir=(0.0, 0.0, 1.0), t0=1.0, width=0.0)
    assert _status_of(lambda: s.set_sources([src])) == WADG_EINVAL
    s.close()
