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


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
@pytest.mark.parametrize("prof", [PML3, None], ids=["pml", "nopml"])
def test_withheld_signal_reports_timeout_and_context_recovers(precision, prof):
    from paper_2006_02551_gb300.wadg import WADG_ETIMEOUT
    s, sim, mask = make_pair(3, 4, 0.15, 5, prof, precision)
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
    s.close()


def test_cuda_core_contexts_have_no_waits_to_arm():
    from paper_2006_02551_gb300.wadg import WADG_EUNSUPPORTED
    for precision in ("fp32", "fp64"):
        s, _, _ = make_pair(2, 2, 0.1, 1, PML3, precision)
        assert _status_of(s.arm_wait_timeout) == WADG_EUNSUPPORTED
        s.close()
