"""Device-resident state exchange at the C ABI: the state set from and read
into CUDA tensors (wadg_set_state / wadg_get_state with on_device = 1), and
the state buffers held in caller-owned (PyTorch) device memory
(wadg_bind_state).  Every result must equal, bit for bit, the one reached
through host memory, and the device path must copy no state bytes between
host and device (wadg_transfer_bytes)."""
import numpy as np
import pytest

from synthetic import workload
from tests.parity_util import pml_mask, random_states, to_lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def solver(precision, stream=None):
    from paper_2006_02551_gb300 import Solver
    from synthetic import cube_tet_mesh
    w = workload("cube4_n3")
    v, e = cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed)
    s = Solver(w.N, precision, stream=stream)
    s.set_mesh(v, e)
    s.set_pml(w.pml)
    s.set_sources(list(w.sources))
    s.set_probes(list(w.probes))
    mask = pml_mask(v, e, w.pml)
    q0 = to_lib(random_states(len(e), s.info()["Np"], 1, 11, mask))
    return s, q0


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32"])
def test_device_exchange_matches_host_exchange(precision):
    stream = torch.cuda.current_stream().cuda_stream
    a, q0 = solver(precision)
    b, _ = solver(precision, stream=stream)
    dt = a.stable_dt(1.0)
    a.set_state(q0, 0.5)
    a.run_steps(7, dt)
    qa, ta = a.get_state()

    qdev = torch.from_numpy(q0).cuda()
    h0 = b.transfer_bytes()
    b.set_state(qdev, 0.5)
    b.run_steps(7, dt, record=False)
    out = torch.empty_like(qdev)
    _, tb = b.get_state(out)
    torch.cuda.current_stream().synchronize()
    h1 = b.transfer_bytes()
    assert ta == tb
    assert np.array_equal(out.cpu().numpy(), qa)
    # no state crossed the host boundary: only the step clocks and flags
    assert h1[0] - h0[0] < 1024 and h1[1] - h0[1] < 1024, (h0, h1)
    # the host path moves the whole state
    b.get_state()
    h2 = b.transfer_bytes()
    assert h2[1] - h1[1] >= q0.size * (8 if precision == "fp64" else 4) // 2
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "tf32"])
def test_bound_state_steps_as_owned_state(precision):
    a, q0 = solver(precision)
    b, _ = solver(precision)
    dt = a.stable_dt(1.0)
    for s in (a, b):
        s.set_state(q0, 0.0)
    held0 = b.set_memory_limit(0)
    buf = torch.empty(b.state_bytes() + 4096, dtype=torch.uint8, device="cuda")
    b.bind_state(buf)
    held1 = b.set_memory_limit(0)
    assert held1 < held0                          # the library released its buffers
    ra = a.run_steps(9, dt)
    rb = b.run_steps(9, dt)
    assert np.array_equal(ra, rb)
    qa, _ = a.get_state()
    qb, _ = b.get_state()
    assert np.array_equal(qa, qb)
    # set-up calls that rebuild the state keep using the bound memory
    b.set_pml(workload("cube4_n3").pml)
    b.set_state(q0, 0.0)
    b.run_steps(9, dt)
    assert np.array_equal(b.get_state()[0], qa)
    # too small a buffer is refused, and unbinding moves the state back
    from paper_2006_02551_gb300 import WadgError
    with pytest.raises(WadgError):
        b.bind_state(torch.empty(1024, dtype=torch.uint8, device="cuda"))
    before = b.set_memory_limit(0)
    b.bind_state(None)
    assert b.set_memory_limit(0) - before == b.memory_report()["state"]
    assert np.array_equal(b.get_state()[0], qa)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_host_exchange_staged_equals_host_loop(precision):
    """The host-memory exchange converts on the device through a staging
    buffer; capped at the bytes it holds, a context converts on the host
    instead.  Both give the same internal state and the same array back, bit
    for bit, and each moves the whole state across the host boundary."""
    a, q0 = solver(precision)
    b, _ = solver(precision)
    dt = a.stable_dt(1.0)
    b.set_memory_limit(b.set_memory_limit(0))     # no room for a staging buffer
    for s in (a, b):
        h0 = s.transfer_bytes()
        s.set_state(q0, 0.25)
        assert s.transfer_bytes()[0] - h0[0] >= q0.size * (8 if precision == "fp64" else 4) // 2
    qa, _ = a.get_state()
    qb, _ = b.get_state()
    assert np.array_equal(qa, qb)
    b.set_memory_limit(0)                          # room for the probe records
    a.run_steps(5, dt, record=False)
    b.run_steps(5, dt, record=False)
    b.set_memory_limit(b.set_memory_limit(0))     # the read back converts on the host
    qa, ta = a.get_state()
    qb, tb = b.get_state()
    assert ta == tb and np.array_equal(qa, qb)
    a.close()
    b.close()
