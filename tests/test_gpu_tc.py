"""GPU parity of the tensor-core (tcgen05, TF32 operands, FP32 accumulation
and state) stage path against the FP64 oracle.

TF32 keeps 10 mantissa bits (relative rounding 2^-11 ~ 4.9e-4 per operand),
so the right-hand side carries errors near 1e-3 of its size.  One-stage cases
compare the state increment (q_new - q_old) with a bound of 1e-2 relative to
the oracle's increment; whole runs state their relative L2 error and bound it
by 2e-2."""
import numpy as np
import pytest

from oracle import lserk
from synthetic import Dipole, PmlProfile, workload
from tests.parity_util import make_pair, random_states, rel_err, to_lib

pytestmark = pytest.mark.gpu

PML3 = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def increment_error(N, prof, n_hex=4, stage=0, sources=(), n_batch=1, seed=0,
                    precision="tf32", mesh=None):
    s, sim, mask = make_pair(N, n_hex, 0.15, seed, prof, precision, sources=sources,
                             n_batch=n_batch, mesh=mesh)
    st = random_states(sim.K, sim.Np, n_batch, 300 + seed, mask)
    q0 = to_lib(st)
    s.set_state(q0, 0.0)
    dt, t = 0.01, 0.37
    s.rk_stage(stage, t, dt)
    q, _ = s.get_state()
    for b in range(n_batch):
        rhs = sim.rhs(st[b], t + lserk.RK_C[stage] * dt, b)
        for f in st[b]:
            st[b][f] = st[b][f] + lserk.RK_B[stage] * dt * rhs[f]
    ref = to_lib(st)
    sel = np.ones(ref.shape[:3], bool)
    sel[:, ~mask, 6:] = False
    inc = (ref - q0)[sel]
    err = np.linalg.norm((q - ref)[sel]) / np.linalg.norm(inc)
    s.close()
    return err


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_tc_one_stage_with_pml(N):
    err = increment_error(N, PML3)
    assert err < 1e-2, err


@pytest.mark.parametrize("N", [2, 4])
def test_tc_one_stage_without_pml(N):
    err = increment_error(N, None, n_hex=3, stage=2)
    assert err < 1e-2, err


def test_tc_one_stage_all_pml_single_hex_with_source():
    prof = PmlProfile(u0=0.1, L=0.9, sigma_max=5.0, p_sigma=2.0)
    src = (Dipole(x=(0.3, -0.2, 0.25), dir=(0.6, 0.0, 0.8), t0=0.3, width=0.2),)
    err = increment_error(3, prof, n_hex=1, sources=src, stage=3)
    assert err < 1e-2, err


def test_tc_batched_one_stage():
    srcs = tuple(Dipole(x=(0.1 * b, -0.05 * b, 0.02), t0=0.4, width=0.25, batch=b)
                 for b in range(3))
    err = increment_error(3, PML3, n_hex=3, sources=srcs, stage=1, n_batch=3)
    assert err < 1e-2, err


def test_tc_small_workload_full_run():
    w = workload("cube4_n3")
    s, sim, mask = make_pair(w.N, w.n_hex, w.jitter, w.mesh_seed, w.pml, "tf32",
                             sources=w.sources, probes=w.probes)
    dt = sim.stable_dt(1.0)
    s.set_state(None, 0.0)
    rec = s.run_steps(w.steps, dt)
    q, _ = s.get_state()
    st = sim.zero_state()
    st, _, rec_ref, _ = sim.run(st, w.steps, dt)
    err = rel_err(q, st, mask)
    perr = np.linalg.norm(rec - rec_ref) / np.linalg.norm(rec_ref)
    print(f"TF32 cube4_n3 200 steps: state rel L2 {err:.3e}, probes {perr:.3e}")
    assert err < 2e-2 and perr < 2e-2, (err, perr)
    s.close()


def test_tc_rejects_kappa_and_high_order():
    from paper_2006_02551_gb300 import Solver, WadgError, wadg
    from synthetic import cube_tet_mesh
    # TF32 at N = 5 takes a PML only with a compact volume rule
    t = Solver(5, "tf32")
    t.set_mesh(*cube_tet_mesh(2, 0.1, 0))
    with pytest.raises(WadgError) as e:
        t.set_pml(PML3)
    assert e.value.status == wadg.WADG_EUNSUPPORTED
    t.close()
    s, sim, mask = make_pair(2, 2, 0.1, 0, None, "tf32")
    with pytest.raises(WadgError) as e:
        s.set_pml(PmlProfile(kappa_max=2.0))
    assert e.value.status == wadg.WADG_EUNSUPPORTED
    s.close()


@pytest.mark.parametrize("precision,bound", [("tf32", 1e-2), ("bf16", 3e-2)])
@pytest.mark.parametrize("drop", ["interior", "pml"])
def test_tc_blocks_off_16_byte_boundaries(precision, bound, drop):
    """Cube meshes have an even element count in each class, so every staged
    E,H and P block starts on a 16-byte boundary.  Removing one element (its
    faces become PEC walls, for the library and the oracle alike) makes the
    PML class start at an odd element ("interior") or holds an odd number of
    PML elements ("pml"); with two excitations the second one's blocks then
    start 8 bytes past a boundary as well, which the staging copies cover.
    (An element block is 24 N_p bytes: only an odd N_p, N = 4 here, leaves
    blocks off the boundary; the geometry blocks are off it at any N.)"""
    from synthetic import cube_tet_mesh
    from tests.parity_util import pml_mask
    v, e = cube_tet_mesh(4, 0.15, 0)
    mask = pml_mask(v, e, PML3)
    k = int(np.flatnonzero(mask if drop == "pml" else ~mask)[0])
    e = np.delete(e, k, axis=0)
    mask = pml_mask(v, e, PML3)
    K1 = int(mask.sum())
    K0 = len(e) - K1
    assert (K0 % 2 == 1) if drop == "interior" else (K1 % 2 == 1)
    err = increment_error(4, PML3, n_batch=2, precision=precision, mesh=(v, e))
    assert err < bound, err


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_tc_stage_is_repeatable_with_the_conical_rule(precision):
    """With the (N+1)^3-point rule both classes run tc_stage_kernel: one stage
    gives the same state bit for bit every time (no atomics in the kernel, so
    a difference would be a race between its warp roles)."""
    prof = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0)
    s, sim, mask = make_pair(4, 4, 0.15, 2, prof, precision,
                             sources=[Dipole(x=(0.1, -0.05, 0.2), t0=0.3, width=0.2)])
    q0 = to_lib(random_states(sim.K, sim.Np, 1, 71, mask))
    outs = []
    for _ in range(6):
        s.set_state(q0, 0.0)
        s.rk_stage(2, 0.3, 0.01)
        outs.append(s.get_state()[0])
    s.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
