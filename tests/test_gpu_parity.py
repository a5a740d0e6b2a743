"""GPU parity: the library (called through the C ABI) against the FP64
oracle, element by element, on seeded synthetic meshes.

Tolerances: 1e-12 for the FP64 path, 1e-5 for the FP32 path (FP32 rounding
of a few hundred operations per value, accumulated over the steps of each
case, stays near 1e-6).  One-stage cases bound the relative L2 error of the
stage increment q_new - q_old (the part the kernel computes; the state itself
is 5-20 times larger at these step sizes), with the FP32 cases' random input
rounded to FP32 on both sides; whole runs bound the relative L2 error of the
state, the probe records and the objective."""
import numpy as np
import pytest

from oracle import lserk
from synthetic import Dipole, PmlProfile, workload
from tests.parity_util import (increment_err, make_pair, random_states, rel_err,
                                 round_states, to_lib)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
PML3 = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0)
PML3K = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0, kappa_max=2.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def one_stage_case(N, prec, prof, n_hex=4, seed=0, eps=None, mu=None, stage=0,
                   sources=(), n_batch=1):
    s, sim, mask = make_pair(N, n_hex, 0.15, seed, prof, prec, sources=sources,
                             eps=eps, mu=mu, n_batch=n_batch)
    K, Np = sim.K, sim.Np
    st = round_states(random_states(K, Np, n_batch, 100 + seed, mask), prec)
    q0 = to_lib(st)
    s.set_state(q0, 0.0)
    dt, t = 0.01, 0.37
    s.rk_stage(stage, t, dt)
    q, _ = s.get_state()
    # oracle: the same stage from res = 0
    for b in range(n_batch):
        rhs = sim.rhs(st[b], t + lserk.RK_C[stage] * dt, b)
        for f in st[b]:
            res = dt * rhs[f]
            st[b][f] = st[b][f] + lserk.RK_B[stage] * res
    err = increment_err(q, st, q0, mask)
    s.close()
    return err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_one_stage_waa_pml(N, prec):
    err = one_stage_case(N, prec, PML3)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [1, 3, 4])
def test_one_stage_kappa(N, prec):
    err = one_stage_case(N, prec, PML3K)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_one_stage_no_pml_and_materials(prec):
    rng = np.random.default_rng(4)
    K = 6 * 27
    err = one_stage_case(2, prec, None, n_hex=3, eps=rng.uniform(1, 4, K),
                         mu=rng.uniform(1, 2, K), stage=3)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_one_stage_everything_in_pml_with_source(prec):
    # a profile that puts every element in the PML class (single hex: 6 tets,
    # all faces PEC) and a source inside a PML element
    prof = PmlProfile(u0=0.1, L=0.9, sigma_max=5.0, p_sigma=2.0, kappa_max=1.5)
    src = (Dipole(x=(0.3, -0.2, 0.25), dir=(0.6, 0.0, 0.8), t0=0.3, width=0.2),)
    err = one_stage_case(3, prec, prof, n_hex=1, sources=src, stage=2)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_sources_one_stage(prec):
    srcs = tuple(Dipole(x=(0.1 * b, -0.05 * b, 0.02), dir=(0, 0, 1), t0=0.4,
                        width=0.2 + 0.05 * b, batch=b) for b in range(3))
    err = one_stage_case(2, prec, PML3, n_hex=3, sources=srcs, stage=1, n_batch=3)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_workload_full_run(prec):
    """The 384-tet N=3 workload with its dipole and 8 probes over all 200
    steps through run_steps (the CUDA-graph path)."""
    w = workload("cube4_n3")
    s, sim, mask = make_pair(w.N, w.n_hex, w.jitter, w.mesh_seed, w.pml, prec,
                             sources=w.sources, probes=w.probes)
    dt = sim.stable_dt(1.0)
    assert abs(s.stable_dt(1.0) - dt) < 1e-15 * dt
    s.set_state(None, 0.0)
    rec = s.run_steps(w.steps, dt)
    q, t = s.get_state()
    st = sim.zero_state()
    st, t_ref, rec_ref, J_ref = sim.run(st, w.steps, dt)
    assert abs(t - t_ref) < 1e-12
    err = rel_err(q, st, mask)
    assert err < TOL[prec], err
    perr = np.linalg.norm(rec - rec_ref) / np.linalg.norm(rec_ref)
    assert perr < TOL[prec], perr
    J = s.objective()[0]
    assert abs(J - J_ref) / J_ref < TOL[prec]
    s.close()


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_kappa_workload_fp64_full_run(N):
    """The kappa_max = 2 variant of the 384-tet workload (the general WAA path
    with a != 1, eqs. 26, 27) over its full 200 steps: state, probe records
    and objective."""
    w = workload("cube4_n3_kappa2")
    s, sim, mask = make_pair(N, w.n_hex, w.jitter, w.mesh_seed, w.pml, "fp64",
                             sources=w.sources, probes=w.probes)
    dt = sim.stable_dt(1.0)
    s.set_state(None, 0.0)
    rec = s.run_steps(w.steps, dt)
    q, _ = s.get_state()
    st = sim.zero_state()
    st, _, rec_ref, J_ref = sim.run(st, w.steps, dt)
    err = rel_err(q, st, mask)
    perr = np.linalg.norm(rec - rec_ref) / np.linalg.norm(rec_ref)
    J = s.objective()[0]
    s.close()
    assert err < TOL["fp64"], (N, err)
    assert perr < TOL["fp64"], (N, perr)
    assert abs(J - J_ref) <= TOL["fp64"] * J_ref


def test_state_roundtrip_and_errors():
    from paper_2006_02551_gb300 import Solver, WadgError, wadg
    s, sim, mask = make_pair(2, 2, 0.1, 3, PML3, "fp64")
    st = random_states(sim.K, sim.Np, 1, 9, mask)
    q0 = to_lib(st)
    s.set_state(q0, 1.25)
    q1, t = s.get_state()
    assert t == 1.25
    assert np.array_equal(q1, q0)
    with pytest.raises(WadgError) as e:
        s.set_probes([(3.0, 0.0, 0.0)])
    assert e.value.status == wadg.WADG_ENOTFOUND
    with pytest.raises(WadgError) as e:
        s.rk_stage(7, 0.0, 0.1)
    assert e.value.status == wadg.WADG_EINVAL
    s.close()
    s2 = Solver(2, "fp64")
    with pytest.raises(WadgError) as e:
        s2.run_steps(1, 0.1)
    assert e.value.status == wadg.WADG_ESTATE
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    with pytest.raises(WadgError) as e:       # inverted element
        s2.set_mesh(v, np.array([[0, 2, 1, 3]]))
    assert e.value.status == wadg.WADG_EINVAL
    s2.close()
