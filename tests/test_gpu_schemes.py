"""GPU parity of the other two PML schemes against the FP64 oracle:

* the stored-matrix scheme of eqs. 10-13 (per element and axis the
  operators M_k^-1 M_k^{b_u, c_u, d_u}, and with kappa_max != 1 also
  M_k^-1 M_k^{1/kappa_u} and (M_k^{a_u})^-1 M_k, built on the device from
  the same Stroud rule with N + 6 points per direction that the oracle
  uses; the oracle solves with M_k^{a_u} where the library multiplies by
  the inverse it formed);
* the element-constant coefficient variant (the weight-adjusted kernels with
  the profile evaluated at the element centroid, the piecewise-constant
  paving of the PML the paper compares with).

Tolerances as in the weight-adjusted parity tests: one-stage cases bound the
relative L2 error of the stage increment by 1e-12 (FP64), 1e-5 (FP32) and
1e-2 (TF32 context); whole runs bound the state and probe records by 1e-12
and 1e-5."""
import numpy as np
import pytest

from oracle import lserk
from synthetic import PmlProfile, workload
from synthetic import cube_tet_mesh
from tests.parity_util import (increment_err, make_pair, pml_mask, random_states, rel_err,
                                 round_states, to_lib)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
PML3 = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0)
PML3K = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0, kappa_max=2.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def one_stage(N, prec, scheme, prof=PML3, n_hex=None, stage=1):
    # the oracle's stored operators cost K N_h N_p^2 per matrix: smaller
    # meshes at the higher orders
    n_hex = n_hex or {1: 4, 2: 4, 3: 4, 4: 3, 5: 2}[N]
    s, sim, mask = make_pair(N, n_hex, 0.15, 3, prof, prec, scheme=scheme)
    st = round_states(random_states(sim.K, sim.Np, 1, 17, mask), prec)
    q0 = to_lib(st)
    s.set_state(q0, 0.0)
    dt, t = 0.01, 0.21
    s.rk_stage(stage, t, dt)
    q, _ = s.get_state()
    rhs = sim.rhs(st[0], t + lserk.RK_C[stage] * dt, 0)
    for f in st[0]:
        st[0][f] = st[0][f] + lserk.RK_B[stage] * dt * rhs[f]
    s.close()
    return increment_err(q, st, q0, mask)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_one_stage_stored(N, prec):
    err = one_stage(N, prec, "stored")
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_one_stage_stored_kappa(N, prec):
    """kappa_max = 2: a_u != 1, so (M^a)^-1 M_k and M_k^-1 M^{1/kappa} are no
    longer the identity (the paper's general 15 N_p^2 operators)."""
    err = one_stage(N, prec, "stored", prof=PML3K)
    assert err < TOL[prec], err


def test_stored_kappa_workload_run():
    """The kappa_max = 2 variant of the 384-tet workload with the stored
    scheme, FP64, its full 200 steps: state, probe records and objective."""
    w = workload("cube4_n3_kappa2")
    s, sim, mask = make_pair(w.N, w.n_hex, w.jitter, w.mesh_seed, w.pml, "fp64",
                             sources=w.sources, probes=w.probes, scheme="stored")
    dt = sim.stable_dt(1.0)
    s.set_state(None, 0.0)
    rec = s.run_steps(w.steps, dt)
    q, _ = s.get_state()
    st, _, rec_ref, J_ref = sim.run(sim.zero_state(), w.steps, dt)
    s_err = rel_err(q, st, mask)
    p_err = np.linalg.norm(rec - rec_ref) / np.linalg.norm(rec_ref)
    J = s.objective()[0]
    s.close()
    assert s_err < TOL["fp64"], s_err
    assert p_err < TOL["fp64"], p_err
    assert abs(J - J_ref) <= TOL["fp64"] * J_ref


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [1, 3, 4])
def test_one_stage_element_constant(N, prec):
    err = one_stage(N, prec, "ec")
    assert err < TOL[prec], err


@pytest.mark.parametrize("scheme", ["stored", "ec"])
def test_one_stage_tf32_context(scheme):
    # stored: the PML class runs the FP32 CUDA-core kernel, the rest the
    # tensor-core kernel; ec: both classes on the tensor-core kernels
    err = one_stage(4, "tf32", scheme)
    assert err < 1e-2, err


@pytest.mark.parametrize("scheme", ["stored", "ec"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_workload_run(scheme, prec):
    """The 384-tet N=3 workload with its dipole and probes through run_steps
    (the CUDA-graph path), 100 steps."""
    w = workload("cube4_n3")
    s, sim, mask = make_pair(w.N, w.n_hex, w.jitter, w.mesh_seed, w.pml, prec,
                             sources=w.sources, probes=w.probes, scheme=scheme)
    dt = sim.stable_dt(1.0)
    nst = 100
    s.set_state(None, 0.0)
    rec = s.run_steps(nst, dt)
    q, _ = s.get_state()
    st = sim.zero_state()
    st, _, rec_ref, J_ref = sim.run(st, nst, dt)
    err = rel_err(q, st, mask)
    assert err < TOL[prec], err
    perr = np.linalg.norm(rec - rec_ref) / np.linalg.norm(rec_ref)
    assert perr < TOL[prec], perr
    s.close()


def test_stored_memory_and_errors():
    from paper_2006_02551_gb300 import WadgError
    w = workload("cube4_n3")
    for prec, rs in (("fp64", 8), ("fp32", 4)):
        s, sim, mask = make_pair(w.N, w.n_hex, w.jitter, w.mesh_seed, w.pml, prec,
                                 probes=w.probes, scheme="stored")
        Np = sim.Np
        NpP = (Np + 3) & ~3
        mem = s.memory_report()
        assert mem["pml_coeff"] == int(mask.sum()) * 9 * Np * NpP * rs
        with pytest.raises(WadgError):   # the adjoint is built for the WAA scheme
            s.adjoint(5, 0.01, 5)
        # kappa != 1: 15 operators per element (the paper's 15 N_p^2)
        s.set_pml(PML3K, "stored")
        mask_k = pml_mask(*cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed), PML3K)
        assert s.memory_report()["pml_coeff"] == int(mask_k.sum()) * 15 * Np * NpP * rs
        s.close()
