"""GPU parity of the weight-adjusted PML on the compact volume rules (degree
2N, fully symmetric, 4 / 14 / 24 / 46 / N=5 points; the fewer-point rules of
Section III) against the FP64 oracle built on the same rule, and the
checks wadg_set_quadrature makes of a caller's rule.

One-stage cases bound the relative L2 error of the stage increment: 1e-12
(FP64), 1e-5 (FP32), 1e-2 (TF32), 3e-2 (BF16); whole runs bound the state
and probe records (1e-12 FP64, 2e-2 TF32)."""
import numpy as np
import pytest

from oracle import lserk
from synthetic import Dipole, PmlProfile, compact_rule, workload
from tests.parity_util import (increment_err, make_pair, random_states, rel_err,
                               round_states, to_lib)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "tf32": 1e-2, "bf16": 3e-2}
PML3 = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0)
PML3K = PmlProfile(u0=0.75, L=0.25, sigma_max=20.0, p_sigma=3.0, kappa_max=2.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def pair(N, prec, prof, n_hex=4, seed=0, sources=(), probes=(), scheme="waa", jitter=0.15):
    from oracle.solver import Simulation
    from paper_2006_02551_gb300 import Solver
    from synthetic import cube_tet_mesh
    rule = compact_rule(N)
    v, e = cube_tet_mesh(n_hex, jitter, seed)
    sim = Simulation(N, v, e, profile=prof, sources=sources, probes=probes,
                     volume_rule=rule)
    if scheme == "ec":
        sim.disc.set_profile(prof, element_constant_at=sim.geom.verts.mean(axis=1).T)
    s = Solver(N, prec)
    s.set_quadrature(rule)
    s.set_mesh(v, e)
    s.set_pml(prof, scheme)
    if sources:
        s.set_sources(list(sources))
    if probes:
        s.set_probes(list(probes))
    from tests.parity_util import pml_mask
    return s, sim, pml_mask(v, e, prof)


def one_stage(N, prec, prof, stage=1, scheme="waa", n_hex=4):
    src = (Dipole(x=(0.1, -0.05, 0.2), dir=(0.0, 0.6, 0.8), t0=0.3, width=0.2),)
    s, sim, mask = pair(N, prec, prof, n_hex=n_hex, sources=src, scheme=scheme)
    st = round_states(random_states(sim.K, sim.Np, 1, 50 + N, mask), prec)
    q0 = to_lib(st)
    s.set_state(q0, 0.0)
    dt, t = 0.01, 0.27
    s.rk_stage(stage, t, dt)
    q, _ = s.get_state()
    info = s.info()
    s.close()
    rhs = sim.rhs(st[0], t + lserk.RK_C[stage] * dt, 0)
    for f in st[0]:
        st[0][f] = st[0][f] + lserk.RK_B[stage] * dt * rhs[f]
    assert info["Nq"] == compact_rule(N).shape[0]
    return increment_err(q, st, q0, mask)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_one_stage_compact_rule(N, prec):
    err = one_stage(N, prec, PML3, n_hex=4 if N < 5 else 3)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [2, 4])
def test_one_stage_compact_rule_kappa(N, prec):
    err = one_stage(N, prec, PML3K, stage=3)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_one_stage_compact_rule_element_constant(prec):
    err = one_stage(3, prec, PML3, scheme="ec")
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_small_workload_full_run_compact_rule(prec):
    w = workload("cube4_n3")
    s, sim, mask = pair(w.N, prec, w.pml, n_hex=w.n_hex, seed=w.mesh_seed,
                        sources=w.sources, probes=w.probes, jitter=w.jitter)
    dt = sim.stable_dt(1.0)
    s.set_state(None, 0.0)
    rec = s.run_steps(w.steps, dt)
    q, _ = s.get_state()
    s.close()
    st = sim.zero_state()
    st, _, rec_ref, _ = sim.run(st, w.steps, dt)
    err = rel_err(q, st, mask)
    perr = np.linalg.norm(rec - rec_ref) / np.linalg.norm(rec_ref)
    print(f"{prec} cube4_n3 compact rule, 200 steps: state {err:.3e} probes {perr:.3e}")
    bound = 1e-12 if prec == "fp64" else 2e-2
    assert err < bound and perr < bound, (err, perr)


def test_rule_checks_and_capacities():
    from paper_2006_02551_gb300 import Solver, WadgError, wadg
    from synthetic import cube_tet_mesh
    v, e = cube_tet_mesh(2, 0.1, 0)

    def status(call):
        try:
            call()
        except WadgError as err:
            return err.status
        return 0

    s = Solver(3, "fp32")
    rule = compact_rule(3)
    assert status(lambda: s.set_quadrature(rule[:-1])) == wadg.WADG_EINVAL      # not exact
    bad = rule.copy()
    bad[0, 3] = -bad[0, 3]
    assert status(lambda: s.set_quadrature(bad)) == wadg.WADG_EINVAL           # negative weight
    out = rule.copy()
    out[0, :3] = (0.5, 0.5, 0.5)
    assert status(lambda: s.set_quadrature(out)) == wadg.WADG_EINVAL           # outside
    big = np.tile(rule, (3, 1))
    big[:, 3] /= 3
    assert status(lambda: s.set_quadrature(big)) == wadg.WADG_EUNSUPPORTED     # > (N+1)^3
    s.set_quadrature(rule)
    s.set_mesh(v, e)
    s.set_pml(PML3)
    K1 = s.info()["K_pml"]
    assert s.info()["Nq"] == rule.shape[0]
    # samples at the compact capacity (24 points at N = 3), FP32
    assert s.memory_report()["pml_coeff"] == K1 * 3 * 24 * 4
    s.set_quadrature(None)                                # back to (N+1)^3 = 64
    assert s.info()["Nq"] == 64
    assert s.memory_report()["pml_coeff"] == K1 * 3 * 64 * 4
    s.close()
    # TF32 at N = 5: only with a compact rule
    t = Solver(5, "tf32")
    t.set_mesh(v, e)
    assert status(lambda: t.set_pml(PML3)) == wadg.WADG_EUNSUPPORTED
    t.set_quadrature(compact_rule(5))
    t.set_pml(PML3)
    assert status(lambda: t.set_quadrature(None)) == wadg.WADG_EUNSUPPORTED
    t.close()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("N", [4, 5])
def test_tensor_core_stage_is_repeatable(N, prec):
    """One stage on the tensor-core kernels (row-owned PML class, non-PML
    class) gives the same state bit for bit every time (they have no
    atomics: a difference is a race between their roles), and matches the
    oracle."""
    src = (Dipole(x=(0.1, -0.05, 0.2), dir=(0.0, 0.6, 0.8), t0=0.3, width=0.2),)
    s, sim, mask = pair(N, prec, PML3, n_hex=4 if N < 5 else 3, sources=src)
    st = round_states(random_states(sim.K, sim.Np, 1, 60 + N, mask), prec)
    q0 = to_lib(st)
    dt, t = 0.01, 0.27
    outs = []
    for _ in range(6):
        s.set_state(q0, 0.0)
        s.rk_stage(1, t, dt)
        outs.append(s.get_state()[0])
    s.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
    rhs = sim.rhs(st[0], t + lserk.RK_C[1] * dt, 0)
    for f in st[0]:
        st[0][f] = st[0][f] + lserk.RK_B[1] * dt * rhs[f]
    assert increment_err(outs[0], st, q0, mask) < TOL[prec]
