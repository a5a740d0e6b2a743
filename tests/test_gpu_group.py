"""Grouped launches (wadg_group_*): meshes of different size and order, one
with two excitations, advanced by one launch per (order, element class)
variant and Runge-Kutta stage, give each member the state and probe records
of its own wadg_run_steps bit for bit (the same per-element arithmetic in the
same order; only the tile sizes, the grid and the launch grouping differ),
before and after the autotuner has picked the tile sizes and the grid; and a
small mixed group meets the FP32 parity bound against the oracle."""
import numpy as np
import pytest

from synthetic import Dipole, PmlProfile, cube_tet_mesh, workload

pytestmark = pytest.mark.gpu

PML = PmlProfile(u0=0.6, L=0.4, sigma_max=15.0, p_sigma=3.0)
PROBES = [(0.3, 0.2, -0.1), (-0.45, 0.1, 0.35)]
MEMBERS = [  # (N, n_hex, pml, n_batch)
    (2, 5, True, 1),
    (3, 4, True, 2),
    (4, 3, False, 1),
    (1, 6, True, 1),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2006_02551_gb300 import build
    build.build()


def make(N, n_hex, pml, nb, prec="fp32"):
    from paper_2006_02551_gb300 import Solver
    v, e = cube_tet_mesh(n_hex, 0.15, 10 + N)
    s = Solver(N, prec, n_batch=nb)
    s.set_mesh(v, e)
    if pml:
        s.set_pml(PML)
    src = [Dipole(x=(0.05, -0.02, 0.03), dir=(0.0, 0.0, 1.0), t0=0.5, width=0.2, batch=0)]
    if nb > 1:
        src.append(Dipole(x=(-0.1, 0.08, 0.0), dir=(1.0, 0.0, 0.0), t0=0.4, width=0.15, batch=1))
    s.set_sources(src)
    s.set_probes(PROBES)
    s.set_state(None, 0.0)
    return s


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("tune", [False, True, "per_item", "per_item_serial"])
def test_group_equals_single_runs(tune):
    from paper_2006_02551_gb300 import Group
    nsteps = 25
    singles = [make(*m) for m in MEMBERS]
    dts = [0.8 * s.stable_dt(1.0) for s in singles]
    ref = []
    for s, dt in zip(singles, dts):
        rec = s.run_steps(nsteps, dt)
        q, t = s.get_state()
        ref.append((q, rec, t))
        s.close()
    members = [make(*m) for m in MEMBERS]
    g = Group(members)
    if tune is True:
        g.autotune(dts, reps=10)
        for s in members:
            s.set_state(None, 0.0)   # the autotuner leaves the state undefined
    elif tune:
        g.set_tuning(per_item=True, parallel=tune == "per_item")
        assert g.info()["per_item"]
    info = g.info()
    assert info["items"] == sum(2 if m[2] else 1 for m in MEMBERS)
    # three calls (10, 7, 8 steps): the second reuses the first's graphs from
    # the same buffer parity, the third from the other one
    rec1 = g.run_steps(10, dts)
    rec2 = g.run_steps(7, dts)
    rec3 = g.run_steps(nsteps - 17, dts)
    for i, s in enumerate(members):
        q, t = s.get_state()
        qr, recr, tr = ref[i]
        assert abs(t - tr) < 1e-12
        rec = np.concatenate([rec1[i], rec2[i], rec3[i]])
        assert np.array_equal(q, qr), (i, rel(q, qr), np.abs(q - qr).max())
        assert np.array_equal(rec, recr), (i, rel(rec, recr))
    g.close()
    for s in members:
        s.close()


def test_group_rejects_repeated_members_and_variants_it_cannot_serve():
    from paper_2006_02551_gb300 import Group, WadgError
    from paper_2006_02551_gb300.wadg import WADG_EUNSUPPORTED
    a = make(3, 3, True, 1)
    b = make(3, 3, True, 1, prec="tf32")
    with pytest.raises(WadgError):
        Group([a, a])
    g = Group([a, b])                 # a tensor-core member: per-item launches only
    assert g.info()["per_item"]
    with pytest.raises(WadgError) as err:
        g.set_tuning(per_item=False)
    assert err.value.status == WADG_EUNSUPPORTED
    g.close()
    a.close()
    b.close()


@pytest.mark.parametrize("parallel", [True, False])
def test_mixed_precision_group_equals_single_runs(parallel):
    """Members of every kind in one group — TF32 and BF16 tensor-core
    contexts with the compact rule, an FP64 context, an FP32 context with the
    stored-matrix scheme — launched per item: each equals its own run_steps
    bit for bit over two calls."""
    from paper_2006_02551_gb300 import Group, Solver
    from synthetic import compact_rule

    def member(kind):
        N, n_hex, prec = {"tf32": (4, 3, "tf32"), "bf16": (3, 4, "bf16"),
                          "fp64": (2, 3, "fp64"), "stored": (3, 3, "fp32")}[kind]
        v, e = cube_tet_mesh(n_hex, 0.15, 30 + N)
        s = Solver(N, prec)
        if prec in ("tf32", "bf16"):
            s.set_quadrature(compact_rule(N))
        s.set_mesh(v, e)
        s.set_pml(PML, "stored" if kind == "stored" else "waa")
        s.set_sources([Dipole(x=(0.05, -0.02, 0.03), dir=(0.0, 0.0, 1.0), t0=0.4, width=0.15)])
        s.set_probes(PROBES)
        s.set_state(None, 0.0)
        return s

    kinds = ["tf32", "bf16", "fp64", "stored"]
    singles = [member(k) for k in kinds]
    dts = [0.8 * s.stable_dt(1.0) for s in singles]
    ref = []
    for s, dt in zip(singles, dts):
        rec = s.run_steps(11, dt)
        ref.append((s.get_state()[0], rec))
        s.close()
    members = [member(k) for k in kinds]
    g = Group(members)
    g.set_tuning(per_item=True, parallel=parallel)
    rec1 = g.run_steps(6, dts)
    rec2 = g.run_steps(5, dts)
    for i, s in enumerate(members):
        q, _ = s.get_state()
        assert np.array_equal(q, ref[i][0]), (kinds[i], rel(q, ref[i][0]))
        assert np.array_equal(np.concatenate([rec1[i], rec2[i]]), ref[i][1]), kinds[i]
    g.close()
    for s in members:
        s.close()


def test_small_mixed_group_matches_oracle():
    """Two members (N = 2 with two excitations, N = 3), each with PML, sources
    and probes, 12 grouped FP32 steps against the FP64 oracle's own runs:
    state (relative to its norm) and probe records within 1e-5."""
    from paper_2006_02551_gb300 import Group
    from tests.parity_util import make_pair, rel_err
    srcs = [Dipole(x=(0.05, -0.02, 0.03), dir=(0.0, 0.0, 1.0), t0=0.3, width=0.12, batch=0),
            Dipole(x=(-0.1, 0.08, 0.0), dir=(1.0, 0.0, 0.0), t0=0.25, width=0.1, batch=1)]
    cases = [(2, 3, 2, srcs), (3, 2, 1, srcs[:1])]   # (N, n_hex, n_batch, sources)
    pairs = [make_pair(N, n, 0.15, 20 + N, PML, "fp32", sources=sr, probes=PROBES, n_batch=nb)
             for N, n, nb, sr in cases]
    nsteps = 12
    dts = []
    for s, sim, _ in pairs:
        s.set_state(None, 0.0)
        dts.append(0.8 * sim.stable_dt(1.0))
    g = Group([p[0] for p in pairs])
    recs = g.run_steps(nsteps, dts)
    g.close()
    for (s, sim, mask), dt, rec in zip(pairs, dts, recs):
        st, _, rec_ref, _ = sim.run(sim.zero_state(), nsteps, dt)
        q, _ = s.get_state()
        err = rel_err(q, st, mask)
        perr = rel(rec, rec_ref)
        assert err < 1e-5, err
        assert perr < 1e-5, perr
        s.close()


def test_l2_clusters_equal_single_runs():
    """A member whose per-step data exceeds half the L2 (20^3 x 6 tets, N = 3,
    PML) with three small ones: the group advances them in L2 clusters (the
    small members together, the large one on its own), which changes only the
    order in time, so every member still equals its own run_steps bit for
    bit; a later call reuses the clusters."""
    from paper_2006_02551_gb300 import Group
    members_spec = [(3, 20, True, 1), (2, 3, True, 1), (3, 3, False, 2), (4, 2, True, 1)]
    nsteps = 9
    singles = [make(*m) for m in members_spec]
    dts = [0.8 * s.stable_dt(1.0) for s in singles]
    ref = []
    for s, dt in zip(singles, dts):
        rec = s.run_steps(nsteps, dt)
        ref.append((s.get_state()[0], rec))
        s.close()
    members = [make(*m) for m in members_spec]
    g = Group(members)
    rec1 = g.run_steps(4, dts)
    assert g.info()["clusters"] >= 2
    rec2 = g.run_steps(nsteps - 4, dts)
    for i, s in enumerate(members):
        q, _ = s.get_state()
        assert np.array_equal(q, ref[i][0]), (i, rel(q, ref[i][0]))
        assert np.array_equal(np.concatenate([rec1[i], rec2[i]]), ref[i][1]), i
    g.close()
    for s in members:
        s.close()
