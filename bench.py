#!/usr/bin/env python
"""Throughput of the DGTD stage path: DOF-updates/s of the weight-adjusted
PML nodal DGTD solver on a synthetic jittered-tetrahedron cube.

One bench step = one full low-storage Runge-Kutta time step (five stages of
the fused right-hand-side + update kernels for both element classes, probe
readout) over the whole workload.  Default workload: 40^3 x 6 = 384,000
jittered tets (+-0.2 h, seed 1), N = 4 (35 nodes), cubic PML (sigma_max 40,
shell 0.2), one dipole and eight probes, FP32 state and arithmetic.

DOF-updates per step = N_p * (6 K + 6 K_pml) * n_batch (all 12 fields of PML
elements, 6 elsewhere), the counting used for the paper's Table I.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank advances its own replica of the workload (replicas
only: the excitations are independent, there is no exchange between ranks).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402



# DRAM traffic per PML element of the tensor-core PML stage kernel, from
# one ncu capture of the small case of the benchmark recipe, valid only for
# the kernel source it was taken on (sha256 of that source file): None until
# a capture of the current source is recorded here
TC_PML_TRAFFIC = {"file": "tc_rows.cu",
                  "sha256": "56e560a33ee57d61047589a4009f0935ad16f49322d2d55378a0debb361e830e",
                  "N": 4, "bytes_per_pml_element": {"tf32": 6344.2, "bf16": 6346.0}}


def tc_pml_traffic(K1, N, precision):
    """Per-launch DRAM bytes of the PML kernel, or None once the kernel changed."""
    import hashlib
    if not TC_PML_TRAFFIC["sha256"]:
        return None
    src = os.path.join(ROOT, "paper_2006_02551_gb300", "csrc", TC_PML_TRAFFIC["file"])
    try:
        with open(src, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    per = TC_PML_TRAFFIC["bytes_per_pml_element"].get(precision)
    if h != TC_PML_TRAFFIC["sha256"] or N != TC_PML_TRAFFIC["N"] or per is None:
        return None
    return per * K1


def describe(w):
    return (f"{w.name}: {w.n_hex}^3x6={w.K} jittered tets (+-{w.jitter}h, seed {w.mesh_seed}), "
            f"N={w.N}, cubic PML sigma_max={w.pml.sigma_max} shell {w.pml.L} "
            f"(u0={w.pml.u0}), kappa_max={w.pml.kappa_max}, {len(w.sources)} dipole(s), "
            f"{len(w.probes)} probes, {w.n_batch} excitation(s)")


def algorithmic_costs(N, Np, Nfp, Nq, rs, kappa, rows=False):
    """Per element per stage launch: (bytes, flops) of the non-PML and the PML
    stage kernel (minimum traffic: each field read and written once).  Per
    element: the fields (read q, res; write res, q; and P, its register in
    PML elements), the metric (double; float in the row-owned tensor-core
    kernel), normals and Fscale (4 x 4 Real), material (3 Real), neighbour
    ids and face codes (4 x 4 + 4 bytes), and the coefficient samples (3 per
    quadrature point; the row-owned kernel reads its capacity)."""
    meta = 9 * 8 + 3 * rs + 4 * 4 + 4 + 16 * rs
    meta_rows = 9 * 4 + 3 * rs + 4 * 4 + 4 + 16 * rs
    b_std = 4 * rs * 6 * Np + meta              # read q, res; write res, q
    b_pml = 4 * rs * 12 * Np + (meta_rows if rows else meta) + (6 if kappa else 3) * Nq * rs
    f_std = 36 * Np * Np + 90 * Np + 240 * Nfp + 48 * Np * Nfp + 4 * 6 * Np
    f_pml = f_std + 48 * Nq * Np + 24 * Nq + 12 * Np + 4 * 6 * Np
    if kappa:
        f_pml += 24 * Nq * Np + 6 * Nq
    return dict(bytes_std=b_std, bytes_pml=b_pml, flops_std=f_std, flops_pml=f_pml)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def setup_solver(w, precision, stream, device, scheme="waa", rule="compact"):
    """rule: "compact" (the fully symmetric degree-2N rule of synthetic/,
    46 points at N = 4) or "default" (the library's (N+1)^3-point rule)."""
    from paper_2006_02551_gb300 import Solver
    from synthetic import compact_rule, cube_tet_mesh
    v, e = cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed)
    s = Solver(w.N, precision, n_batch=w.n_batch, device=device, stream=stream)
    if rule == "compact":
        s.set_quadrature(compact_rule(w.N))
    s.set_mesh(v, e)
    s.set_pml(w.pml, scheme)
    s.set_sources(list(w.sources))
    s.set_probes(list(w.probes))
    s.set_state(None, 0.0)
    return s


def oracle_rate(w, n_hex, steps, warmup=1, rule="compact"):
    """The FP64 oracle (as it stands) on a smaller cube of the same recipe:
    DOF-updates/s over `steps` LSERK steps after `warmup` steps."""
    from dataclasses import replace
    from oracle.solver import Simulation
    from synthetic import compact_rule, cube_tet_mesh
    ws = replace(w, n_hex=n_hex)
    v, e = cube_tet_mesh(ws.n_hex, ws.jitter, ws.mesh_seed)
    sim = Simulation(ws.N, v, e, profile=ws.pml, sources=ws.sources, probes=ws.probes,
                     n_batch=ws.n_batch,
                     volume_rule=compact_rule(ws.N) if rule == "compact" else None)
    dt = sim.stable_dt(1.0)
    st = sim.zero_state()
    t = 0.0
    if warmup:
        st, t, _, _ = sim.run(st, warmup, dt, t=t)
    # the oracle carries the PML fields on every element; count DOFs the same
    # way as the library (12 fields on PML-class elements, 6 elsewhere)
    vv = v[e]
    pml = np.any(np.abs(vv) > ws.pml.u0, axis=(1, 2))
    dofs = sim.Np * (6 * ws.K + 6 * int(pml.sum())) * ws.n_batch
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        st, t, _, _ = sim.run(st, 1, dt, t=t)
        times.append(time.perf_counter() - t0)
    return dofs, times, ws


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, w):
    dofs, times, ws = oracle_rate(w, args.ref_hex, args.steps, warmup=args.warmup, rule=args.rule)
    tot = sum(times)
    value = dofs * len(times) / tot
    sample = (f"FP64 numpy oracle on {ws.n_hex}^3x6={ws.K} tets of the same recipe "
              f"(N={ws.N}, same PML, sources, probes), {len(times)} steps after "
              f"{args.warmup} warm-up steps")
    line = {"impl": "reference", "metric": args.metric, "value": value,
            "unit": "DOF-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(w), "sample": sample},
            "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": cpu_cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def job_time_max(t_local, dist, device):
    """Replicas only: the job ends when its slowest rank does, so every rank
    takes the maximum of the ranks' times (t_local unchanged without dist)."""
    if dist is None:
        return t_local
    import torch
    tt = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(units_per_rank, world, t_max):
    """Units all ranks processed per unit of the slowest rank's time."""
    return world * units_per_rank / t_max


def mesh_dofs(s):
    i = s.info()
    return i["Np"] * 6 * (i["K"] + i["K_pml"]) * s.n_batch


def group_vs_sequential(meshes, pml, sh, local, stream, nst, precision="fp32", rule="default"):
    """The meshes [(n_hex, N)] advanced one after the other (run_steps each)
    and together (per stage one grouped launch per (order, element class)
    variant, on parallel graph branches; autotuned): DOF-updates/s."""
    import torch
    from paper_2006_02551_gb300 import Group, Solver
    from synthetic import compact_rule, cube_tet_mesh
    ss = []
    for n, N in meshes:
        v, e = cube_tet_mesh(n, 0.2, 100 + n)
        s = Solver(N, precision, device=local, stream=sh)
        if rule == "compact":
            s.set_quadrature(compact_rule(N))
        s.set_mesh(v, e)
        s.set_pml(pml)
        s.set_state(None, 0.0)
        ss.append(s)
    dts = [s.stable_dt(1.0) for s in ss]
    dofs = sum(mesh_dofs(s) for s in ss)
    k_pml = [s.info()["K_pml"] for s in ss]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for s, dt in zip(ss, dts):
        s.run_steps(2, dt, record=False)
    ev[0].record(stream)
    for s, dt in zip(ss, dts):
        s.run_steps(nst, dt, record=False)
    ev[1].record(stream)
    ev[1].synchronize()
    seq = ev[0].elapsed_time(ev[1]) / nst
    g = Group(ss)
    g.autotune(dts, reps=20)
    for s in ss:
        s.set_state(None, 0.0)
    g.run_steps(2, dts, record=False)
    ev[2].record(stream)
    g.run_steps(nst, dts, record=False)
    ev[3].record(stream)
    ev[3].synchronize()
    grp = ev[2].elapsed_time(ev[3]) / nst
    info = g.info()
    variants = info["variants"]
    g.close()
    for s in ss:
        s.close()
    return {"meshes": len(meshes), "dofs_per_step": dofs,
            "sequential": {"ms_per_step": seq, "value": dofs / (seq * 1e-3),
                           "launches_per_step": 5 * sum(1 + (s_k > 0) for s_k in k_pml)},
            "grouped": {"ms_per_step": grp, "value": dofs / (grp * 1e-3),
                        "launches_per_step": 5 * variants, "variants": variants,
                        "autotuned": info}}


def batching_runs(sh, local, stream):
    """The batching form: 64 independent excitations on one 162,000-tet N=3
    mesh (FP32, one launch per class and stage), and meshes of uneven size and
    order advanced as one group against one launch sequence per mesh (FP32,
    and the mixed set also as TF32 tensor-core contexts)."""
    import torch
    from synthetic import workload
    w = workload("cube30_n3_batch64")
    s = setup_solver(w, "fp32", sh, local)
    dt = s.stable_dt(1.0)
    s.run_steps(1, dt, record=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nst = 3
    e0.record(stream)
    s.run_steps(nst, dt, record=False)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / nst
    dofs = mesh_dofs(s)
    s.close()
    out = {"excitations": {"workload": describe(w), "precision": "fp32", "ms_per_step": ms,
                           "value": dofs / (ms * 1e-3), "unit": "DOF-updates/s"}}
    mixed = [(8 + round(16 * i / 15), 2 + (i % 3)) for i in range(16)]
    out["mixed_meshes"] = dict(
        recipe="16 meshes n^3 x 6 tets, n = 8 + round(16 i/15), N = 2 + (i mod 3), jitter 0.2h, "
               "PML as the benchmark workload, FP32",
        **group_vs_sequential(mixed, w.pml, sh, local, stream, 20))
    out["mixed_meshes_tf32"] = dict(
        recipe="the same 16 meshes as TF32 tensor-core contexts with the compact rule "
               "(grouped: per-item launches)",
        **group_vs_sequential(mixed, w.pml, sh, local, stream, 20, "tf32", "compact"))
    small = [(4 + (i % 3), 2 + (i % 3)) for i in range(48)]
    out["small_meshes"] = dict(
        recipe="48 meshes n^3 x 6 tets, n = 4 + (i mod 3), N = 2 + (i mod 3), FP32",
        **group_vs_sequential(small, w.pml, sh, local, stream, 20))
    return out


def precision_form_run(sh, local, stream):
    """The precision form: 64^3 x 6 = 1,572,864 tets, N = 5, compact volume
    rule, the contractions on the tensor cores with TF32 or BF16 operands and
    FP32 accumulation and state, against the FP32 CUDA-core path (itself
    within 1.3e-7 of FP64): DOF-updates/s of each and the relative L2
    difference of E, H after 20 steps."""
    import torch
    from paper_2006_02551_gb300 import Solver
    from synthetic import cube_tet_mesh, workload
    from synthetic import compact_rule
    w = workload("cube64_n5")
    v, e = cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed)
    out = {"workload": describe(w), "volume_rule": f"compact degree-10 rule, "
                                                   f"{compact_rule(w.N).shape[0]} points"}
    states = {}
    for prec, nrate in (("tf32", 20), ("bf16", 20), ("fp32", 10)):
        s = Solver(w.N, prec, device=local, stream=sh)
        s.set_quadrature(compact_rule(w.N))
        s.set_mesh(v, e)
        s.set_pml(w.pml)
        s.set_sources(list(w.sources))
        s.set_probes(list(w.probes))
        dt = s.stable_dt(1.0)
        s.set_state(None, 0.0)
        s.run_steps(2, dt, record=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.run_steps(nrate, dt, record=False)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / nrate
        dofs = mesh_dofs(s)
        s.set_state(None, 0.0)
        s.run_steps(20, dt, record=False)
        q, _ = s.get_state()
        states[prec] = np.array(q[:, :, 0:6], dtype=np.float32)   # FP32 state either way
        del q
        out[prec] = {"ms_per_step": ms, "value": dofs / (ms * 1e-3), "unit": "DOF-updates/s"}
        s.close()
    out["dofs_per_step"] = dofs
    for prec in ("tf32", "bf16"):
        out[f"l2_rel_{prec}_vs_fp32_20_steps"] = float(
            np.linalg.norm(states[prec] - states["fp32"]) / np.linalg.norm(states["fp32"]))
    return out


def gradient_run(sh, local, stream, rule, steps=None, ckpt=45):
    """The differentiation form: J = sum over 8 probes and 2000 steps of |E|^2 on
    the 82,944-tet N=3 mesh with eps_r ~ U[1,4]; gradient with respect to every
    eps_r and the PML (sigma_max, p_sigma) by the FP32 discrete adjoint with a
    checkpoint every 45 steps, against the forward run alone (both on the
    same volume rule)."""
    import torch
    from paper_2006_02551_gb300 import Solver
    from synthetic import compact_rule, cube_tet_mesh, workload
    from synthetic.workloads import eps_r
    w = workload("cube24_n3_grad")
    v, e = cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed)
    s = Solver(w.N, "fp32", device=local, stream=sh)
    if rule == "compact":
        s.set_quadrature(compact_rule(w.N))
    s.set_mesh(v, e)
    s.set_materials(eps_r(w))
    s.set_pml(w.pml)
    s.set_sources(list(w.sources))
    s.set_probes(list(w.probes))
    dt = s.stable_dt(1.0)
    s.set_state(None, 0.0)
    s.run_steps(5, dt)
    torch.cuda.synchronize()
    nst = steps or w.steps
    s.set_state(None, 0.0)
    t0 = time.perf_counter()
    s.run_steps(nst, dt)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    s.set_state(None, 0.0)
    t0 = time.perf_counter()
    J, ge, gs, gp = s.adjoint(nst, dt, ckpt_every=ckpt)
    t_adj = time.perf_counter() - t0
    s.close()
    return {"workload": describe(w) + ", eps_r ~ U[1,4] (seed 5)", "steps": nst,
            "volume_rule": rule, "ckpt_every": ckpt, "precision": "fp32", "forward_s": t_fwd,
            "gradient_s": t_adj, "gradient_over_forward": t_adj / t_fwd,
            "J": float(J[0]), "parameters": int(ge.shape[1]) + 6}


def t_end_accuracy(w, precision, sh, local, rule):
    """E, H at the workload's final time (its full step count) and the probe
    records of the whole run, mixed precision against the FP32 path (which
    `bench.py --accuracy` finds within 1e-6 of the FP64 path there); the
    states are compared on the device."""
    import torch
    out = {"steps": w.steps, "reference": "fp32 path on the GPU (within 1e-6 of fp64 at t_end)"}
    res = {}
    for prec in (precision, "fp32"):
        s = setup_solver(w, prec, sh, local, rule=rule)
        dt = s.stable_dt(1.0)
        s.set_state(None, 0.0)
        rec = s.run_steps(w.steps, dt)
        q = torch.empty(s.state_shape(), dtype=torch.float64, device=f"cuda:{local}")
        s.get_state(q)
        s.synchronize()
        res[prec] = (q[:, :, 0:6].contiguous(), rec, s.objective()[0])
        s.close()
        del q
    (qa, ra, Ja), (qb, rb, Jb) = res[precision], res["fp32"]
    out[f"l2_rel_{precision}_vs_fp32"] = {
        "state": float(torch.linalg.vector_norm(qa - qb) / torch.linalg.vector_norm(qb)),
        "probes": float(np.linalg.norm(ra - rb) / np.linalg.norm(rb)),
        "objective": float(abs(Ja - Jb) / abs(Jb))}
    del res, qa, qb
    torch.cuda.empty_cache()
    return out


def accuracy_runs(sh, local, rule):
    """Relative L2 error of E, H (all elements) and of the probe records at
    each workload's final time (its full step count), mixed precision against
    the FP64 GPU path (parity-proven against the oracle to 1e-12), or against
    the FP32 path where FP64 at full size takes hours (the N = 5 workload; the
    FP32 path is within ~1e-7 of FP64 at N = 4).  States are compared on the
    device (state exchange into CUDA tensors)."""
    import torch
    from paper_2006_02551_gb300 import Solver
    from synthetic import Dipole, compact_rule, cube_tet_mesh, workload
    from synthetic.workloads import eps_r

    def run(w, prec, steps, sources=None, n_batch=None, eps=None):
        v, e = cube_tet_mesh(w.n_hex, w.jitter, w.mesh_seed)
        nb = n_batch or w.n_batch
        s = Solver(w.N, prec, n_batch=nb, device=local, stream=sh)
        if rule == "compact":
            s.set_quadrature(compact_rule(w.N))
        s.set_mesh(v, e)
        if eps is not None:
            s.set_materials(eps)
        s.set_pml(w.pml)
        s.set_sources(list(sources if sources is not None else w.sources))
        s.set_probes(list(w.probes))
        dt = s.stable_dt(1.0)
        s.set_state(None, 0.0)
        t0 = time.perf_counter()
        rec = s.run_steps(steps, dt)
        wall = time.perf_counter() - t0
        q = torch.empty(s.state_shape(), dtype=torch.float64, device=f"cuda:{local}")
        s.get_state(q)
        s.synchronize()
        J = s.objective()
        s.close()
        return q[:, :, 0:6].contiguous(), rec, J, wall

    def rel(a, b):
        if isinstance(a, np.ndarray):
            return float(np.linalg.norm(a - b) / np.linalg.norm(b))
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    out = {"rule": rule}
    # N = 4 production workload: 1000 steps
    w = workload("cube40_n4")
    q64, r64, J64, t64 = run(w, "fp64", w.steps)
    row = {"steps": w.steps, "reference": "fp64 (GPU)", "fp64_wall_s": t64}
    for prec in ("fp32", "tf32", "bf16"):
        q, r, J, _ = run(w, prec, w.steps)
        row[prec] = {"state": rel(q, q64), "probes": rel(r, r64), "objective": abs(J[0] - J64[0]) / J64[0]}
        del q
    del q64
    out["cube40_n4"] = row
    torch.cuda.empty_cache()
    # N = 5 precision workload: 500 steps against FP32
    w = workload("cube64_n5")
    q32, r32, J32, t32 = run(w, "fp32", w.steps)
    row = {"steps": w.steps, "reference": "fp32 (GPU; FP64 at this size takes hours)",
           "fp32_wall_s": t32}
    for prec in ("tf32", "bf16"):
        q, r, J, _ = run(w, prec, w.steps)
        row[prec] = {"state": rel(q, q32), "probes": rel(r, r32), "objective": abs(J[0] - J32[0]) / J32[0]}
        del q
    del q32
    out["cube64_n5"] = row
    torch.cuda.empty_cache()
    # batching workload: 800 steps of the 64-excitation FP32 batch; its first
    # two excitations against an FP64 run of those two alone
    w = workload("cube30_n3_batch64")
    qb, rb, Jb, _ = run(w, "fp32", w.steps)
    two = [Dipole(x=d.x, dir=d.dir, t0=d.t0, width=d.width, amplitude=d.amplitude, batch=d.batch)
           for d in w.sources if d.batch < 2]
    q2, r2, J2, t2 = run(w, "fp64", w.steps, sources=two, n_batch=2)
    out["cube30_n3_batch64"] = {
        "steps": w.steps, "reference": "fp64 (GPU) runs of excitations 0 and 1",
        "fp32": {"state": rel(qb[:2], q2), "probes": rel(rb[..., :2], r2),
                 "objective": float(np.max(np.abs(Jb[:2] - J2) / J2))}}
    del qb, q2
    torch.cuda.empty_cache()
    # differentiation workload: 2000 steps, FP32 forward against FP64
    w = workload("cube24_n3_grad")
    er = eps_r(w)
    q64, r64, J64, _ = run(w, "fp64", w.steps, eps=er)
    q32, r32, J32, _ = run(w, "fp32", w.steps, eps=er)
    out["cube24_n3_grad"] = {"steps": w.steps, "reference": "fp64 (GPU)",
                             "fp32": {"state": rel(q32, q64), "probes": rel(r32, r64),
                                      "objective": abs(J32[0] - J64[0]) / J64[0]}}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube40_n4")
    ap.add_argument("--precision", default="tf32", choices=["fp32", "fp64", "tf32", "bf16"])
    ap.add_argument("--rule", default="compact", choices=["compact", "default"],
                    help="volume quadrature of the PML terms: the compact degree-2N rule "
                         "(46 points at N = 4) or the (N+1)^3-point conical rule")
    ap.add_argument("--hex", type=int, default=None,
                    help="override the cube size of the workload (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-stored", action="store_true",
                    help="skip the stored-matrix scheme comparison run")
    ap.add_argument("--no-batching", action="store_true",
                    help="skip the batching-form runs (excitation batch, grouped meshes)")
    ap.add_argument("--no-gradient", action="store_true",
                    help="skip the differentiation-form run (FP32 adjoint)")
    ap.add_argument("--no-precision-form", action="store_true",
                    help="skip the N = 5 precision-form run (BF16 vs FP32)")
    ap.add_argument("--ref-hex", type=int, default=4,
                    help="cube size of the oracle sample for --impl reference")
    ap.add_argument("--cpu-hex", type=int, default=12,
                    help="cube size of the oracle sample for the cpu_baseline entry")
    ap.add_argument("--grad-steps", type=int, default=None,
                    help="steps of the gradient block (default: the workload's 2000; fewer "
                         "for a profiling capture)")
    ap.add_argument("--grad-ckpt", type=int, default=45,
                    help="checkpoint spacing of the gradient block")
    ap.add_argument("--no-t-end", action="store_true",
                    help="skip the final-time accuracy block (workload's full step count)")
    ap.add_argument("--accuracy", action="store_true",
                    help="only the L2 errors at every workload's final time (about 15 "
                         "minutes: the FP64 references), one JSON line")
    args = ap.parse_args()
    args.metric = "DOF-updates/s (WADG-PML DGTD, N=4), mixed-precision vs FP64 at stated L2 error"
    if args.warmup < 3:
        args.warmup = 3

    from synthetic import workload
    w = workload(args.workload)
    if args.hex:
        from dataclasses import replace as _replace
        w = workload(args.workload, n_hex=args.hex)
        if args.hex != workload(args.workload).n_hex:
            w = _replace(w, name=f"{w.name} resized to {args.hex}^3 cells")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, w)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2006_02551_gb300 import build as _b
    if rank == 0 or world == 1:
        _b.build()
    if dist:
        dist.barrier()
    stream = torch.cuda.Stream(device=local)
    sh = stream.cuda_stream
    if args.accuracy:
        if rank == 0:
            print(json.dumps({"accuracy_at_t_end": accuracy_runs(sh, local, args.rule)}))
        return

    s = setup_solver(w, args.precision, sh, local, rule=args.rule)
    info = s.info()
    K, K1, Np, Nq = info["K"], info["K_pml"], info["Np"], info["Nq"]
    N = w.N
    Nfp = (N + 1) * (N + 2) // 2
    dofs = Np * (6 * K + 6 * K1) * w.n_batch
    dt = s.stable_dt(1.0)
    rs = 8 if args.precision == "fp64" else 4

    # warm-up (graph capture happens here)
    s.run_steps(args.warmup, dt, record=False)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.run_steps(args.steps, dt, record=False)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    dev = f"cuda:{local}" if dist is not None and dist.get_backend() == "nccl" else "cpu"
    ms = job_time_max(ev0.elapsed_time(ev1), dist, dev)
    value = whole_job_rate(dofs * args.steps, world, ms * 1e-3)

    # per-kernel durations (CUDA events on the library stream, eager launches)
    kms = s.profile_stage(50, dt)
    rows = args.precision in ("tf32", "bf16") and args.rule == "compact"
    mem0 = s.memory_report()
    # coefficient samples per element as stored (the kernels read the stored
    # stride, which includes a compact rule's padding to its capacity)
    nq_read = mem0["pml_coeff"] / max(1, K1 * 3 * rs) if K1 else Nq
    cost = algorithmic_costs(N, Np, Nfp, nq_read, rs, w.pml.kappa_max != 1.0, rows=rows)
    per = {"std": (kms[0], cost["bytes_std"] * (K - K1) * w.n_batch,
                   cost["flops_std"] * (K - K1) * w.n_batch),
           "pml": (kms[1], cost["bytes_pml"] * K1 * w.n_batch,
                   cost["flops_pml"] * K1 * w.n_batch)}
    dom = max(per, key=lambda k: per[k][0])
    d_ms, d_bytes, d_flops = per[dom]
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved = d_flops / (d_ms * 1e-3) / 1e12
    achieved_gbs = d_bytes / (d_ms * 1e-3) / 1e9
    if args.precision in ("tf32", "bf16"):
        # tensor-core contractions: the stage is bound by HBM traffic
        traffic = (tc_pml_traffic(K1 * w.n_batch, N, args.precision)
                   if dom == "pml" and rows else None)
        kname = "tc_rows_kernel" if (rows and dom == "pml") else "tc_stage_kernel"
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                    "frac": achieved_gbs / hbm, "traffic": traffic,
                    "traffic_note": "ncu DRAM bytes per PML element of the 24^3 case (mean "
                                    "of two launches), scaled by the PML elements of this "
                                    "launch; null when the kernel source has changed since",
                    "kernel": f"{kname}<{dom}>",
                    "peak_source": f"{hbm_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "alu": {"achieved_tflops": achieved}}
    else:
        from paper_2006_02551_gb300.wadg import fma_peak
        peak = fma_peak(local, fp64=args.precision == "fp64")
        peak_note = (f"measured {'FP64' if args.precision == 'fp64' else 'FP32'} FMA "
                     f"throughput (wadg_fma_peak: register FMA chains on every SM)")
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None, "kernel": f"stage_kernel<{dom}>",
                    "peak_source": peak_note,
                    "hbm": {"achieved_gbs": achieved_gbs, "peak_gbs": hbm,
                            "frac": achieved_gbs / hbm}}
    roofline.update({"kernel_ms": {"std": kms[0], "pml": kms[1]},
                     "bytes_per_launch": d_bytes, "flops_per_launch": d_flops})

    # end to end through the public API with host buffers
    rec_bytes = len(w.probes) * 6 * w.n_batch * 8
    q_host = np.zeros((w.n_batch, K, 12, Np))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    s.set_state(q_host, 0.0)
    s.run_steps(args.steps, dt, record=True)
    t1 = time.perf_counter()
    e2e_val = whole_job_rate(dofs * args.steps, world, job_time_max(t1 - t0, dist, dev))
    h2d = (w.n_batch * (K + K1) * 6 * Np * rs) / args.steps
    e2e = {"value": e2e_val, "unit": "DOF-updates/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": rec_bytes}

    mem = s.memory_report()
    out_extra = {}
    # accuracy against the FP64 path over the same steps, and the other rates
    if not args.no_fp64 and rank == 0:
        nst = 20
        s.set_state(None, 0.0)
        s.run_steps(nst, dt, record=False)
        q_main, _ = s.get_state()
        s.close()
        others = {}
        for prec in ("fp64", "fp32", "bf16"):
            if prec == args.precision or (prec == "bf16" and N > 4):
                continue
            so = setup_solver(w, prec, sh, local, rule=args.rule)
            nrate = 20 if prec == "fp64" else 200
            so.run_steps(3, dt, record=False)
            so.set_state(None, 0.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            so.run_steps(nrate, dt, record=False)
            e1.record(stream)
            e1.synchronize()
            mso = e0.elapsed_time(e1) / nrate
            so.set_state(None, 0.0)
            so.run_steps(nst, dt, record=False)
            qo, _ = so.get_state()
            so.close()
            others[prec] = ({"value": dofs / (mso * 1e-3), "ms_per_step": mso}, qo)
        sel = (slice(None), slice(None), slice(0, 6))
        if "fp64" in others:
            q64 = others["fp64"][1]
            acc = {"fields": "E,H", "steps": nst, "reference": "FP64 path on the GPU",
                   f"l2_rel_{args.precision}_vs_fp64":
                       float(np.linalg.norm(q_main[sel] - q64[sel]) / np.linalg.norm(q64[sel]))}
            for prec in ("fp32", "bf16"):
                if prec in others:
                    qo = others[prec][1]
                    acc[f"l2_rel_{prec}_vs_fp64"] = float(np.linalg.norm(qo[sel] - q64[sel]) /
                                                          np.linalg.norm(q64[sel]))
            out_extra["accuracy"] = acc
        for prec, (rate, _) in others.items():
            out_extra[prec] = rate
        if args.precision in ("tf32", "bf16") and not args.no_t_end:
            out_extra["accuracy_t_end"] = t_end_accuracy(w, args.precision, sh, local, args.rule)
        # the CUDA-core paths against the measured FMA throughput (the
        # algorithmic flops of a step: 5 stages of both classes)
        from paper_2006_02551_gb300.wadg import fma_peak
        peaks_fma = {"fp32": fma_peak(local, fp64=False), "fp64": fma_peak(local, fp64=True)}
        out_extra["cuda_core_peaks_tflops"] = peaks_fma
        for prec in ("fp32", "fp64"):
            if prec in out_extra:
                c2 = algorithmic_costs(N, Np, Nfp, Nq, 8 if prec == "fp64" else 4,
                                       w.pml.kappa_max != 1.0)
                fl = 5 * (c2["flops_std"] * (K - K1) + c2["flops_pml"] * K1) * w.n_batch
                ach = fl / (out_extra[prec]["ms_per_step"] * 1e-3) / 1e12
                out_extra[prec]["alu"] = {"achieved_tflops": ach, "peak_tflops": peaks_fma[prec],
                                          "frac": ach / peaks_fma[prec],
                                          "peak_source": "measured FMA throughput"}
    else:
        s.close()

    # the stored-matrix scheme (eqs. 10-13) on the same workload: FP32 state,
    # CUDA-core PML kernel reading 9 N_p^2 operator values per PML element
    if not args.no_stored and rank == 0 and w.pml.kappa_max == 1.0:
        t0s = time.perf_counter()
        ss = setup_solver(w, "fp32", sh, local, scheme="stored")
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0s
        nrate = 50
        ss.run_steps(3, dt, record=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ss.run_steps(nrate, dt, record=False)
        e1.record(stream)
        e1.synchronize()
        mss = e0.elapsed_time(e1) / nrate
        kss = ss.profile_stage(10, dt)
        mems = ss.memory_report()
        ss.close()
        NpP = (Np + 3) & ~3
        field_b = 4 * 4 * 12 * Np + 9 * 8 + 4 * 3 + 16
        sb = K1 * w.n_batch * field_b + mems["pml_coeff"] * w.n_batch
        out_extra["stored_scheme"] = {
            "value": dofs / (mss * 1e-3), "unit": "DOF-updates/s", "ms_per_step": mss,
            "precision": "fp32", "kernel_ms": {"std": kss[0], "pml": kss[1]},
            "pml_coeff_bytes": mems["pml_coeff"],
            "pml_coeff_bytes_per_pml_element": mems["pml_coeff"] / max(K1, 1),
            "operators_per_pml_element": f"9 x {Np} x {NpP} (kappa = 1)",
            "setup_s": setup_s,
            "pml_kernel_hbm": {"bytes_per_launch": sb, "achieved_gbs": sb / (kss[1] * 1e-3) / 1e9,
                               "peak_gbs": hbm, "frac": sb / (kss[1] * 1e-3) / 1e9 / hbm},
            "vs_waa": {"memory_ratio": mems["pml_coeff"] / max(mem["pml_coeff"], 1),
                       "time_ratio_vs_this_run": mss / (ms / args.steps),
                       "this_run_precision": args.precision,
                       # the same arithmetic on both sides: FP32 CUDA-core
                       # kernels, stored matrices against weight-adjusted
                       "time_ratio_fp32_vs_fp32": (mss / out_extra["fp32"]["ms_per_step"]
                                                   if "fp32" in out_extra else None)}}

    if not args.no_batching and rank == 0:
        out_extra["batching"] = batching_runs(sh, local, stream)
    if not args.no_gradient and rank == 0:
        out_extra["gradient"] = gradient_run(sh, local, stream, args.rule, args.grad_steps, args.grad_ckpt)
    if not args.no_precision_form and rank == 0:
        out_extra["precision_form"] = precision_form_run(sh, local, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cdofs, ctimes, ws = oracle_rate(w, args.cpu_hex, 2, warmup=1, rule=args.rule)
        cpu = {"value": cdofs * len(ctimes) / sum(ctimes), "unit": "DOF-updates/s",
               "cores": cpu_cores(), "kind": "oracle",
               "sample": (f"FP64 numpy oracle on {ws.n_hex}^3x6={ws.K} tets of the same "
                          f"recipe (N={ws.N}, same PML/source/probes), 2 steps after 1 "
                          f"warm-up step")}

    launches_per_step = 5 * (1 + (1 if K1 else 0)) + (1 if len(w.probes) else 0) + 1
    if rank == 0:
        line = {"metric": args.metric, "value": value, "unit": "DOF-updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp64": "f64", "tf32": "tf32 x tf32 -> f32",
                          "bf16": "bf16 x bf16 -> f32"}[args.precision],
                "data": "synthetic",
                "config": {"workload": describe(w), "K": K, "K_pml": K1, "N": N, "Np": Np,
                           "Nq": Nq, "volume_rule": (f"compact fully symmetric degree-{2 * N} "
                                                     f"rule, {Nq} points" if args.rule == "compact"
                                                     else f"conical product, {Nq} points"),
                           "dofs_per_step": dofs, "precision": args.precision,
                           "l2_flush": f"inputs larger than L2 (state {mem['state'] / 1e9:.2f} GB)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches_per_step * args.steps + 1,
                "memory": {"state_bytes": mem["state"], "pml_coeff_bytes": mem["pml_coeff"],
                           "pml_coeff_bytes_per_pml_element": mem["pml_coeff"] / max(K1, 1),
                           "stored_scheme_bytes_per_pml_element": 15 * Np * Np * rs,
                           "operator_bytes": mem["operators"],
                           "geometry_bytes": mem["geometry"]}}
        line.update(out_extra)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
