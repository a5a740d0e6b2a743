"""Host-side logic of the benchmark: the algorithmic cost model behind the
roofline object, the DRAM-traffic pin, and the whole-job rate.  No GPU."""
import hashlib
import os

import pytest

import bench

N4 = dict(N=4, Np=35, Nfp=15)   # (N+1)(N+2)(N+3)/6 nodes, (N+1)(N+2)/2 per face


def test_costs_of_the_n4_workload_classes():
    """Bytes per element and stage launch at N = 4 with FP32 state: every field
    value is read (q, res) and written (res, q) once, plus the per-element
    geometry and tables, plus three sigma samples per stored quadrature slot."""
    c = bench.algorithmic_costs(**N4, Nq=48, rs=4, kappa=False, rows=True)
    fields_std = 6 * 35 * 4 * 4                     # 6 components x 35 nodes x 4 accesses x 4 B
    fields_pml = 12 * 35 * 4 * 4                    # E, H and the 6 auxiliary P components
    normals, material, tables = 16 * 4, 3 * 4, 4 * 4 + 4
    metric_double, metric_float = 9 * 8, 9 * 4
    assert c["bytes_std"] == fields_std + metric_double + normals + material + tables == 3528
    assert c["bytes_pml"] == (fields_pml + metric_float + normals + material + tables
                              + 3 * 48 * 4) == 7428
    # flops: curl (3 derivative matrices on 6 components, 2 flops per entry)
    # and LIFT dominate the non-PML class; V_q and P_q on 12 components add
    # 2 x 12 x 2 flops per (node, point) pair in the PML class
    assert c["flops_std"] == 76890
    assert c["flops_pml"] - c["flops_std"] >= 48 * 48 * 35
    assert c["flops_pml"] == 159942


def test_costs_scale_with_the_rule_and_with_kappa():
    small = bench.algorithmic_costs(**N4, Nq=48, rs=4, kappa=False)
    large = bench.algorithmic_costs(**N4, Nq=128, rs=4, kappa=False)
    # only the sigma samples and the V_q / P_q work depend on the rule
    assert large["bytes_pml"] - small["bytes_pml"] == 3 * (128 - 48) * 4
    assert large["bytes_std"] == small["bytes_std"]
    assert large["flops_pml"] - small["flops_pml"] == (48 * 35 + 24) * (128 - 48)
    kap = bench.algorithmic_costs(**N4, Nq=48, rs=4, kappa=True)
    # kappa != 1: three more samples per point (kappa_u) and the a^{-1} pass
    assert kap["bytes_pml"] - small["bytes_pml"] == 3 * 48 * 4
    assert kap["flops_pml"] > small["flops_pml"]
    # FP64 state doubles the field bytes
    d = bench.algorithmic_costs(**N4, Nq=48, rs=8, kappa=False)
    assert d["bytes_std"] - small["bytes_std"] == 6 * 35 * 4 * 4 + 3 * 4 + 16 * 4


def _with_pin(monkeypatch, sha):
    pin = dict(bench.TC_PML_TRAFFIC)
    pin["sha256"] = sha
    monkeypatch.setattr(bench, "TC_PML_TRAFFIC", pin)
    return pin


def _source_sha():
    src = os.path.join(bench.ROOT, "paper_2006_02551_gb300", "csrc", bench.TC_PML_TRAFFIC["file"])
    with open(src, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def test_traffic_is_reported_only_for_the_captured_source(monkeypatch):
    pin = _with_pin(monkeypatch, _source_sha())
    per = pin["bytes_per_pml_element"]["tf32"]
    assert bench.tc_pml_traffic(1000, 4, "tf32") == pytest.approx(per * 1000)
    assert bench.tc_pml_traffic(1000, 5, "tf32") is None      # another order
    assert bench.tc_pml_traffic(1000, 4, "fp32") is None      # no capture for it
    _with_pin(monkeypatch, "0" * 64)                          # the source changed
    assert bench.tc_pml_traffic(1000, 4, "tf32") is None
    _with_pin(monkeypatch, "")
    assert bench.tc_pml_traffic(1000, 4, "tf32") is None


def test_pinned_traffic_is_below_the_algorithmic_bytes():
    """A capture above the algorithmic bytes would mean re-reads; below them,
    part of the writes still sat in L2 when the kernel ended."""
    alg = bench.algorithmic_costs(**N4, Nq=48, rs=4, kappa=False, rows=True)["bytes_pml"]
    for prec, per in bench.TC_PML_TRAFFIC["bytes_per_pml_element"].items():
        assert 0.5 * alg < per <= alg, prec


def test_whole_job_rate_counts_every_rank():
    # units of all ranks over the slowest rank's time
    assert bench.whole_job_rate(1e9, 1, 0.5) == pytest.approx(2e9)
    assert bench.whole_job_rate(1e9, 4, 0.5) == pytest.approx(8e9)
