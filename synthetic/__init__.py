"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only *generates* inputs: vertex coordinates and tetrahedron
connectivity of jittered cube and box meshes (with the periodic vertex
identification of a box), dipole sources, probe positions, the workload
definitions and the compact volume quadrature rules (points and weights).  It contains none of the DGTD method's arithmetic (no
basis, no operators, no geometric factors, no PML coefficients); each side of
the parity comparison computes those on its own.
"""
from .mesh import box_tet_mesh, cube_tet_mesh
from .quadrature import compact_rule, compact_rule_info
from .workloads import (Dipole, PmlProfile, Workload, WORKLOADS, workload,
                        random_dipoles)

__all__ = ["box_tet_mesh", "compact_rule", "compact_rule_info", "cube_tet_mesh", "Dipole", "PmlProfile", "Workload", "WORKLOADS",
           "workload", "random_dipoles"]
