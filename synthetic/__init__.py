"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only *generates* inputs: vertex coordinates and tetrahedron
connectivity of jittered cube meshes, dipole sources, probe positions and the
workload definitions.  It contains none of the DGTD method's arithmetic (no
basis, no operators, no geometric factors, no PML coefficients); each side of
the parity comparison computes those on its own.
"""
from .mesh import cube_tet_mesh
from .workloads import (Dipole, PmlProfile, Workload, WORKLOADS, workload,
                        random_dipoles)

__all__ = ["cube_tet_mesh", "Dipole", "PmlProfile", "Workload", "WORKLOADS",
           "workload", "random_dipoles"]
