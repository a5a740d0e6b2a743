"""FP64 CPU oracle of the WAA smoothly-varying SC-PML nodal DGTD method.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of what the GPU library computes; it is imported only by the
tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``.  The product library never imports, links or calls it, and it
shares no code with the CUDA path (only the seeded input generators in
``synthetic/`` feed both sides).

Modules follow the paper's structure:

* ``refelem``  -- reference tetrahedron: orthonormal basis, nodes, M, S via
  Dr/Ds/Dt, F via LIFT (eqs. 14, 16, 17), quadrature, V_q and P_q (eqs. 20, 21)
* ``geometry`` -- affine element maps, J_k, metric terms, normals, face
  connectivity (Section II.A, nodal DG setting)
* ``pml``      -- stretching profiles (eq. 4, Section III) and the diagonal
  tensors a, b, c, d, kappa (eq. 9)
* ``maxwell``  -- curl operator with upwind flux, the WAA update equations
  (eqs. 26-29) and the stored per-element-mass-matrix update equations
  (eqs. 10-15)
* ``lserk``    -- the explicit low-storage Runge-Kutta time marching
* ``solver``   -- sources, probes, the time loop and the energy

Readings of the paper that the oracle takes where the text is silent or
garbled are stated in the docstrings where they are used.  Everything is
pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
