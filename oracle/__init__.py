"""CPU oracle for the finite-difference Schroedinger-wave eikonal solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
anything under ``oracle/``: only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.
It shares no code with the CUDA path (no kernels, headers, helpers or
constants); the two meet only in the seeded input generators of
``paper_1403_1937_gb300.workloads``, which hold none of the method's
arithmetic.

Modules
-------
fd            assembled sparse FP64 system, direct solve, S = -hbar log phi,
              log-domain identity residual, adjoint gradient dL/df.
dense         independent dense construction of the same discrete problem
              from mirror ghost nodes (used to pin ``fd``).
closed_forms  exact 1D-reducible discrete solution, lattice Green's function
              with mirror images, continuum Green's functions.
cg            plain FP64 Jacobi-PCG on the assembled CSR matrix, in C with
              OpenMP (large grids and the timed CPU baseline).
paths         nodal gradient of S and Euler backtracking of optimal paths
              (path-planning section, Eq. PathPlanning-backTrackOnS).
sfs           shape-from-shading forcing f = sqrt(1/P^2 - 1)
              (Eq. SfS-forcingFunc).
"""
