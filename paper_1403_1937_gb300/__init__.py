"""GB300-native finite-difference Schroedinger-wave eikonal solver.

Solves |grad S| = f through the linear screened-Poisson equation
-hbar^2 Lap(phi) + f^2 phi = 0, phi = exp(-S/hbar) (arXiv 1403.1937, Sec. 4
and Sec. 6), with hand-written CUDA kernels for sm_103a behind the C ABI of
``include/eik.h``.

Submodules are imported lazily so that the seeded input generators
(``workloads``) can be used without loading the CUDA library:

    from paper_1403_1937_gb300 import eik        # binding (needs libeik.so)
    from paper_1403_1937_gb300 import workloads  # inputs only
"""

__all__ = ["eik", "workloads", "build"]
