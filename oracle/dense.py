"""Independent dense construction of the discrete problem (small grids only).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

This builds the same finite-difference problem as ``oracle.fd`` by a
different route, node by node with explicit coordinates: the textbook
5-point (7-point in 3D) Laplacian of Sec. 6, Eq. (sparse-system), applied to
-hbar^2 Lap(phi) + f^2 phi = 0 (Sec. 4, Eq. (phiEquation)), with zero flux
imposed through mirror ghost nodes (phi at index -1 equals phi at index 1,
phi at n equals phi at n-2) and a Dirichlet row phi_k = exp(-U_k/hbar) at
every source.  The matrix is not symmetric (face rows carry doubled
couplings) and includes the source rows, so it shares neither the
symmetrisation nor the elimination of ``oracle.fd``; it is solved with a dense
LU.  For ``boundary=1`` a missing neighbour is simply dropped.
"""
from __future__ import annotations

import itertools

import numpy as np


def dense_system(f, dims, h, hbar, src_idx, src_U=None, boundary=0):
    dims = tuple(int(v) for v in dims)
    nd = len(dims)
    n = int(np.prod(dims))
    f = np.asarray(f, dtype=np.float64).ravel()
    src_idx = [int(s) for s in np.asarray(src_idx).ravel()]
    U = (np.zeros(len(src_idx)) if src_U is None
         else np.asarray(src_U, dtype=np.float64).ravel())
    val = {}
    for s, u in zip(src_idx, U):
        val[s] = u
    coef = hbar * hbar / (h * h)
    M = np.zeros((n, n))
    rhs = np.zeros(n)

    def flat(cs):
        k, stride = 0, 1
        for cc, nn in zip(cs, dims):
            k += cc * stride
            stride *= nn
        return k

    for cs in itertools.product(*[range(nn) for nn in dims[::-1]]):
        cs = tuple(reversed(cs))              # (x, y[, z])
        i = flat(cs)
        if i in val:
            M[i, i] = 1.0
            rhs[i] = np.exp(-val[i] / hbar)
            continue
        M[i, i] += f[i] * f[i]
        for ax in range(nd):
            for step in (-1, 1):
                nb = list(cs)
                nb[ax] += step
                if nb[ax] < 0 or nb[ax] > dims[ax] - 1:
                    if boundary == 1:
                        continue
                    # mirror ghost: index -1 -> 1, index n -> n-2
                    nb[ax] = 1 if nb[ax] < 0 else dims[ax] - 2
                j = flat(nb)
                M[i, i] += coef
                M[i, j] -= coef
    return M, rhs


def dense_solve(f, dims, h, hbar, src_idx, src_U=None, boundary=0):
    """phi on the full grid (unshifted) and S = -hbar log(phi)."""
    M, rhs = dense_system(f, dims, h, hbar, src_idx, src_U, boundary)
    phi = np.linalg.solve(M, rhs)
    return phi, -hbar * np.log(phi)
