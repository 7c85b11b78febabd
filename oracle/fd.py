"""Assembled FP64 finite-difference system and its direct solution.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What is computed (paper passages followed):

* Sec. 4, Eq. (phiEquation): for general forcing f the wave function solves
  -hbar^2 Lap(phi) + f^2 phi = 0 and S = -hbar log(phi), Eq. (SfromPhi).
* Sec. 6, Eq. (sparse-system): the Laplacian is replaced by the standard
  5-point stencil (7-point in 3D), giving a sparse block-tridiagonal system.
  The printed matrix omits the hbar^2/h^2 factor and shows f instead of f^2;
  this oracle discretises Eq. (phiEquation) itself: (hbar^2/h^2) L_h + f^2.
* Sec. 3.2, Eq. (forcedPhiEquation) and the text after it: the source points
  y_k carry known values of S (S = 0 in the paper).  Here they are Dirichlet
  nodes with phi = exp(-U_k/hbar), so S = U exactly at the sources.
* Zero-flux outer faces, second-order "half-cell" form: nodes sit on the
  faces; a node on a face of axis b owns half a cell along b.  With
  w_i = prod_b (1/2 if i is on a b-face) and, for an edge i~j along axis a,
  omega_ij = prod_{b != a} (1/2 if i is on a b-face), every non-source row is

      sum_{j~i} c*omega_ij*(phi_i - phi_j) + w_i*f_i^2*phi_i = 0,
      c = hbar^2/h^2,

  which is the mirror-ghost discretisation (phi_{-1} = phi_{1}) multiplied by
  w_i, so the matrix is symmetric.  ``boundary=1`` instead drops the missing
  neighbours with unit weights (first-order zero flux).

The unknowns are the non-source nodes; source neighbours move to the right
hand side.  The reduced matrix is a symmetric M-matrix, solved here by sparse
LU without pivoting (SuperLU, symmetric ordering).  All source values are
shifted by U_min = min_k U_k (phi is rescaled by exp(U_min/hbar)), which is an
exact rescaling of a linear problem and keeps phi <= 1.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass
class System:
    dims: tuple
    h: float
    hbar: float
    c: float
    f: np.ndarray            # flat, float64 (N,)
    w: np.ndarray            # node weights (N,)
    a: np.ndarray            # diagonal a_i = w_i f_i^2 + c sum_j omega_ij (N,)
    K: sp.csr_matrix         # full symmetric N x N operator (all nodes)
    src: np.ndarray          # unique source indices
    U: np.ndarray            # source values (aligned with src)
    U_min: float
    phiY: np.ndarray         # shifted source values exp(-(U - U_min)/hbar)
    unk: np.ndarray          # indices of the unknowns (non-source nodes)
    A: sp.csc_matrix         # K restricted to the unknowns
    b: np.ndarray            # right-hand side on the unknowns
    boundary: int

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))


def _face_weights(dims: Sequence[int], boundary: int):
    """Per-axis flat arrays h_b with 1/2 on the two b-faces (boundary 0) and
    1 elsewhere; all ones for boundary 1."""
    shape = tuple(dims[::-1])
    out = []
    for ax, n in enumerate(dims):
        v = np.ones(n)
        if boundary == 0:
            v[0] = 0.5
            v[-1] = 0.5
        # broadcast along numpy axis (ndim-1-ax)
        bshape = [1] * len(dims)
        bshape[len(dims) - 1 - ax] = n
        out.append(np.broadcast_to(v.reshape(bshape), shape).ravel().copy())
    return out


def dedup_sources(src_idx, src_U, n: int):
    """Sorted unique sources; a repeated index with two different values, or
    an index outside the grid, is an error."""
    src_idx = np.asarray(src_idx, dtype=np.int64).ravel()
    src_U = (np.zeros(len(src_idx)) if src_U is None
             else np.asarray(src_U, dtype=np.float64).ravel())
    if len(src_idx) == 0:
        raise ValueError("at least one source is required")
    if src_idx.min() < 0 or src_idx.max() >= n:
        raise ValueError("source index out of range")
    order = np.argsort(src_idx, kind="stable")
    s, u = src_idx[order], src_U[order]
    keep = np.ones(len(s), dtype=bool)
    keep[1:] = s[1:] != s[:-1]
    dup = ~keep
    if dup.any():
        first = np.maximum.accumulate(np.where(keep, np.arange(len(s)), 0))
        if np.any(u[dup] != u[first[dup]]):
            raise ValueError("duplicate source with conflicting values")
    return s[keep], u[keep]


def assemble(f, dims, h, hbar, src_idx, src_U=None, boundary: int = 0) -> System:
    """Assemble the discrete system of Eq. (phiEquation) on the grid."""
    dims = tuple(int(v) for v in dims)
    n = int(np.prod(dims))
    f = np.asarray(f, dtype=np.float64).ravel()
    if f.shape[0] != n:
        raise ValueError("f has the wrong size")
    if not np.all(np.isfinite(f)) or np.any(f <= 0):
        raise ValueError("f must be finite and positive")
    if h <= 0 or hbar <= 0:
        raise ValueError("h and hbar must be positive")
    c = hbar * hbar / (h * h)
    hw = _face_weights(dims, boundary)
    w = np.ones(n)
    for v in hw:
        w = w * v
    rows, cols, vals = [], [], []
    diag = w * f * f
    stride = 1
    idx = np.arange(n, dtype=np.int64)
    coords = np.unravel_index(idx, dims[::-1])   # (z,) y, x
    for ax, nax in enumerate(dims):
        xa = coords[len(dims) - 1 - ax]
        lo = idx[xa < nax - 1]                   # edge lo -> lo + stride
        hi = lo + stride
        om = np.ones(len(lo))
        for b, v in enumerate(hw):
            if b != ax:
                om = om * v[lo]
        wgt = c * om
        rows += [lo, hi]
        cols += [hi, lo]
        vals += [-wgt, -wgt]
        np.add.at(diag, lo, wgt)
        np.add.at(diag, hi, wgt)
        stride *= nax
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows),
                                               np.concatenate(cols))),
                      shape=(n, n))
    src, U = dedup_sources(src_idx, src_U, n)
    U_min = float(U.min())
    phiY = np.exp(-(U - U_min) / hbar)
    is_src = np.zeros(n, dtype=bool)
    is_src[src] = True
    unk = idx[~is_src]
    A = K[unk][:, unk].tocsc()
    b = -(K[unk][:, src] @ phiY)
    return System(dims, float(h), float(hbar), c, f, w, diag, K, src, U, U_min,
                  phiY, unk, A, np.asarray(b).ravel(), boundary)


def factor(sys: System):
    """Sparse LU of the reduced SPD M-matrix without pivoting."""
    return spla.splu(sys.A, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                     options=dict(SymmetricMode=True))


def full_phi(sys: System, phi_unk: np.ndarray) -> np.ndarray:
    """Scatter the unknowns and the source values into a full-grid vector."""
    phi = np.empty(sys.n, dtype=phi_unk.dtype)
    phi[sys.unk] = phi_unk
    phi[sys.src] = sys.phiY
    return phi


def solve_phi(sys: System, lu=None) -> np.ndarray:
    """Shifted wave function phi' = phi * exp(U_min/hbar) on the full grid."""
    if len(sys.unk) == 0:
        return full_phi(sys, np.zeros(0))
    lu = factor(sys) if lu is None else lu
    return full_phi(sys, lu.solve(sys.b))


def S_from_phi(sys: System, phi: np.ndarray) -> np.ndarray:
    """Eq. (SfromPhi): S = -hbar log(phi), undoing the U_min shift; exact U
    on the sources."""
    with np.errstate(divide="ignore"):       # phi = 0 (unconverged) -> inf
        S = sys.U_min - sys.hbar * np.log(phi)
    S[sys.src] = sys.U
    return S


def solve(f, dims, h, hbar, src_idx, src_U=None, boundary=0):
    """Direct solve.  Returns (S, phi_shifted, system)."""
    sys = assemble(f, dims, h, hbar, src_idx, src_U, boundary)
    phi = solve_phi(sys)
    return S_from_phi(sys, phi), phi, sys


def graph_distance(sys: System) -> np.ndarray:
    """Shortest-path distance from the sources over the grid graph with the
    axis and diagonal neighbours of every node (edge cost: Euclidean length
    times the mean of f at the two ends), plus the source values U - U_min.
    Computed with scipy's Dijkstra; used only as a scale for the relative
    solve below, never as the answer."""
    from scipy.sparse import csgraph
    dims = sys.dims
    n = sys.n
    idx = np.arange(n).reshape(dims[::-1])
    rows, cols, vals = [], [], []
    nd = len(dims)
    import itertools
    for off in itertools.product((-1, 0, 1), repeat=nd):
        if all(o == 0 for o in off) or off[::-1] < tuple([0] * nd):
            continue
        sl_a, sl_b = [], []
        for o in off:                       # numpy axis order matches off
            sl_a.append(slice(max(-o, 0), None if o <= 0 else -o))
            sl_b.append(slice(max(o, 0), None if o >= 0 else o))
        a = idx[tuple(sl_a)].ravel()
        b = idx[tuple(sl_b)].ravel()
        length = sys.h * np.sqrt(sum(o * o for o in off))
        w = length * 0.5 * (sys.f[a] + sys.f[b])
        rows += [a, b]
        cols += [b, a]
        vals += [w, w]
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    # a super-source joined to every source with cost U - U_min
    G = sp.bmat([[G, None], [None, sp.csr_matrix((1, 1))]], format="lil")
    for s_, u in zip(sys.src, sys.U):
        G[n, s_] = u - sys.U_min + 1e-300
    d = csgraph.dijkstra(G.tocsr(), directed=True, indices=n)
    return d[:n]


def solve_relative(sys: System, S_scale: Optional[np.ndarray] = None):
    """Direct solve of the same system in relative form, for problems whose
    phi underflows float64 (S/hbar > ~700).

    With D = diag(exp(-St/hbar)) for any finite scale St (default: the graph
    distance above), phi = D psi and the diagonally similar system
    (D^-1 A D) psi = D^-1 b has entries A_ij exp((St_i - St_j)/hbar), which
    stay O(1) between neighbours.  It is solved by sparse LU (it is no longer
    symmetric), and S = U_min + St - hbar log(psi).  In exact arithmetic this
    is the same solution as ``solve_phi``.  Returns S on the full grid."""
    St = graph_distance(sys) if S_scale is None else np.asarray(S_scale, float).ravel()
    u = sys.unk
    A = sys.A.tocoo()
    Su = St[u]
    data = A.data * np.exp((Su[A.row] - Su[A.col]) / sys.hbar)
    Ar = sp.csc_matrix((data, (A.row, A.col)), shape=A.shape)
    # b_i / D_i = sum_{k in Y} c omega_ik exp(-(U_k - U_min)/hbar + St_i/hbar)
    K = sys.K[u][:, sys.src].tocoo()
    br = np.zeros(len(u))
    np.add.at(br, K.row, -K.data * np.exp((Su[K.row] - (sys.U[K.col] - sys.U_min))
                                          / sys.hbar))
    lu = spla.splu(Ar, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0)
    psi = lu.solve(br)
    S = np.empty(sys.n)
    S[u] = sys.U_min + Su - sys.hbar * np.log(psi)
    S[sys.src] = sys.U
    return S


def componentwise_residual(sys: System, phi: np.ndarray) -> np.ndarray:
    """|r_i| / (a_i |phi_i|) on the unknowns for a full-grid phi (shifted),
    with r = b - A phi restricted to the unknowns."""
    r = -(sys.K @ phi)[sys.unk]
    return np.abs(r) / (sys.a[sys.unk] * np.abs(phi[sys.unk]))


def identity_residual(sys: System, S: np.ndarray) -> np.ndarray:
    """Log-domain form of each non-source row: dividing the row by phi_i
    gives  c sum_j omega_ij (exp((S_i - S_j)/hbar) - 1) = w_i f_i^2.
    Returns the row defect divided by a_i (equal to the componentwise
    residual of phi = exp(-S/hbar)), evaluated from S alone."""
    K = sys.K.tocoo()
    off = K.row != K.col
    i, j, kij = K.row[off], K.col[off], -K.data[off]     # kij = c*omega_ij
    lhs = np.zeros(sys.n)
    np.add.at(lhs, i, kij * np.expm1((S[i] - S[j]) / sys.hbar))
    d = (lhs - sys.w * sys.f ** 2) / sys.a
    return d[sys.unk]


def grad_f(sys: System, dLdS: np.ndarray, lu=None, phi=None):
    """Adjoint gradient dL/df for a loss L(S).

    With A(f) phi = b and A_ii = w_i f_i^2 + ..., dA/df_i = 2 w_i f_i e_i e_i^T,
    so dL/df_i = -2 w_i f_i phi_i lambda_i where A lambda = dL/dphi and
    dL/dphi = -hbar (dL/dS)/phi (from Eq. (SfromPhi)); A is symmetric, so the
    adjoint solve reuses the factorisation.  Zero on source nodes."""
    lu = factor(sys) if lu is None else lu
    if phi is None:
        phi = solve_phi(sys, lu)
    pu = phi[sys.unk]
    g = -sys.hbar * np.asarray(dLdS, dtype=np.float64).ravel()[sys.unk] / pu
    lam = lu.solve(g)
    out = np.zeros(sys.n)
    out[sys.unk] = -2.0 * sys.w[sys.unk] * sys.f[sys.unk] * lam * pu
    return out


def solve_complex(sys: System, fc: np.ndarray) -> np.ndarray:
    """Direct solve of the same system with a complex forcing field (used for
    complex-step derivatives).  Returns the complex shifted S on the grid."""
    dims = sys.dims
    n = sys.n
    fc = np.asarray(fc, dtype=np.complex128).ravel()
    # same operator with f^2 -> fc^2 on the diagonal
    K = sys.K.astype(np.complex128).tolil()
    d = sys.a - sys.w * sys.f ** 2 + sys.w * fc * fc
    K.setdiag(d)
    K = K.tocsr()
    A = K[sys.unk][:, sys.unk].tocsc()
    b = -(K[sys.unk][:, sys.src] @ sys.phiY.astype(np.complex128))
    lu = spla.splu(A, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    phi = np.empty(n, dtype=np.complex128)
    phi[sys.unk] = lu.solve(np.asarray(b).ravel())
    phi[sys.src] = sys.phiY
    S = sys.U_min - sys.hbar * np.log(phi)
    S[sys.src] = sys.U
    return S
