"""Gradient of S and backtracking of optimal paths (CPU reference).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Passage followed: the path-planning section, Eq. (PathPlanning-backTrackOnS):
an optimal path is the solution of  dx/dt = -grad S(x) / |grad S(x)|  from a
target point, stopped once |x(t) - x_0| < eps for a source x_0.  The paper
gives no discretisation; the reading used here (and by the CUDA path):

* grad S at the nodes: central differences (S[k+1] - S[k-1]) / (2h) inside,
  one-sided (S[1] - S[0]) / h and (S[n-1] - S[n-2]) / h on the faces
  (``numpy.gradient`` with edge_order=1).
* grad S between nodes: multilinear interpolation of the nodal gradient in
  the cell that holds the point (cells clamped to the grid).
* The ODE: explicit Euler steps of fixed arc length `step`,
  x_{k+1} = clamp(x_k - step * g / |g|) with g the interpolated gradient;
  before each step the path stops if its distance to the nearest source is
  below eps (status 0), or if |g| is zero or not finite (status 2); after
  max_steps steps it stops with status 1.
Coordinates are world coordinates x = i h, axes in the order (x, y[, z]).
"""
from __future__ import annotations

import numpy as np


def grad_S(S: np.ndarray, dims, h: float) -> np.ndarray:
    """Nodal gradient, shape (ndim, N): component a is dS/dx_a, flat C order
    with x fastest."""
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    A = np.asarray(S, dtype=np.float64).reshape(dims[::-1])
    out = []
    for ax in range(nd):
        out.append(np.gradient(A, h, axis=nd - 1 - ax, edge_order=1).ravel())
    return np.stack(out)


def interp(G: np.ndarray, dims, h: float, x: np.ndarray) -> np.ndarray:
    """Multilinear interpolation of the nodal field G (ndim, N) at the world
    points x (P, ndim)."""
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    P = x.shape[0]
    c = np.empty((P, nd), dtype=np.int64)
    t = np.empty((P, nd))
    for a in range(nd):
        u = x[:, a] / h
        ca = np.clip(np.floor(u), 0, dims[a] - 2).astype(np.int64)
        c[:, a] = ca
        t[:, a] = u - ca
    strides = [1]
    for a in range(1, nd):
        strides.append(strides[-1] * dims[a - 1])
    out = np.zeros((P, G.shape[0]))
    for corner in range(1 << nd):
        wgt = np.ones(P)
        idx = np.zeros(P, dtype=np.int64)
        for a in range(nd):
            bit = (corner >> a) & 1
            wgt = wgt * (t[:, a] if bit else 1.0 - t[:, a])
            idx = idx + (c[:, a] + bit) * strides[a]
        out += wgt[:, None] * G[:, idx].T
    return out


def backtrack(G: np.ndarray, dims, h: float, starts, step: float, max_steps: int,
              src_idx, eps: float):
    """Euler backtracking of every start point.  Returns (paths, lengths,
    status): paths (P, max_steps + 1, ndim) with the points x_0 .. x_len
    (the rest NaN), lengths = number of steps taken."""
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    x = np.array(starts, dtype=np.float64).reshape(-1, nd)
    P = x.shape[0]
    src = np.asarray(src_idx, dtype=np.int64).ravel()
    ys = np.empty((len(src), nd))
    rem = src.copy()
    for a in range(nd):
        ys[:, a] = (rem % dims[a]) * h
        rem //= dims[a]
    hi = np.array([(d - 1) * h for d in dims])
    paths = np.full((P, max_steps + 1, nd), np.nan)
    lengths = np.zeros(P, dtype=np.int64)
    status = np.ones(P, dtype=np.int64)
    active = np.ones(P, dtype=bool)
    paths[:, 0] = x
    for k in range(max_steps):
        if not active.any():
            break
        dist = np.sqrt(((x[:, None, :] - ys[None, :, :]) ** 2).sum(-1)).min(1)
        reached = active & (dist < eps)
        status[reached] = 0
        active &= ~reached
        g = interp(G, dims, h, x)
        gn = np.sqrt((g * g).sum(1))
        flat = active & ~(gn > 0)          # zero or not finite
        status[flat] = 2
        active &= ~flat
        idx = np.where(active)[0]
        xn = x[idx] - step * g[idx] / gn[idx, None]
        x[idx] = np.clip(xn, 0.0, hi)
        lengths[idx] += 1
        paths[idx, k + 1] = x[idx]
    # paths still active after max_steps: reached on the last point?
    if active.any():
        dist = np.sqrt(((x[:, None, :] - ys[None, :, :]) ** 2).sum(-1)).min(1)
        status[active & (dist < eps)] = 0
    return paths, lengths, status
