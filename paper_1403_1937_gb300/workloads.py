"""Seeded synthetic inputs for the screened-Poisson eikonal solve.

This module only draws inputs: forcing fields f on a vertex-centred grid,
source (seed) node indices with their prescribed values U, receiver nodes and
noise.  It holds none of the method's arithmetic, so the CPU oracle and the
CUDA path can both be fed from it without sharing any of the solve.

The paper's own workloads (maze images, vessel images, shape-from-shading
photographs, Sec. 6.2-6.4) are not available, so seeded fields with the same
structure stand in for them:

* smooth fields built from a few low-wavenumber Fourier modes (the cost maps
  of Sec. 6.1 and the two-Gaussian / sinusoidal forcings of Sec. 5.4),
* piecewise-constant fields made of axis-aligned boxes (maze-like cost maps
  with obstacles, Sec. 6.2),
* the closed-form forcing f = exp(r) of Sec. 5.4, Example 1.

Layout convention (shared by every consumer): a grid with ``dims = (n_x, n_y)``
or ``(n_x, n_y, n_z)`` stores node (i_x, i_y[, i_z]) at flat index
``i_x + n_x*(i_y + n_y*i_z)`` (x fastest, C order), node coordinates are
``x_a = i_a * h``; numpy arrays therefore have shape ``dims[::-1]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 1937


@dataclass
class Instance:
    """One solve: grid, spacing, hbar, forcing field and sources."""

    dims: Tuple[int, ...]          # (n_x, n_y) or (n_x, n_y, n_z)
    h: float
    hbar: float
    f: np.ndarray                  # float64, shape dims[::-1]
    src_idx: np.ndarray            # int64 flat node indices
    src_U: np.ndarray              # float64 prescribed S at the sources
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))

    @property
    def ndim(self) -> int:
        return len(self.dims)


def flat_index(dims: Sequence[int], coords: Sequence[int]) -> int:
    """Flat index of node ``coords`` (x first) on a grid of size ``dims``."""
    idx = 0
    stride = 1
    for n, c in zip(dims, coords):
        idx += int(c) * stride
        stride *= int(n)
    return idx


def node_coords(dims: Sequence[int], h: float):
    """Coordinate arrays (x, y[, z]) of every node, each of shape dims[::-1]."""
    axes = [np.arange(n, dtype=np.float64) * h for n in dims]
    grids = np.meshgrid(*axes[::-1], indexing="ij")   # (z,) y, x order
    return tuple(reversed(grids))                     # x, y[, z]


def _wavevectors(rng: np.random.Generator, ndim: int, count: int, kmax: int):
    """Integer wave vectors k with 1 <= |k|_2 <= kmax, drawn uniformly."""
    rngs = [np.arange(-kmax, kmax + 1)] * ndim
    cand = np.stack(np.meshgrid(*rngs, indexing="ij"), -1).reshape(-1, ndim)
    norm = np.sqrt((cand.astype(np.float64) ** 2).sum(1))
    cand = cand[(norm >= 1.0) & (norm <= kmax)]
    pick = rng.integers(0, len(cand), size=count)
    return cand[pick]


def fourier_field(rng: np.random.Generator, dims: Sequence[int], h: float,
                  modes: int = 8, kmax: int = 4, lo: float = 0.5,
                  hi: float = 1.5) -> np.ndarray:
    """Smooth positive field: ``mid + half*g`` with g a sum of ``modes``
    random Fourier modes (integer wave vectors, |k| <= kmax, N(0,1)
    amplitudes, uniform phases) min-max normalised to [-1, 1], then clipped
    to [lo, hi]."""
    ndim = len(dims)
    ks = _wavevectors(rng, ndim, modes, kmax)
    amp = rng.standard_normal(modes)
    phase = rng.uniform(0.0, 2.0 * np.pi, modes)
    xs = node_coords(dims, h)
    g = np.zeros(tuple(dims[::-1]), dtype=np.float64)
    for m in range(modes):
        arg = phase[m]
        for a in range(ndim):
            arg = arg + 2.0 * np.pi * ks[m, a] * xs[a]
        g += amp[m] * np.cos(arg)
    gmin, gmax = g.min(), g.max()
    if gmax > gmin:
        g = 2.0 * (g - gmin) / (gmax - gmin) - 1.0
    else:
        g = np.zeros_like(g)
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    return np.clip(mid + half * g, lo, hi)


def box_field(rng: np.random.Generator, dims: Sequence[int], h: float,
              nboxes: int = 32, background: float = 1.0,
              lo_max: float = 0.8, side: Tuple[float, float] = (0.05, 0.3),
              value: Tuple[float, float] = (0.5, 2.0)) -> np.ndarray:
    """Piecewise-constant field: a background plus ``nboxes`` axis-aligned
    boxes painted in order (later boxes overwrite earlier ones)."""
    ndim = len(dims)
    f = np.full(tuple(dims[::-1]), background, dtype=np.float64)
    extent = [(n - 1) * h for n in dims]
    xs = node_coords(dims, h)
    for _ in range(nboxes):
        lo = rng.uniform(0.0, lo_max, ndim)
        sd = rng.uniform(side[0], side[1], ndim)
        hi = np.minimum(lo + sd, extent)
        val = rng.uniform(value[0], value[1])
        mask = np.ones_like(f, dtype=bool)
        for a in range(ndim):
            mask &= (xs[a] >= lo[a]) & (xs[a] <= hi[a])
        f[mask] = val
    return f


def random_sources(rng: np.random.Generator, n: int, count: int) -> np.ndarray:
    """``count`` distinct uniformly random flat node indices (sorted)."""
    count = min(count, n)
    return np.sort(rng.choice(n, size=count, replace=False)).astype(np.int64)


# --------------------------------------------------------------------------
# The five benchmark workloads.  Config k draws from default_rng(1937 + k).
# --------------------------------------------------------------------------

def config1() -> Instance:
    """2D 129x129 on [0,1]^2, f = 1, one source at node (64, 64), hbar=0.01."""
    dims = (129, 129)
    f = np.ones(dims[::-1])
    src = np.array([flat_index(dims, (64, 64))], dtype=np.int64)
    return Instance(dims, 1.0 / 128, 0.01, f, src, np.zeros(1), name="c1_2d_129")


def config2(n: int = 2048, nsrc: int = 16, hbar: float = 0.005) -> Instance:
    """2D n x n (default 2048^2) on [0,1]^2, Fourier-mode f in [0.5, 1.5],
    16 uniformly random sources, hbar = 0.005."""
    rng = np.random.default_rng(SEED_BASE + 2)
    dims = (n, n)
    h = 1.0 / (n - 1)
    f = fourier_field(rng, dims, h)
    src = random_sources(rng, n * n, nsrc)
    return Instance(dims, h, hbar, f, src, np.zeros(len(src)),
                    name=f"c2_2d_{n}")


def config3(n: int = 256, nsrc: int = 4, hbar: float = 0.02) -> Instance:
    """3D n^3 (default 256^3) on [0,1]^3, background 1 plus 32 random boxes
    with values in [0.5, 2], 4 random sources, hbar = 0.02."""
    rng = np.random.default_rng(SEED_BASE + 3)
    dims = (n, n, n)
    h = 1.0 / (n - 1)
    f = box_field(rng, dims, h)
    src = random_sources(rng, n ** 3, nsrc)
    return Instance(dims, h, hbar, f, src, np.zeros(len(src)),
                    name=f"c3_3d_{n}")


def config4(count: int = 256, side: Tuple[int, int] = (64, 1024)) -> List[Instance]:
    """Batch of ``count`` independent 2D instances: sides n_x, n_y uniform in
    ``side``, h = 1/(max side - 1), Fourier f in [0.5, 1.5], 1-8 sources,
    hbar in {2h, 4h, 8h}."""
    rng = np.random.default_rng(SEED_BASE + 4)
    out = []
    for k in range(count):
        nx, ny = (int(v) for v in rng.integers(side[0], side[1] + 1, size=2))
        dims = (nx, ny)
        h = 1.0 / (max(nx, ny) - 1)
        f = fourier_field(rng, dims, h)
        nsrc = int(rng.integers(1, 9))
        src = random_sources(rng, nx * ny, nsrc)
        hbar = float(rng.choice([2.0, 4.0, 8.0])) * h
        out.append(Instance(dims, h, hbar, f, src, np.zeros(len(src)),
                            name=f"c4_{k}_{nx}x{ny}"))
    return out


def config5(count: int = 32, n: int = 512, nrecv: int = 4096,
            hbar: float = 0.01, noise: float = 0.01):
    """Differentiation batch: ``count`` 2D n x n instances with Fourier f in
    [0.5, 1.5] and one source, plus per instance 4096 distinct receivers (not
    the source), a separately seeded reference field f_ref and the noise draws
    for the targets T_i = S_ref(x_i) + noise_i.  Returns a list of
    ``(instance, receivers, f_ref, noise_draws)``; S_ref is left to the
    caller, since computing it is the method itself."""
    rng = np.random.default_rng(SEED_BASE + 5)
    dims = (n, n)
    h = 1.0 / (n - 1)
    out = []
    for k in range(count):
        f = fourier_field(rng, dims, h)
        src = random_sources(rng, n * n, 1)
        pool = np.setdiff1d(np.arange(n * n, dtype=np.int64), src)
        recv = np.sort(rng.choice(pool, size=min(nrecv, len(pool)),
                                  replace=False)).astype(np.int64)
        f_ref = fourier_field(rng, dims, h)
        eps = noise * rng.standard_normal(len(recv))
        inst = Instance(dims, h, hbar, f, src, np.zeros(1), name=f"c5_{k}_{n}")
        out.append((inst, recv, f_ref, eps))
    return out


def example1(h: float = 2.0 ** -10, half_width: float = 0.125,
             hbar: float = 0.006) -> Instance:
    """Sec. 5.4 Example 1 grid: [-w, w]^2 with spacing h, f = exp(r) with r
    the distance to the origin, one source at the origin (S = 0 there).  The
    node at index (i, j) sits at (-w + i h, -w + j h)."""
    n = int(round(2 * half_width / h)) + 1
    dims = (n, n)
    x = -half_width + np.arange(n) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    f = np.exp(np.sqrt(X * X + Y * Y))
    mid = n // 2
    src = np.array([flat_index(dims, (mid, mid))], dtype=np.int64)
    return Instance(dims, h, hbar, f, src, np.zeros(1), name="example1",
                    extra={"origin_offset": half_width})


def random_small(seed: int, ndim: int = 2, max_side: int = 16,
                 min_side: int = 2, nsrc_max: int = 4,
                 hbar_over_h: Tuple[float, float] = (0.5, 4.0),
                 with_U: bool = False) -> Instance:
    """Small random instance for exhaustive checks: random sides, random
    positive f, 1..nsrc_max sources (faces and corners allowed), hbar a random
    multiple of h, optional non-zero source values U."""
    rng = np.random.default_rng(SEED_BASE * 1000 + seed)
    dims = tuple(int(v) for v in rng.integers(min_side, max_side + 1, size=ndim))
    h = 1.0 / (max(dims) - 1)
    f = rng.uniform(0.5, 2.0, size=dims[::-1])
    n = int(np.prod(dims))
    nsrc = int(rng.integers(1, nsrc_max + 1))
    src = random_sources(rng, n, nsrc)
    hbar = float(rng.uniform(*hbar_over_h)) * h
    U = rng.uniform(0.0, 0.05, len(src)) if with_U else np.zeros(len(src))
    return Instance(dims, h, hbar, f, src, U, name=f"small_{seed}")
