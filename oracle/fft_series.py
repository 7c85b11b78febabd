"""FFT perturbation series for 2D grids (Sec. 5, Table 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What is computed (paper passages followed):

* Sec. 5, Eqs. (Ldef), (invApprox), (phiSolution), (phiRecRelation),
  (phi_i_Solution): with a constant f~, phi = phi_0 - phi_1 + phi_2 - ... +
  (-1)^T phi_T, where phi_i = G * [(f^2 - f~^2) phi_{i-1}] is the convolution
  with the Green's function G of -hbar^2 Lap + f~^2.
* Sec. 3.2, Eq. (forcedPhiEquation) with the modified Green's function
  G~(x) = exp(-f~ |x| / hbar) (C = 1): phi_0 = G~ * delta_kron, the sources
  entering as Kronecker deltas (Eq. deltakron).  Eq. (GreensFunction2D):
  G(x) = K_0(f~ |x| / hbar) / (2 pi hbar^2).
* Table 1, steps 1-15, in that order: sample G~ and delta_kron on the grid,
  FFT, multiply, inverse FFT for phi_0; FFT of G; for i = 1..T the FFT of
  psi_i = (f^2 - f~^2) phi_{i-1}, the product with G's transform, the inverse
  FFT times the cell area h^2, and the signed update of phi; S = -hbar log phi.
* Sec. 5.1, Eq. (fTildeValue): f~ = sqrt((f_min^2 + f_max^2) / 2) minimises
  the bound sup|f^2 - f~^2| / f~^2 on the operator norm of L.

Readings (where the paper is silent):

* F1: a discrete convolution of two grid functions is the linear (aperiodic)
  one over the grid, sum_j K(x_i - x_j) g_j; the transforms are of arrays
  zero-padded to P_a >= 2 n_a - 1 points per axis (here the next power of
  two; any P_a >= 2 n_a - 1 gives the same convolution up to rounding), with
  the kernel sampled at the offsets -(n_a - 1) .. n_a - 1 and wrapped, so that
  no product wraps onto the grid.
* F2: G is singular at the origin; its sample at offset 0 is the average of
  G over the grid cell [-h/2, h/2]^2, using int_0^R r K_0(a r) dr =
  (1 - a R K_1(a R)) / a^2 along each ray of the cell.
* F3: "iteration T" of Table eikonalexp1 is the partial sum up to phi_T.
* F4: S = -hbar log phi with C = 1 (the constant hbar log C of Eq. STilde
  is dropped, as the paper does).
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, special


def f_tilde_optimal(f) -> float:
    """Eq. (fTildeValue): sqrt((f_min^2 + f_max^2) / 2)."""
    f = np.asarray(f, dtype=np.float64)
    return float(np.sqrt((f.min() ** 2 + f.max() ** 2) / 2.0))


def fft_size(n: int) -> int:
    """Transform length for an axis of n nodes (reading F1)."""
    p = 1
    while p < 2 * n - 1:
        p *= 2
    return p


def offsets(n: int, h: float) -> np.ndarray:
    """Offsets -(n - 1) h .. (n - 1) h of one axis."""
    return (np.arange(2 * n - 1) - (n - 1)) * h


def cell_average_green(ft: float, hbar: float, h: float) -> float:
    """Reading F2: (1/h^2) times the integral of G over [-h/2, h/2]^2, by
    rays: the square is 8 copies of the triangle 0 <= theta <= pi/4, whose ray
    at angle theta ends at R = (h/2) / cos(theta)."""
    a = ft / hbar

    def ray(theta):
        R = 0.5 * h / np.cos(theta)
        return (1.0 - a * R * special.k1(a * R)) / (a * a)

    val, _ = integrate.quad(ray, 0.0, np.pi / 4, epsabs=0.0, epsrel=1e-13, limit=200)
    return 8.0 * val / (h * h) / (2.0 * np.pi * hbar * hbar)


def green_2d(ft: float, hbar: float, h: float, nx: int, ny: int) -> np.ndarray:
    """G of Eq. (GreensFunction2D) on the offset grid, shape (2ny-1, 2nx-1);
    the origin takes the cell average (reading F2)."""
    ox, oy = offsets(nx, h), offsets(ny, h)
    r = np.hypot(ox[None, :], oy[:, None])
    with np.errstate(divide="ignore"):
        G = special.k0(ft * r / hbar) / (2.0 * np.pi * hbar * hbar)
    G[ny - 1, nx - 1] = cell_average_green(ft, hbar, h)
    return G


def green_tilde(ft: float, hbar: float, h: float, nx: int, ny: int) -> np.ndarray:
    """Table 1 step 1: G~ = exp(-f~ |x| / hbar) on the offset grid."""
    ox, oy = offsets(nx, h), offsets(ny, h)
    return np.exp(-ft * np.hypot(ox[None, :], oy[:, None]) / hbar)


def convolve(kern: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Linear convolution out_i = sum_j kern(x_i - x_j) g_j on the grid of g
    (shape (ny, nx)); kern on the offset grid (2ny-1, 2nx-1).  By FFT of
    zero-padded arrays with the kernel wrapped (reading F1)."""
    ny, nx = g.shape
    Py, Px = fft_size(ny), fft_size(nx)
    K = np.zeros((Py, Px))
    iy = (np.arange(2 * ny - 1) - (ny - 1)) % Py
    ix = (np.arange(2 * nx - 1) - (nx - 1)) % Px
    K[np.ix_(iy, ix)] = kern
    gp = np.zeros((Py, Px))
    gp[:ny, :nx] = g
    out = np.fft.ifft2(np.fft.fft2(K) * np.fft.fft2(gp))
    return out.real[:ny, :nx]


def convolve_direct(kern: np.ndarray, g: np.ndarray) -> np.ndarray:
    """The same convolution by its definition (brute force, small grids)."""
    ny, nx = g.shape
    out = np.zeros((ny, nx))
    for i in range(ny):
        for j in range(nx):
            out[i, j] = np.sum(kern[i - np.arange(ny)[:, None] + ny - 1,
                                    j - np.arange(nx)[None, :] + nx - 1] * g)
    return out


def series(f, dims, h: float, hbar: float, src_idx, terms: int, ft: float = 0.0):
    """Table 1 for a 2D grid dims = (nx, ny); f of shape (ny, nx) (x fastest).
    Returns S, phi (flat, x fastest), the list of phi_i (shape (ny, nx)) and
    f~ (the optimal one when ft <= 0)."""
    nx, ny = int(dims[0]), int(dims[1])
    f = np.asarray(f, dtype=np.float64).reshape(ny, nx)
    if ft <= 0.0:
        ft = f_tilde_optimal(f)
    # steps 1-5: phi_0 = G~ * delta_kron
    delta = np.zeros((ny, nx))
    delta.reshape(-1)[np.asarray(src_idx, dtype=np.int64)] = 1.0
    phi0 = convolve(green_tilde(ft, hbar, h, nx, ny), delta)
    # step 6
    phi = phi0.copy()
    # step 7
    G = green_2d(ft, hbar, h, nx, ny)
    # steps 8-14
    parts = [phi0]
    prev = phi0
    for i in range(1, terms + 1):
        psi = (f * f - ft * ft) * prev
        cur = convolve(G, psi) * h * h
        phi = phi + (-1) ** i * cur
        parts.append(cur)
        prev = cur
    # step 15
    with np.errstate(divide="ignore", invalid="ignore"):
        S = -hbar * np.log(phi)
    return S.reshape(-1), phi.reshape(-1), parts, ft


def operator_matrix(f, dims, h: float, hbar: float, ft: float) -> np.ndarray:
    """The discrete operator L_h g = h^2 G * [(f^2 - f~^2) g] as a dense
    matrix on the grid (small grids), built from its definition."""
    nx, ny = int(dims[0]), int(dims[1])
    f = np.asarray(f, dtype=np.float64).reshape(ny, nx)
    G = green_2d(ft, hbar, h, nx, ny)
    n = nx * ny
    iy, ix = np.divmod(np.arange(n), nx)
    Kij = G[iy[:, None] - iy[None, :] + ny - 1, ix[:, None] - ix[None, :] + nx - 1]
    return h * h * Kij * (f.reshape(-1) ** 2 - ft * ft)[None, :]
