"""Closed forms that pin the oracle from outside.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``slab_phi`` -- exact discrete solution when the problem reduces to one
  dimension (constant f, sources filling the face x = 0, zero flux on every
  other face).  Every row then reads c(2 phi_m - phi_{m-1} - phi_{m+1})
  + f^2 phi_m = 0, whose decaying solution is phi_m ~ exp(-kappa m) with
  cosh(kappa) = 1 + f^2 h^2 / (2 hbar^2); the mirror condition at the far face
  selects phi_m = cosh(kappa (n-1-m)) / cosh(kappa (n-1)).  This is the
  discrete counterpart of the 1D Green's function of Sec. 3.2,
  Eq. (GreensFunction1D), which decays as exp(-f|x|/hbar).

* ``lattice_green`` / ``image_phi`` -- the Green's function of the infinite
  lattice operator c sum_a (2u - u_{+a} - u_{-a}) + f^2 u = delta, written as
  a Laplace transform of the lattice heat kernel,
      G(m) = int_0^inf exp(-f^2 t) prod_a exp(-2ct) I_{m_a}(2ct) dt,
  and, for a single source on a finite grid with zero-flux faces, the sum of
  G over the mirror images of the source (period 2(n_a - 1) per axis),
  normalised to phi = 1 at the source.  It is the discrete analogue of the
  closed-form Green's functions of Sec. 3.2, Eqs. (GreensFunction2D/3D).

* ``continuum_S`` -- S = -hbar log G for the continuum Green's functions of
  Sec. 3.2: K0(f r/hbar) in 2D and exp(-f r/hbar)/r in 3D (up to constants).
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, special


def slab_kappa(f: float, h: float, hbar: float) -> float:
    x = f * f * h * h / (2.0 * hbar * hbar)
    return float(np.log1p(x + np.sqrt(x * (x + 2.0))))     # arccosh(1 + x)


def slab_S(n: int, f: float, h: float, hbar: float) -> np.ndarray:
    """S_m = -hbar log phi_m for phi_m = cosh(kappa(n-1-m))/cosh(kappa(n-1)),
    m = 0..n-1, evaluated without overflow."""
    k = slab_kappa(f, h, hbar)
    m = np.arange(n, dtype=np.float64)
    L = n - 1
    log_phi = (-k * m + np.log1p(np.exp(-2.0 * k * (L - m)))
               - np.log1p(np.exp(-2.0 * k * L)))
    return -hbar * log_phi


def slab_phi(n: int, f: float, h: float, hbar: float) -> np.ndarray:
    return np.exp(-slab_S(n, f, h, hbar) / hbar)


def _log_time_grid(step: float = 0.004, lo: float = -34.0, hi: float = 12.0):
    s = np.arange(lo, hi + step, step)
    return s, step


def green_table(max_off: int, f: float, c: float, ndim: int) -> np.ndarray:
    """G(m) for every offset 0 <= m_a <= max_off of the infinite lattice
    operator, as an ndim-dimensional array.

    The substitution t = exp(s) turns the Laplace integral into an integral
    over the real line whose integrand decays exponentially as s -> -inf and
    doubly exponentially as s -> +inf, so the trapezoid rule on a uniform s
    grid converges geometrically in the step; with step 0.004 the rule is
    exact to rounding for the offsets used here."""
    s, ds = _log_time_grid()
    t = np.exp(s)
    m = np.arange(max_off + 1, dtype=np.float64)
    # per-axis factors exp(-2ct) I_m(2ct), shape (max_off+1, len(s))
    T = special.ive(m[:, None], 2.0 * c * t[None, :])
    wgt = ds * t * np.exp(-f * f * t)          # dt = t ds, times exp(-f^2 t)
    if ndim == 2:
        return (T * wgt[None, :]) @ T.T
    if ndim == 3:
        return np.einsum("as,bs,cs,s->abc", T, T, T, wgt, optimize=True)
    raise ValueError("ndim must be 2 or 3")


def lattice_green(m, f: float, c: float) -> float:
    """G(m) for one integer offset vector (direct adaptive quadrature of the
    same Laplace integral; used to cross-check ``green_table``)."""
    mm = np.array(sorted(abs(int(v)) for v in m), dtype=np.float64)

    def integrand(tt):
        val = np.exp(-f * f * tt)
        for q in mm:
            val = val * special.ive(q, 2.0 * c * tt)
        return val

    v1, _ = integrate.quad(integrand, 0.0, 1.0, epsabs=0.0, epsrel=1e-12,
                           limit=400)
    v2, _ = integrate.quad(integrand, 1.0, np.inf, epsabs=0.0, epsrel=1e-12,
                           limit=400)
    return float(v1 + v2)


def image_phi(dims, h: float, hbar: float, f: float, src_coords,
              kmax: int = -1) -> np.ndarray:
    """phi on the full grid for constant f and one source (phi = 1 there),
    zero-flux faces, by summing lattice Green's functions over the mirror
    images of the source (offsets s*y + 2k(n-1), s = +-1, |k| <= kmax, per
    axis).  ``kmax < 0`` picks the smallest count whose next image is at
    least exp(-45) below the nearest one along that axis.  Returns an array
    of shape dims[::-1]."""
    dims = tuple(int(v) for v in dims)
    nd = len(dims)
    c = hbar * hbar / (h * h)
    if kmax < 0:
        kap = slab_kappa(f, h, hbar)
        kmax = 1 + int(np.ceil(45.0 / (kap * 2 * (min(dims) - 1))))
    per_axis = []
    max_off = 0
    for a, n in enumerate(dims):
        y = int(src_coords[a])
        P = 2 * (n - 1)
        imgs = [sg * y + k * P for sg in (1, -1) for k in range(-kmax, kmax + 1)]
        per_axis.append(imgs)
        max_off = max(max_off, max(abs(n - 1 - v) for v in imgs),
                      max(abs(v) for v in imgs))
    # The image set is a product over axes, so the image sum of the Laplace
    # integrand factorises: u(x) = int w(t) prod_a V_a(x_a, t) dt with
    # V_a(x, t) = sum_{images y} exp(-2ct) I_{|x - y|}(2ct).
    sgrid, ds = _log_time_grid()
    t = np.exp(sgrid)
    T = special.ive(np.arange(max_off + 1, dtype=np.float64)[:, None],
                    2.0 * c * t[None, :])
    wgt = ds * t * np.exp(-f * f * t)
    V = []
    for a, n in enumerate(dims):
        x = np.arange(n)
        Va = np.zeros((n, len(sgrid)))
        for img in per_axis[a]:
            Va += T[np.abs(x - img)]
        V.append(Va)
    if nd == 2:
        u = (V[1] * wgt[None, :]) @ V[0].T                  # (y, x)
    else:
        u = np.einsum("zs,ys,xs,s->zyx", V[2], V[1], V[0], wgt, optimize=True)
    return u / u[tuple(int(src_coords[a]) for a in reversed(range(nd)))]


def continuum_S(r: np.ndarray, f: float, hbar: float, ndim: int) -> np.ndarray:
    """-hbar log G(r) for the continuum Green's function (constants dropped):
    2D K0(f r/hbar) (Eq. GreensFunction2D), 3D exp(-f r/hbar)/r
    (Eq. GreensFunction3D)."""
    z = f * np.asarray(r, dtype=np.float64) / hbar
    if ndim == 2:
        return -hbar * (np.log(special.k0e(z)) - z)
    if ndim == 3:
        return hbar * (z + np.log(np.asarray(r, dtype=np.float64)))
    raise ValueError("ndim must be 2 or 3")
