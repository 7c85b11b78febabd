"""Pins of the backtracking oracle (oracle/paths.py): gradient of S and the
Euler integration of dx/dt = -grad S / |grad S| (path-planning section,
Eq. PathPlanning-backTrackOnS), against closed forms."""
import numpy as np
import pytest

from oracle import fd, paths
from paper_1403_1937_gb300 import workloads as wl


def _grid(dims, h):
    axes = [np.arange(n) * h for n in dims]
    return np.meshgrid(*axes[::-1], indexing="ij")[::-1]   # x, y(, z) arrays of shape dims[::-1]


@pytest.mark.parametrize("dims", [(7, 5), (6, 4, 5)])
def test_gradient_of_linear_field_is_exact(dims):
    h = 0.1
    X = _grid(dims, h)
    coef = [3.0, -2.0, 0.5][:len(dims)]
    S = sum(c * x for c, x in zip(coef, X))
    G = paths.grad_S(S.ravel(), dims, h)
    for a, c in enumerate(coef):
        assert np.max(np.abs(G[a] - c)) <= 1e-12


def test_gradient_of_quadratic_central_and_one_sided():
    dims, h = (9, 3), 0.25
    X, Y = _grid(dims, h)
    S = X ** 2
    G = paths.grad_S(S.ravel(), dims, h).reshape(2, 3, 9)
    x = np.arange(9) * h
    # central differences are exact for a quadratic inside
    assert np.allclose(G[0][:, 1:-1], 2 * x[1:-1], atol=1e-13)
    # one-sided on the faces: (S1 - S0)/h = h, (S8 - S7)/h = 2 x_8 - h
    assert np.allclose(G[0][:, 0], h, atol=1e-13)
    assert np.allclose(G[0][:, -1], 2 * x[-1] - h, atol=1e-13)
    assert np.max(np.abs(G[1])) == 0.0


def test_interpolation_reproduces_multilinear_fields():
    dims, h = (5, 4, 3), 0.5
    X, Y, Z = _grid(dims, h)
    F = 1.0 + 2 * X - Y + 0.5 * Z + 0.25 * X * Y - 0.75 * Y * Z + 0.1 * X * Y * Z
    G = F.ravel()[None, :]
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, (50, 3)) * np.array([(d - 1) * h for d in dims])
    got = paths.interp(G, dims, h, pts)[:, 0]
    x, y, z = pts.T
    want = 1.0 + 2 * x - y + 0.5 * z + 0.25 * x * y - 0.75 * y * z + 0.1 * x * y * z
    assert np.max(np.abs(got - want)) <= 1e-12


@pytest.mark.parametrize("nd", [2, 3])
def test_backtracking_on_a_cone_goes_straight_to_the_source(nd):
    """S = |x - y0| (the eikonal solution for f = 1 and one source): every
    path runs along the segment to y0, ends within eps, after the number of
    steps the arc length fixes."""
    n = 33 if nd == 3 else 65
    h = 1.0 / (n - 1)
    dims = (n,) * nd
    X = _grid(dims, h)
    c = n // 2
    y0 = np.full(nd, c * h)
    S = np.sqrt(sum((x - y0[a]) ** 2 for a, x in enumerate(X)))
    src = np.array([sum(c * n ** a for a in range(nd))])
    G = paths.grad_S(S.ravel(), dims, h)
    rng = np.random.default_rng(nd)
    starts = rng.uniform(0.05, 0.95, (12, nd))
    step, eps = 0.5 * h, 1.5 * h
    P, L, st = paths.backtrack(G, dims, h, starts, step, 2000, src, eps)
    assert np.all(st == 0)
    for p in range(len(starts)):
        pts = P[p, :L[p] + 1]
        d0 = np.linalg.norm(starts[p] - y0)
        u = (y0 - starts[p]) / d0
        rel = pts - starts[p]
        perp = rel - np.outer(rel @ u, u)
        assert np.max(np.linalg.norm(perp, axis=1)) <= 2 * h
        assert np.linalg.norm(pts[-1] - y0) < eps
        assert abs(L[p] - (d0 - eps) / step) <= 3


def test_backtracking_descends_the_discrete_solution():
    """On the discrete solution of a random 2D problem the interpolated S
    decreases along every path and every path reaches a source."""
    inst = wl.random_small(21, ndim=2, max_side=60, min_side=40, nsrc_max=3,
                           hbar_over_h=(2.0, 4.0))
    S, _, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    G = paths.grad_S(S, inst.dims, inst.h)
    rng = np.random.default_rng(5)
    hi = np.array([(d - 1) * inst.h for d in inst.dims])
    starts = rng.uniform(0, 1, (20, 2)) * hi
    P, L, st = paths.backtrack(G, inst.dims, inst.h, starts, 0.25 * inst.h, 5000,
                               inst.src_idx, 2.0 * inst.h)
    assert np.all(st == 0)
    Sg = S[None, :]
    for p in range(len(starts)):
        s = paths.interp(Sg, inst.dims, inst.h, P[p, :L[p] + 1])[:, 0]
        assert np.all(np.diff(s) <= 1e-12)


# ---- shape-from-shading forcing (Eq. SfS-forcingFunc)
from oracle import sfs   # noqa: E402


def test_sfs_forcing_inverts_the_imaging_operator():
    """f = sqrt(1/P^2 - 1) returns |grad S*| for P = 1/sqrt(|grad S*|^2 + 1),
    checked on the analytic gradient of a paraboloid; f_min clamps flat
    points; P outside (0, 1] is rejected as NaN."""
    x = np.linspace(-1, 1, 41)
    X, Y = np.meshgrid(x, x)
    gz = np.sqrt((2 * 0.7 * X) ** 2 + (2 * 0.7 * Y) ** 2)     # |grad| of 0.7 (x^2 + y^2)
    P = sfs.image_of_height(gz ** 2)
    f = sfs.forcing(P, 0.0)
    assert np.max(np.abs(f - gz)) <= 1e-12
    f2 = sfs.forcing(P, 0.05)
    assert np.all(f2 >= 0.05) and np.allclose(f2[gz > 0.05], gz[gz > 0.05], atol=1e-12)
    bad = sfs.forcing(np.array([0.0, -0.1, 1.5, np.nan, 1.0]), 0.01)
    assert np.all(np.isnan(bad[:4])) and bad[4] == 0.01
