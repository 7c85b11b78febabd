"""Pins of the CPU oracle against facts that do not come from the oracle itself:
an independent dense construction, exact discrete closed forms, the lattice
Green's function with mirror images, continuum Green's functions, the
hbar -> 0 limit, M-matrix invariants and complex-step derivatives.

Each pin is chosen so that a plausible slip in ``oracle/fd.py`` (a dropped
f^2 term, h instead of h^2, a wrong face weight, a transposed axis, a sign)
fails at least one test.
"""
import json
import os

import numpy as np
import pytest

from oracle import cg, closed_forms, dense, fd
from paper_1403_1937_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- O1 dense
@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("boundary", [0, 1])
def test_dense_independent_construction(seed, boundary):
    """Mirror-ghost dense system with Dirichlet rows == symmetric half-cell
    sparse system (Sec. 6 Eq. sparse-system, Sec. 3.2 sources)."""
    ndim = 2 if seed < 5 else 3
    inst = wl.random_small(seed, ndim=ndim, max_side=14 if ndim == 2 else 6,
                           with_U=(seed % 2 == 1))
    S, phi, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx,
                           inst.src_U, boundary)
    phid, Sd = dense.dense_solve(inst.f, inst.dims, inst.h, inst.hbar,
                                 inst.src_idx, inst.src_U, boundary)
    phi_unshifted = phi * np.exp(-sys.U_min / sys.hbar)
    assert np.max(np.abs(phi_unshifted / phid - 1)) < 1e-12
    assert np.max(np.abs(S - Sd)) < 1e-12


def test_dense_nonsquare_axis_order():
    """Strongly anisotropic f on a non-square grid: swapping the x and y
    axes anywhere in the assembly changes the answer."""
    dims = (9, 5)
    h, hbar = 0.125, 0.2
    X, Y = wl.node_coords(dims, h)
    f = 0.5 + 2.0 * X + 0.1 * Y
    src = [wl.flat_index(dims, (0, 4)), wl.flat_index(dims, (8, 0))]
    S, _, _ = fd.solve(f, dims, h, hbar, src)
    _, Sd = dense.dense_solve(f, dims, h, hbar, src)
    assert np.max(np.abs(S - Sd)) < 1e-12
    _, Sd_t = dense.dense_solve(f.T.copy(), (5, 9), h, hbar,
                                [wl.flat_index((5, 9), (4, 0)),
                                 wl.flat_index((5, 9), (0, 8))])
    assert np.max(np.abs(S.reshape(5, 9) - Sd_t.reshape(9, 5).T)) < 1e-12
    assert np.max(np.abs(S.reshape(5, 9) - Sd.reshape(5, 9))) < 1e-12


# ---------------------------------------------------------------- 1D exact
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("f,hbar,n", [(1.0, 0.01, 60), (1.7, 0.03, 33),
                                      (0.6, 0.002, 41)])
def test_slab_exact(axis, f, hbar, n):
    """Sources filling one face, constant f: the discrete problem is 1D and
    phi_m = cosh(kappa(n-1-m))/cosh(kappa(n-1)), cosh kappa = 1 +
    f^2 h^2/(2 hbar^2) (discrete analogue of Eq. GreensFunction1D)."""
    ndim = 3 if axis == 2 else 2
    h = 1.0 / (n - 1)
    dims = [2] * ndim
    dims[axis] = n
    dims = tuple(dims)
    F = np.full(dims[::-1], f)
    src = []
    for flat in range(int(np.prod(dims))):
        coords = np.unravel_index(flat, dims[::-1])[::-1]
        if coords[axis] == 0:
            src.append(flat)
    S, _, _ = fd.solve(F, dims, h, hbar, src)
    Sg = np.moveaxis(S.reshape(dims[::-1]), ndim - 1 - axis, -1)
    ex = closed_forms.slab_S(n, f, h, hbar)
    assert np.max(np.abs(Sg - ex)) < 1e-12 * max(1.0, ex.max())


# ------------------------------------------------- O4 lattice Green + images
def test_lattice_green_table_vs_quadrature():
    c = 0.9
    G = closed_forms.green_table(30, 1.3, c, 2)
    ref = [closed_forms.lattice_green(m, 1.3, c) for m in [(0, 0), (5, 2), (30, 11)]]
    got = [G[0, 0], G[5, 2], G[30, 11]]
    # the two quadratures of the same integral agree up to a common factor
    # near 1 (the trapezoid weight), which the normalisation phi(y) = 1 removes
    ratio = np.array(got) / np.array(ref)
    assert np.max(np.abs(ratio / ratio[0] - 1)) < 1e-10
    assert abs(ratio[0] - 1) < 1e-9


def test_c1_equals_lattice_green_closed_form():
    """Config 1 (129^2, f=1, hbar=0.01, centre source) equals the image sum of
    the lattice Green's function to rounding, including the far corners
    where phi ~ 1e-31."""
    inst = wl.config1()
    S, phi, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    ph = closed_forms.image_phi(inst.dims, inst.h, inst.hbar, 1.0, (64, 64))
    assert np.max(np.abs(phi.reshape(129, 129) / ph - 1)) < 1e-12
    gold = json.load(open(os.path.join(GOLDEN, "c1_closed_form.json")))
    S2 = S.reshape(129, 129)
    for (x, y), s in zip(gold["nodes"], gold["S"]):
        assert abs(S2[y, x] - s) < 1e-13


@pytest.mark.parametrize("dims,h,hbar,src", [
    ((17, 13), 1 / 16, 0.05, (5, 4)),
    ((12, 5, 7), 1 / 11, 0.08, (0, 4, 3)),
    ((9, 9, 9), 1 / 8, 0.1, (4, 4, 4)),
    ((21, 8), 1 / 20, 0.02, (20, 7)),
])
def test_images_off_centre_and_3d(dims, h, hbar, src):
    ph = closed_forms.image_phi(dims, h, hbar, 1.0, src)
    _, phi, _ = fd.solve(np.ones(dims[::-1]), dims, h, hbar,
                         [wl.flat_index(dims, src)])
    assert np.max(np.abs(phi.reshape(dims[::-1]) / ph - 1)) < 1e-12


# -------------------------------------------------------- O3 invariants
def _neighbours(dims):
    n = int(np.prod(dims))
    idx = np.arange(n)
    coords = np.unravel_index(idx, dims[::-1])
    out = []
    stride = 1
    for ax, nax in enumerate(dims):
        xa = coords[len(dims) - 1 - ax]
        lo = idx[xa < nax - 1]
        out.append((lo, lo + stride))
        stride *= nax
    return out


@pytest.mark.parametrize("seed", range(4))
def test_m_matrix_invariants(seed):
    inst = wl.random_small(100 + seed, ndim=2 if seed < 3 else 3,
                           max_side=24 if seed < 3 else 10)
    S, phi, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.all(phi > 0) and np.all(phi <= 1 + 1e-15)
    assert np.all(S >= -1e-15)
    assert np.all(S[sys.src] == 0)
    # discrete maximum principle: off the sources phi_i < max neighbour
    mx = np.zeros(sys.n)
    for lo, hi in _neighbours(inst.dims):
        np.maximum.at(mx, lo, phi[hi])
        np.maximum.at(mx, hi, phi[lo])
    assert np.all(phi[sys.unk] < mx[sys.unk])
    # monotone in f: raising f raises S (not at sources)
    S_up, _, _ = fd.solve(inst.f * 1.1, inst.dims, inst.h, inst.hbar,
                          inst.src_idx)
    assert np.all(S_up[sys.unk] > S[sys.unk])
    # adding a source lowers S
    extra = np.setdiff1d(np.arange(sys.n), sys.src)[7]
    S_more, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar,
                            np.append(inst.src_idx, extra))
    keep = np.setdiff1d(sys.unk, [extra])
    assert np.all(S_more[keep] < S[keep])


def test_c1_symmetry():
    inst = wl.config1()
    S, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    S = S.reshape(129, 129)
    for T in (S.T, S[::-1, :], S[:, ::-1], S[::-1, ::-1].T):
        assert np.max(np.abs(T - S)) < 1e-13


def test_source_values_and_shift():
    """Non-zero source values: S = U exactly at the sources, and adding a
    constant to every U shifts S by that constant (linearity in phi)."""
    inst = wl.random_small(7, ndim=2, max_side=12, nsrc_max=4, with_U=True)
    S, _, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx,
                         inst.src_U)
    assert np.array_equal(S[sys.src], sys.U)
    S2, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx,
                        inst.src_U + 0.3)
    assert np.max(np.abs(S2 - S - 0.3)) < 1e-12


def test_duplicate_and_invalid_sources():
    dims = (5, 4)
    f = np.ones((4, 5))
    S1, _, _ = fd.solve(f, dims, 0.25, 0.1, [3, 3, 7], [0.0, 0.0, 0.1])
    S2, _, _ = fd.solve(f, dims, 0.25, 0.1, [7, 3], [0.1, 0.0])
    assert np.array_equal(S1, S2)
    with pytest.raises(ValueError):
        fd.assemble(f, dims, 0.25, 0.1, [3, 3], [0.0, 0.1])
    with pytest.raises(ValueError):
        fd.assemble(f, dims, 0.25, 0.1, [20])
    with pytest.raises(ValueError):
        fd.assemble(-f, dims, 0.25, 0.1, [2])


# -------------------------------------------------- O2 identity residual
def test_identity_residual_of_direct_solution():
    inst = wl.random_small(11, ndim=2, max_side=30)
    S, phi, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(fd.identity_residual(sys, S))) < 1e-11
    assert np.max(fd.componentwise_residual(sys, phi)) < 1e-12
    # a 1e-6 perturbation of S at one node is visible in the identity
    S2 = S.copy()
    S2[sys.unk[3]] += 1e-6
    assert np.max(np.abs(fd.identity_residual(sys, S2))) > 1e-6 / inst.hbar * 0.5


# ------------------------------------------- O5 continuum Green's function
def test_continuum_green_2d_second_order():
    """With the source far from the faces, S(r1) - S(r2) along the x axis
    tends to the K0 prediction of Eq. (GreensFunction2D) at second order in
    h/hbar."""
    hbar = 0.05
    errs = []
    for n in (81, 161, 321):
        h = 2.0 / (n - 1)
        dims = (n, n)
        mid = (n - 1) // 2
        S, _, _ = fd.solve(np.ones((n, n)), dims, h, hbar,
                           [wl.flat_index(dims, (mid, mid))])
        S = S.reshape(n, n)
        r1, r2 = 0.1, 0.3
        i1, i2 = mid + int(round(r1 / h)), mid + int(round(r2 / h))
        dS = S[mid, i2] - S[mid, i1]
        ref = (closed_forms.continuum_S(r2, 1.0, hbar, 2)
               - closed_forms.continuum_S(r1, 1.0, hbar, 2))
        errs.append(abs(dS - ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_continuum_green_3d_second_order():
    """3D analogue with exp(-f r/hbar)/r (Eq. GreensFunction3D); faces 16
    hbar away from the source so the images are negligible."""
    hbar, L = 0.05, 1.6
    errs = []
    for n in (33, 65, 129):
        h = L / (n - 1)
        dims = (n, n, n)
        mid = (n - 1) // 2
        S, _, _, info = cg.solve(np.ones((n, n, n)), dims, h, hbar,
                                 [wl.flat_index(dims, (mid, mid, mid))],
                                 tol=1e-12)
        assert info["status"] == 0
        S = S.reshape(n, n, n)
        r1, r2 = 0.3, 0.6
        i1, i2 = mid + int(round(r1 / h)), mid + int(round(r2 / h))
        dS = S[mid, mid, i2] - S[mid, mid, i1]
        ref = (closed_forms.continuum_S(r2, 1.0, hbar, 3)
               - closed_forms.continuum_S(r1, 1.0, hbar, 3))
        errs.append(abs(dS - ref))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


# ------------------------------------------------------- O6 hbar -> 0
def test_hbar_limit_distance():
    """S -> f * (Euclidean distance to the nearest source) as hbar -> 0 with
    h = hbar/16 (Sec. 3.2: S converges to f r); the error falls roughly like
    hbar log(1/hbar)."""
    f0 = 1.5
    errs = []
    for hbar in (0.04, 0.02, 0.01):
        h = hbar / 16
        n = int(round(0.5 / h)) + 1
        dims = (n, n)
        src = (n // 4, n // 3)
        S, _, _ = fd.solve(np.full((n, n), f0), dims, h, hbar,
                           [wl.flat_index(dims, src)])
        X, Y = wl.node_coords(dims, h)
        d = np.hypot(X - src[0] * h, Y - src[1] * h)
        far = d >= 0.1
        errs.append(np.max(np.abs(S.reshape(n, n)[far] - f0 * d[far])))
    assert errs[0] > errs[1] > errs[2]
    for e, hb in zip(errs, (0.04, 0.02, 0.01)):
        assert e < 3.0 * hb * np.log(1.0 / hb)


def test_example1_context():
    """Sec. 5.4 Example 1 (exact R = exp(r) - 1): the finite-difference S
    approaches R as hbar falls; the paper's printed errors for its FFT
    perturbation series (Table eikonalexp1) are context, not parity."""
    gold = json.load(open(os.path.join(GOLDEN, "example1_paper.json")))
    assert gold["setup"]["hbar"] == 0.006
    inst = wl.example1()
    n = inst.dims[0]
    x = -0.125 + np.arange(n) * inst.h
    X, Y = np.meshgrid(x, x)
    R = np.exp(np.hypot(X, Y)) - 1
    m = R > 0
    lam, mx = [], []
    for hbar in (0.006, 0.003, 0.0015):
        S, _, _ = fd.solve(inst.f, inst.dims, inst.h, hbar, inst.src_idx)
        d = np.abs(S.reshape(n, n) - R)
        lam.append(100 * np.mean(d[m] / R[m]))
        mx.append(d.max())
    assert lam[0] > lam[1] > lam[2]
    assert mx[0] > mx[1] > mx[2]
    # at the paper's hbar the max difference is a few hbar (log prefactor of
    # the Dirichlet source), the same order as the printed 0.0021-0.0027
    assert mx[0] < 5 * 0.006


# ------------------------------------------------------------ O8 gradient
@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_complex_step(seed):
    """Adjoint dL/df against complex-step derivatives of the forward solve
    for every node (L = sum_i v_i S_i with random v)."""
    inst = wl.random_small(200 + seed, ndim=2, max_side=9, min_side=4)
    sys = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(sys.n)
    g = fd.grad_f(sys, v)
    eps = 1e-30
    f = sys.f
    cs = np.zeros(sys.n)
    for k in range(sys.n):
        fc = f.astype(np.complex128)
        fc[k] += 1j * eps
        Sc = fd.solve_complex(sys, fc)
        cs[k] = np.dot(v, Sc.imag) / eps
    assert np.max(np.abs(g - cs)) < 1e-10 * np.max(np.abs(cs))
    assert np.all(g[sys.src] == 0)


def test_gradient_central_difference_3d():
    inst = wl.random_small(300, ndim=3, max_side=7, min_side=4)
    sys = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(sys.n)
    g = fd.grad_f(sys, v)
    d = rng.standard_normal(sys.n)
    d[sys.src] = 0
    eps = 1e-6
    Sp, _, _ = fd.solve(sys.f + eps * d, inst.dims, inst.h, inst.hbar, inst.src_idx)
    Sm, _, _ = fd.solve(sys.f - eps * d, inst.dims, inst.h, inst.hbar, inst.src_idx)
    fdiff = (np.dot(v, Sp) - np.dot(v, Sm)) / (2 * eps)
    assert abs(np.dot(g, d) - fdiff) < 1e-7 * abs(fdiff)


# ------------------------------------------------------------- CG oracle
def test_cg_oracle_matches_direct_2d():
    inst = wl.config2(n=256)
    Sd, phid, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    S, phi, _, info = cg.solve(inst.f, inst.dims, inst.h, inst.hbar,
                               inst.src_idx, tol=1e-13)
    assert info["status"] == 0 and info["cw"] <= 1e-13
    assert np.max(np.abs(phi / phid - 1)) < 1e-11
    assert np.max(np.abs(S - Sd)) < 1e-12


def test_cg_oracle_matches_direct_3d():
    inst = wl.config3(n=20)
    Sd, phid, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    S, phi, _, info = cg.solve(inst.f, inst.dims, inst.h, inst.hbar,
                               inst.src_idx, tol=1e-13)
    assert info["status"] == 0
    assert np.max(np.abs(phi / phid - 1)) < 1e-11


def test_cg_oracle_max_iter_reports_not_converged():
    inst = wl.config1()
    _, _, _, info = cg.solve(inst.f, inst.dims, inst.h, inst.hbar,
                             inst.src_idx, tol=1e-13, max_iter=20)
    assert info["status"] == 1 and info["iters"] == 20


# ------------------------------------------- relative-form (underflow) solve
# fd.solve_relative is the oracle for every problem whose phi underflows
# float64 (S/hbar > ~700).  It rests on fd.graph_distance for its scale.  The
# pins below tie both to facts outside them: closed-form grid distances, a
# brute-force shortest path, the direct solve where both work, the exact
# slab solution beyond the float64 range, and the lattice Green's function.

def _octile(d):
    """Shortest path length on the 8- (2D) / 26- (3D) neighbour lattice with
    unit spacing: straight moves, face diagonals and (3D) body diagonals."""
    a = sorted((abs(v) for v in d), reverse=True) + [0, 0]
    return (a[0] - a[1]) + np.sqrt(2.0) * (a[1] - a[2]) + np.sqrt(3.0) * a[2]


@pytest.mark.parametrize("dims,srcs,U", [
    ((9, 7), [(2, 3)], [0.0]),
    ((11, 6), [(0, 0), (10, 5)], [0.0, 0.3]),
    ((5, 6, 4), [(1, 4, 2)], [0.0]),
    ((6, 5, 7), [(0, 0, 0), (5, 4, 6)], [0.2, 0.0]),
])
def test_graph_distance_uniform_is_lattice_metric(dims, srcs, U):
    """Constant f: the graph distance is f h times the lattice (octile)
    metric, minimised over the sources with the offsets U_k - U_min."""
    h, f0 = 0.1, 1.7
    F = np.full(dims[::-1], f0)
    sys = fd.assemble(F, dims, h, 0.05, [wl.flat_index(dims, s) for s in srcs], U)
    d = fd.graph_distance(sys)
    coords = np.stack(np.unravel_index(np.arange(sys.n), dims[::-1])[::-1], -1)
    Umin = min(U)
    want = np.full(sys.n, np.inf)
    for s, u in zip(srcs, U):
        dd = np.array([_octile(c - np.array(s)) for c in coords])
        want = np.minimum(want, (u - Umin) + f0 * h * dd)
    assert np.max(np.abs(d - want)) < 1e-12


def test_graph_distance_brute_force_bellman_ford():
    """Random f on a small grid: pure-Python Bellman-Ford over the same
    neighbour set and edge cost (length x mean of f at the two ends)."""
    rng = np.random.default_rng(5)
    for dims in [(5, 4), (3, 4, 3)]:
        n = int(np.prod(dims))
        F = rng.uniform(0.5, 2.0, size=dims[::-1])
        h = 0.3
        src = [0, n - 2]
        U = [0.1, 0.0]
        sys = fd.assemble(F, dims, h, 0.05, src, U)
        d = fd.graph_distance(sys)
        fl = F.ravel()
        coords = [tuple(int(v) for v in np.unravel_index(i, dims[::-1])[::-1]) for i in range(n)]
        index = {c: i for i, c in enumerate(coords)}
        dist = [np.inf] * n
        dist[src[0]] = U[0] - min(U)
        dist[src[1]] = U[1] - min(U)
        import itertools
        offs = [o for o in itertools.product((-1, 0, 1), repeat=len(dims)) if any(o)]
        for _ in range(n):
            for i, c in enumerate(coords):
                for o in offs:
                    j = index.get(tuple(a + b for a, b in zip(c, o)))
                    if j is None:
                        continue
                    cost = h * np.sqrt(sum(v * v for v in o)) * 0.5 * (fl[i] + fl[j])
                    if dist[j] + cost < dist[i]:
                        dist[i] = dist[j] + cost
        assert np.max(np.abs(d - np.array(dist))) < 1e-12


@pytest.mark.parametrize("seed,ndim,boundary,with_U", [
    (0, 2, 0, False), (1, 2, 1, True), (2, 3, 0, True), (3, 3, 1, False),
    (4, 2, 0, True),
])
def test_solve_relative_equals_direct(seed, ndim, boundary, with_U):
    """Where phi is representable, the relative-form solve (diagonal
    similarity D^-1 A D) gives the direct solution, for the graph-distance
    scale and for arbitrary other scales: the result must not depend on D."""
    inst = wl.random_small(400 + seed, ndim=ndim, max_side=18 if ndim == 2 else 8,
                           nsrc_max=3, with_U=with_U)
    S, _, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx,
                         inst.src_U, boundary)
    rng = np.random.default_rng(seed)
    gd = fd.graph_distance(sys)
    scales = [None, np.zeros(sys.n), 0.7 * gd + inst.hbar * rng.uniform(-5, 5, sys.n),
              rng.uniform(0.0, 40 * inst.hbar, sys.n)]
    for sc in scales:
        Sr = fd.solve_relative(sys, sc)
        assert np.array_equal(Sr[sys.src], sys.U)
        assert np.max(np.abs(Sr - S)) < 1e-11 * max(1.0, np.abs(S).max())


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_solve_relative_slab_beyond_float64(axis):
    """Sources filling one face, constant f, S/hbar up to ~830 at the far
    face: phi = exp(-S/hbar) underflows float64 there, so the direct solve
    fails, while the relative solve matches the exact slab solution
    (discrete analogue of Eq. GreensFunction1D) to rounding."""
    n, f0 = 600, 1.0
    h = 1.0 / (n - 1)
    hbar = h / 1.5                      # kappa = arccosh(2.125) = ln 4
    ndim = 3 if axis == 2 else 2
    dims = [2] * ndim
    dims[axis] = n
    dims = tuple(dims)
    F = np.full(dims[::-1], f0)
    src = [k for k in range(int(np.prod(dims)))
           if np.unravel_index(k, dims[::-1])[::-1][axis] == 0]
    ex = closed_forms.slab_S(n, f0, h, hbar)
    assert ex.max() / hbar > 800
    sys = fd.assemble(F, dims, h, hbar, src)
    Sr = fd.solve_relative(sys)
    Sg = np.moveaxis(Sr.reshape(dims[::-1]), ndim - 1 - axis, -1)
    assert np.max(np.abs(Sg - ex)) < 1e-12 * ex.max()
    with np.errstate(all="ignore"):
        Sd, _, _ = fd.solve(F, dims, h, hbar, src)
    Sdg = np.moveaxis(Sd.reshape(dims[::-1]), ndim - 1 - axis, -1)
    assert not np.all(np.abs(Sdg - ex) < 1e-6)      # the direct solve cannot
    # a second, unrelated scale gives the same answer beyond float64 too
    Sr2 = fd.solve_relative(sys, fd.graph_distance(sys) * 0.9 + 3 * hbar)
    assert np.max(np.abs(Sr2 - Sr)) < 1e-12 * ex.max()


@pytest.mark.parametrize("dims,h,hbar,src", [
    ((17, 13), 1 / 16, 0.05, (5, 4)),
    ((9, 9, 9), 1 / 8, 0.1, (4, 4, 4)),
    ((21, 8), 1 / 20, 0.02, (20, 7)),
])
def test_solve_relative_lattice_green_log_form(dims, h, hbar, src):
    """Single source, constant f: S of the relative solve equals
    -hbar log of the image sum of the lattice Green's function."""
    ph = closed_forms.image_phi(dims, h, hbar, 1.0, src)
    sys = fd.assemble(np.ones(dims[::-1]), dims, h, hbar, [wl.flat_index(dims, src)])
    Sr = fd.solve_relative(sys).reshape(dims[::-1])
    assert np.max(np.abs(Sr - (-hbar * np.log(ph)))) < 1e-12 * max(1.0, Sr.max())
