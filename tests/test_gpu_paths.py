"""grad S and backtracking on the GPU (eik_grad_S, eik_backtrack) against
the oracle (oracle/paths.py) on the same S.  Both sides evaluate the same
explicitly rounded steps, so gradients, path points, lengths and statuses
are compared exactly."""
import numpy as np
import pytest

from oracle import paths as opaths
from paper_1403_1937_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eik():
    import torch
    from paper_1403_1937_gb300 import build
    build.build()
    from paper_1403_1937_gb300 import eik as e
    assert torch.cuda.is_available()
    return e


def _solve(eik, inst):
    import torch
    opt = eik.make_options(precision="mixed", tol=1e-8)
    f = torch.from_numpy(np.ascontiguousarray(inst.f)).cuda()
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, inst.src_idx, None, opt)
    S, _, _ = eik.eik_solve(h)
    eik.eik_destroy(h)
    return S.reshape(-1).contiguous()


@pytest.mark.parametrize("dims", [(37, 23), (16, 9, 11), (2, 2)])
def test_grad_S_bitwise(eik, dims):
    import torch
    rng = np.random.default_rng(sum(dims))
    S = rng.standard_normal(int(np.prod(dims)))
    G = eik.grad_S(torch.from_numpy(S).cuda(), dims, 0.37)
    np.testing.assert_array_equal(G.cpu().numpy(), opaths.grad_S(S, dims, 0.37))


@pytest.mark.parametrize("cfg", ["c2", "c3"])
def test_backtrack_matches_oracle(eik, cfg):
    inst = wl.config2(n=256) if cfg == "c2" else wl.config3(n=40)
    S = _solve(eik, inst)
    G = eik.grad_S(S, inst.dims, inst.h)
    S_h = S.cpu().numpy()
    G_ref = opaths.grad_S(S_h, inst.dims, inst.h)
    np.testing.assert_array_equal(G.cpu().numpy(), G_ref)
    nd = len(inst.dims)
    rng = np.random.default_rng(11)
    hi = np.array([(d - 1) * inst.h for d in inst.dims])
    starts = rng.uniform(0, 1, (64 if nd == 2 else 24, nd)) * hi
    step, eps, ms = 0.5 * inst.h, 2.0 * inst.h, 4000
    P, L, st = eik.backtrack(G, inst.dims, inst.h, starts, inst.src_idx, step, ms, eps)
    P_ref, L_ref, st_ref = opaths.backtrack(G_ref, inst.dims, inst.h, starts, step, ms,
                                           inst.src_idx, eps)
    np.testing.assert_array_equal(L.cpu().numpy(), L_ref)
    np.testing.assert_array_equal(st.cpu().numpy(), st_ref)
    np.testing.assert_array_equal(P.cpu().numpy(), P_ref)    # NaN tails compare equal
    assert np.all(st_ref == 0)          # every path reaches a source
    # S decreases along the paths (interpolated nodal S)
    for p in range(len(starts)):
        s = opaths.interp(S_h[None, :], inst.dims, inst.h, P_ref[p, :L_ref[p] + 1])[:, 0]
        assert np.all(np.diff(s) <= 1e-12)


def test_backtrack_edge_cases(eik):
    import torch
    from paper_1403_1937_gb300 import _lib
    dims, h = (9, 7), 0.125
    S = np.zeros(63)
    G = eik.grad_S(torch.from_numpy(S).cuda(), dims, h)       # flat field
    src = np.array([4 + 9 * 3])
    y0 = np.array([4 * h, 3 * h])
    # no paths
    P, L, st = eik.backtrack(G, dims, h, np.zeros((0, 2)), src, 0.1, 10, 0.2)
    assert P.shape == (0, 11, 2)
    # start on the source: reached before any step; flat field elsewhere: status 2;
    # max_steps = 0: status 1 unless already within eps
    P, L, st = eik.backtrack(G, dims, h, np.stack([y0, [0.0, 0.0]]), src, 0.1, 10, 0.2)
    assert L.tolist() == [0, 0] and st.tolist() == [0, 2]
    assert np.isnan(P[0, 1:].cpu().numpy()).all()
    P, L, st = eik.backtrack(G, dims, h, np.stack([y0, [0.0, 0.0]]), src, 0.1, 0, 0.2)
    assert L.tolist() == [0, 0] and st.tolist() == [0, 1]
    with pytest.raises(_lib.EikError):
        eik.backtrack(G, dims, h, np.zeros((1, 2)), src, -1.0, 10, 0.2)
    with pytest.raises(_lib.EikError):
        eik.grad_S(torch.zeros(63, dtype=torch.float64).cuda(), (63,), h)


def test_sfs_forcing_bitwise(eik):
    import torch
    from oracle import sfs
    rng = np.random.default_rng(4)
    P = np.concatenate([rng.uniform(1e-3, 1.0, 4093), [1.0, 0.0, -0.5, 1.5, np.nan]])
    f = eik.sfs_forcing(torch.from_numpy(P).cuda(), 0.01).cpu().numpy()
    np.testing.assert_array_equal(f, sfs.forcing(P, 0.01))


def test_shape_from_shading_recovers_height(eik):
    """A paraboloid height field z imaged under vertical light: the forcing
    from the image, one seed at the minimum with its height, and the mixed
    solve give the oracle's discrete solution (S within 1e-6) and a height
    field whose distance to z shrinks with hbar (O(hbar) plus the source's
    logarithmic term)."""
    import torch
    from oracle import fd, sfs
    errs = []
    for n in (129, 257):
        h = 1.0 / (n - 1)
        x = np.arange(n) * h
        X, Y = np.meshgrid(x, x)
        z = 0.7 * ((X - 0.5) ** 2 + (Y - 0.5) ** 2)
        P = sfs.image_of_height((1.4 * (X - 0.5)) ** 2 + (1.4 * (Y - 0.5)) ** 2)
        f = eik.sfs_forcing(torch.from_numpy(P.ravel()).cuda(), 1e-3)
        src = np.array([(n // 2) * n + n // 2], dtype=np.int64)
        hbar = 2 * h
        opt = eik.make_options(precision="mixed", tol=1e-9)
        hd = eik.eik_create((n, n), h, hbar, f, src, np.array([z.ravel()[src[0]]]), opt)
        S, _, _ = eik.eik_solve(hd)
        eik.eik_destroy(hd)
        S = S.cpu().numpy().ravel()
        S_ref, _, _ = fd.solve(sfs.forcing(P.ravel(), 1e-3), (n, n), h, hbar, src)
        assert np.max(np.abs(S - S_ref)) <= 1e-6
        errs.append(np.max(np.abs(S - z.ravel())))
        assert errs[-1] <= 15 * hbar
    assert errs[1] < 0.7 * errs[0]
