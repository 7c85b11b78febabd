"""FP64 CUDA path vs the CPU oracle, through the C ABI.

Bar: phi pointwise relative error <= 1e-10 and
S absolute error <= 1e-6 against the oracle's direct (or tight CG) solution.
"""
import numpy as np
import pytest

from oracle import cg, closed_forms, fd
from paper_1403_1937_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PHI_REL = 1e-10
S_ABS = 1e-6


@pytest.fixture(scope="module")
def eik():
    import torch
    from paper_1403_1937_gb300 import build
    build.build()
    from paper_1403_1937_gb300 import eik as e
    assert torch.cuda.is_available()
    return e


def gpu_solve(eik, inst, tol=1e-12, boundary="half_cell", host=False, **kw):
    import torch
    opt = eik.make_options(precision="fp64", tol=tol, boundary=boundary, **kw)
    if host:
        f = np.ascontiguousarray(inst.f)
        src = inst.src_idx
        U = inst.src_U
    else:
        f = torch.from_numpy(np.ascontiguousarray(inst.f)).cuda()
        src = torch.from_numpy(inst.src_idx).cuda()
        U = torch.from_numpy(np.asarray(inst.src_U, dtype=np.float64)).cuda()
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, src, U, opt)
    S, phi, stats = eik.eik_solve(h, want_phi=True)
    eik.eik_destroy(h)
    if not host:
        S, phi = S.cpu().numpy(), phi.cpu().numpy()
    return S.ravel(), phi.ravel(), stats


def check(S, phi, S_ref, phi_ref):
    e_phi = np.max(np.abs(phi / phi_ref - 1))
    e_S = np.max(np.abs(S - S_ref))
    assert e_phi <= PHI_REL, e_phi
    assert e_S <= S_ABS, e_S
    return e_phi, e_S


def test_c1_against_closed_form_and_oracle(eik):
    inst = wl.config1()
    S, phi, stats = gpu_solve(eik, inst)
    ph = closed_forms.image_phi(inst.dims, inst.h, inst.hbar, 1.0, (64, 64)).ravel()
    check(S, phi, -inst.hbar * np.log(ph), ph)
    S_ref, phi_ref, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    check(S, phi, S_ref, phi_ref)
    assert S[inst.src_idx[0]] == 0.0
    assert stats["res_cw"] <= 1e-12
    assert 150 <= stats["inner_iters"] <= 200


@pytest.mark.parametrize("seed,ndim,boundary,with_U", [
    (0, 2, "half_cell", False), (1, 2, "half_cell", True), (2, 2, "drop_edge", False),
    (3, 3, "half_cell", False), (4, 3, "drop_edge", True), (5, 2, "half_cell", True),
    (6, 3, "half_cell", True),
])
def test_random_ragged(eik, seed, ndim, boundary, with_U):
    """Sizes that leave ragged tiles in every direction, random f, faces and
    corners allowed as sources."""
    inst = wl.random_small(400 + seed, ndim=ndim, max_side=150 if ndim == 2 else 40,
                           min_side=3, nsrc_max=6, with_U=with_U,
                           hbar_over_h=(1.0, 6.0))
    S, phi, _ = gpu_solve(eik, inst, boundary=boundary)
    S_ref, phi_ref, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx,
                                   inst.src_U, boundary=1 if boundary == "drop_edge" else 0)
    phi_u = phi * 1.0   # library returns phi * exp(U_min/hbar), as the oracle
    check(S, phi_u, S_ref, phi_ref)
    assert np.array_equal(S[sys.src], sys.U)


@pytest.mark.parametrize("dims,src", [
    ((2, 2), [0]),
    ((2, 2), [0, 1, 2]),                    # one unknown
    ((3, 3), [0, 2, 6, 8]),                 # corners
    ((5, 4), [7, 8]),                       # adjacent sources
    ((65, 2), list(range(0, 130, 65))),     # slab, x = 0 face
    ((2, 2, 2), [7]),
    ((33, 2, 2), [0, 33, 66, 99]),          # 3D slab
    ((64, 32), [5, 5, 5]),                  # exact tile size, duplicate source
    ((65, 33), [64 + 65 * 32]),             # one past the tile, far corner source
    ((3, 2), [0, 1, 2, 3, 4, 5]),           # every node a source: no unknowns
])
def test_edge_cases(eik, dims, src):
    n = int(np.prod(dims))
    inst = wl.Instance(dims, 1.0 / (max(dims) - 1), 0.3 / (max(dims) - 1) * 4,
                       np.random.default_rng(n).uniform(0.5, 2.0, dims[::-1]),
                       np.array(src, dtype=np.int64), np.zeros(len(src)))
    S, phi, _ = gpu_solve(eik, inst)
    S_ref, phi_ref, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    check(S, phi, S_ref, phi_ref)


def test_slab_closed_form(eik):
    n = 300
    dims = (n, 2)
    inst = wl.Instance(dims, 1.0 / (n - 1), 0.004, np.full((2, n), 1.3),
                       np.array([0, n], dtype=np.int64), np.zeros(2))
    S, phi, _ = gpu_solve(eik, inst)
    ex = closed_forms.slab_S(n, 1.3, inst.h, inst.hbar)
    assert np.max(np.abs(S.reshape(2, n) - ex)) < 1e-9


def test_c2_reduced_size(eik):
    inst = wl.config2(n=512)
    S, phi, stats = gpu_solve(eik, inst)
    S_ref, phi_ref, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    check(S, phi, S_ref, phi_ref)


def test_c3_reduced_size(eik):
    inst = wl.config3(n=48)
    S, phi, stats = gpu_solve(eik, inst)
    S_ref, phi_ref, _, info = cg.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx,
                                       tol=1e-13)
    assert info["status"] == 0
    check(S, phi, S_ref, phi_ref)


@pytest.mark.slow
def test_c2_full_size(eik):
    """Config 2 at its full 2048^2 size, in the launch configuration the
    bench uses, against the oracle CG run to 1e-13 componentwise."""
    inst = wl.config2()
    S, phi, stats = gpu_solve(eik, inst)
    S_ref, phi_ref, _, info = cg.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx,
                                       tol=1e-13)
    assert info["status"] == 0
    check(S, phi, S_ref, phi_ref)


@pytest.mark.slow
def test_c3_full_size_properties(eik):
    """Config 3 at 256^3: checked through properties that hold at any size
    (the log-domain identity of every row, evaluated by the oracle's
    assembled matrix, and the M-matrix invariants)."""
    inst = wl.config3()
    S, phi, stats = gpu_solve(eik, inst)
    sys = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    ident = fd.identity_residual(sys, S)
    assert np.max(np.abs(ident)) <= 1e-11
    assert np.all(S[sys.src] == 0) and np.all(S >= 0)
    assert np.all(phi > 0) and np.all(phi <= 1)


def test_host_pointers_match_device(eik):
    inst = wl.random_small(77, ndim=2, max_side=90, min_side=50)
    S_d, phi_d, _ = gpu_solve(eik, inst)
    S_h, phi_h, _ = gpu_solve(eik, inst, host=True)
    assert np.array_equal(S_d, S_h) and np.array_equal(phi_d, phi_h)


def test_deterministic(eik):
    inst = wl.config2(n=300)
    S1, _, s1 = gpu_solve(eik, inst)
    S2, _, s2 = gpu_solve(eik, inst)
    assert np.array_equal(S1, S2) and s1["inner_iters"] == s2["inner_iters"]


def test_normwise_stop_reports_residual(eik):
    inst = wl.config1()
    _, _, stats = gpu_solve(eik, inst, tol=1e-12, stop_norm="normwise")
    # the normwise rule stops far earlier than the componentwise one
    assert stats["inner_iters"] < 120


def test_errors(eik):
    import torch
    from paper_1403_1937_gb300 import _lib
    inst = wl.random_small(9, ndim=2, max_side=20, min_side=10)
    f = torch.from_numpy(inst.f).cuda()
    bad = f.clone()
    bad[3, 4] = -1.0
    with pytest.raises(_lib.EikError) as ei:
        eik.eik_create(inst.dims, inst.h, inst.hbar, bad, inst.src_idx)
    assert ei.value.status == _lib.EIK_ERR_ARG
    bad[3, 4] = float("nan")
    with pytest.raises(_lib.EikError):
        eik.eik_create(inst.dims, inst.h, inst.hbar, bad, inst.src_idx)
    with pytest.raises(_lib.EikError):
        eik.eik_create(inst.dims, inst.h, inst.hbar, f, [0, 0], [0.0, 1.0])
    with pytest.raises(_lib.EikError):
        eik.eik_create(inst.dims, inst.h, inst.hbar, f, [inst.f.size])
    with pytest.raises(_lib.EikError):
        eik.eik_create(inst.dims, -1.0, inst.hbar, f, [0])
    # max_iter -> NOT_CONVERGED, outputs still written
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, inst.src_idx,
                       options=eik.make_options(max_iter=3))
    S, _, st = eik.eik_solve(h, allow_not_converged=True)
    assert st["status"] == _lib.EIK_ERR_NOT_CONVERGED and st["inner_iters"] == 3
    with pytest.raises(_lib.EikError) as ei:
        eik.eik_grad(h, torch.zeros_like(f))
    assert ei.value.status == _lib.EIK_ERR_STATE
    eik.eik_destroy(h)


def test_set_f_reuses_handle(eik):
    import torch
    inst = wl.random_small(12, ndim=2, max_side=60, min_side=40)
    f = torch.from_numpy(inst.f).cuda()
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, inst.src_idx)
    eik.eik_solve(h)
    f2 = f * 1.25
    eik.eik_set_f(h, f2)
    S, _, _ = eik.eik_solve(h)
    S_ref, _, _ = fd.solve(inst.f * 1.25, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(S.cpu().numpy().ravel() - S_ref)) < S_ABS
    eik.eik_destroy(h)


def test_user_stream_ordering(eik):
    """Work is ordered on the caller's stream: f written on a side stream just
    before the call is seen, and S is ready for that stream afterwards."""
    import torch
    inst = wl.random_small(13, ndim=2, max_side=80, min_side=60)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        f = torch.from_numpy(inst.f).cuda(non_blocking=False)
        f2 = f * 1.0
        h = eik.eik_create(inst.dims, inst.h, inst.hbar, f2, inst.src_idx, stream=s)
        S, _, _ = eik.eik_solve(h)
        S2 = S * 2.0
    torch.cuda.synchronize()
    S_ref, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(S2.cpu().numpy().ravel() / 2.0 - S_ref)) < S_ABS
    eik.eik_destroy(h)


@pytest.mark.parametrize("ndim", [2, 3])
def test_adjoint_fp64_vs_oracle(eik, ndim):
    import torch
    inst = wl.random_small(500 + ndim, ndim=ndim, max_side=40 if ndim == 2 else 14,
                           min_side=8, nsrc_max=2, hbar_over_h=(1.0, 3.0))
    f = torch.from_numpy(inst.f).cuda()
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, inst.src_idx,
                       options=eik.make_options(tol=1e-13))
    S, _, _ = eik.eik_solve(h)
    rng = np.random.default_rng(ndim)
    v = rng.standard_normal(inst.f.shape)
    g, st = eik.eik_grad(h, torch.from_numpy(v).cuda())
    eik.eik_destroy(h)
    sys = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    g_ref = fd.grad_f(sys, v.ravel())
    g = g.cpu().numpy().ravel()
    assert np.max(np.abs(g - g_ref)) <= 1e-8 * np.max(np.abs(g_ref))
