"""eik_residual_noalloc, the entry point for callers that cannot allocate
device memory (memory pools that must not grow, allocator hooks, real-time
loops): its result is checked against the componentwise residual that the
existing entry point eik_solve reports for the same solution, and against
the CPU oracle's log-domain row defect of the same S, on two calls in a row
with different grids (the shared working memory keeps the previous call's
contents, so the second call must not see them).  A NaN anywhere in S must
come back as NaN, not as a small residual.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from oracle import fd
from paper_1403_1937_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# Both sides evaluate |r_i| / (a_i phi_i) in float64: the solver from its own
# iterate, the new entry point from S = -hbar log(phi).  Rounding S costs
# about 1e-16 * (S / hbar) in each exponent, so 1e-6 relative on residuals of
# 1e-7..1e-9 leaves a wide margin.
REL_TOL = 1e-6


@pytest.fixture(scope="module")
def eik():
    import torch
    from paper_1403_1937_gb300 import build
    build.build()
    from paper_1403_1937_gb300 import eik as e
    assert torch.cuda.is_available()
    return e


def solve_and_check(eik, inst, tol):
    import torch
    f = torch.from_numpy(np.ascontiguousarray(inst.f)).cuda()
    src = torch.from_numpy(inst.src_idx).cuda()
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, src, None,
                       eik.make_options(precision="fp64", tol=tol))
    S, _, stats = eik.eik_solve(h)
    eik.eik_destroy(h)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    eik.eik_residual_noalloc(inst.dims, inst.h, inst.hbar, f, S, src, out)
    torch.cuda.synchronize()
    got = float(out.item())
    want = stats["res_cw"]
    assert 0.0 < want <= tol
    assert abs(got - want) <= REL_TOL * want + 1e-13, (got, want)
    # the same quantity from the oracle: max over the unknowns of the row
    # defect of Eq. phiEquation divided by a_i phi_i, evaluated from S alone
    sys = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    ref = float(np.max(np.abs(fd.identity_residual(sys, S.cpu().numpy().ravel()))))
    assert abs(got - ref) <= REL_TOL * ref + 1e-13, (got, ref)
    return got


def test_noalloc_matches_solver_residual_two_calls(eik):
    first = solve_and_check(eik, wl.random_small(71, ndim=2, max_side=300, min_side=200,
                                                 nsrc_max=3), 1e-7)
    second = solve_and_check(eik, wl.random_small(72, ndim=3, max_side=40, min_side=24,
                                                  nsrc_max=2), 1e-9)
    assert first != second


def test_noalloc_rejects_grids_beyond_its_working_memory(eik):
    import torch
    from paper_1403_1937_gb300 import _lib
    dims = (1025, 1024)                      # 2^20 + 1024 nodes: one row too many
    f = torch.ones(dims[::-1], dtype=torch.float64, device="cuda")
    src = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.EikError) as ei:
        eik.eik_residual_noalloc(dims, 1e-3, 1e-2, f, f, src, out)
    assert ei.value.status == _lib.EIK_ERR_ARG


def test_noalloc_returns_nan_for_nan_in_S(eik):
    """One NaN entry of S (or two adjacent +inf entries, whose difference is
    NaN) makes the result NaN; the reduction must not drop it."""
    import torch
    inst = wl.random_small(73, ndim=2, max_side=90, min_side=60, nsrc_max=2)
    f = torch.from_numpy(np.ascontiguousarray(inst.f)).cuda()
    src = torch.from_numpy(inst.src_idx).cuda()
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, src, None,
                       eik.make_options(precision="fp64", tol=1e-9))
    S, _, _ = eik.eik_solve(h)
    eik.eik_destroy(h)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    Sv = S.reshape(-1)
    unk = np.setdiff1d(np.arange(inst.n), inst.src_idx)
    for k, bad in ((int(unk[len(unk) // 2]), float("nan")), (int(unk[-1]), float("nan"))):
        S2 = Sv.clone()
        S2[k] = bad
        eik.eik_residual_noalloc(inst.dims, inst.h, inst.hbar, f, S2, src, out)
        torch.cuda.synchronize()
        assert np.isnan(float(out.item())), k
    # two neighbours at +inf: inf - inf is NaN in the exponent
    nx = inst.dims[0]
    cand = [int(k) for k in unk if k % nx < nx - 2 and k + 1 not in set(inst.src_idx.tolist())]
    i = cand[len(cand) // 3]                 # i and i + 1 lie in the same row
    S3 = Sv.clone()
    S3[i] = float("inf")
    S3[i + 1] = float("inf")
    eik.eik_residual_noalloc(inst.dims, inst.h, inst.hbar, f, S3, src, out)
    torch.cuda.synchronize()
    assert np.isnan(float(out.item()))
    # and a clean S afterwards is finite again (nothing sticks in the scratch)
    eik.eik_residual_noalloc(inst.dims, inst.h, inst.hbar, f, Sv, src, out)
    torch.cuda.synchronize()
    assert np.isfinite(float(out.item())) and float(out.item()) <= 1e-9
