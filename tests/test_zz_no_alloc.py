"""eik_residual_noalloc, the entry point for callers that cannot allocate
device memory (memory pools that must not grow, allocator hooks, real-time
loops): its result is checked against the componentwise residual that the
existing entry point eik_solve reports for the same solution, on two calls in
a row with different grids (the shared working memory keeps the previous
call's contents, so the second call must not see them).

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

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
