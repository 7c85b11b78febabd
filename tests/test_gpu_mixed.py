"""Mixed-precision path (FP32 single-reduction inner CG in per-cell exponent
units + FP64 iterative refinement) vs the CPU oracle, through the C ABI.

Bar: S absolute error <= 1e-6 against the FP64 oracle, on every
config, including problems whose phi underflows float64 (S/hbar > 700), where
the oracle uses its relative-form direct solve.
"""
import numpy as np
import pytest

from oracle import cg, fd
from paper_1403_1937_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

S_ABS = 1e-6


@pytest.fixture(scope="module")
def eik():
    import torch
    from paper_1403_1937_gb300 import build
    build.build()
    from paper_1403_1937_gb300 import eik as e
    assert torch.cuda.is_available()
    return e


def mixed_solve(eik, inst, tol=1e-9, boundary="half_cell", want_phi=False, band_bits=0):
    import torch
    opt = eik.make_options(precision="mixed", tol=tol, boundary=boundary, band_bits=band_bits)
    f = torch.from_numpy(np.ascontiguousarray(inst.f)).cuda()
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, inst.src_idx, inst.src_U, opt)
    S, phi, stats = eik.eik_solve(h, want_phi=want_phi)
    kst = eik.eik_kernel_stats(h)
    eik.eik_destroy(h)
    return S.cpu().numpy().ravel(), (phi.cpu().numpy().ravel() if want_phi else None), stats, kst


def test_c1_mixed(eik):
    inst = wl.config1()
    S, phi, stats, kst = mixed_solve(eik, inst, want_phi=True)
    S_ref, phi_ref, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(S - S_ref)) <= S_ABS
    assert S[inst.src_idx[0]] == 0.0
    assert stats["res_cw"] <= 1e-9
    assert kst["mixed_cg_init"][0] > 0 and kst["mixed_cg"][0] > 0
    assert kst["cg_pass1_64"][0] == 0      # the FP64 CG did not run


def test_c1_mixed_bench_tolerance(eik):
    """Config 1 in mixed precision at the bench's componentwise tolerance
    1e-6: S within 1e-6 of the direct oracle everywhere (including the far
    corners, where phi ~ 1e-31)."""
    inst = wl.config1()
    S, _, stats, _ = mixed_solve(eik, inst, tol=1e-6)
    S_ref, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert stats["res_cw"] <= 1e-6
    assert np.max(np.abs(S - S_ref)) <= S_ABS
    assert S[inst.src_idx[0]] == 0.0


@pytest.mark.parametrize("seed,ndim,boundary,with_U", [
    (0, 2, "half_cell", False), (1, 2, "drop_edge", True), (2, 3, "half_cell", False),
    (3, 3, "half_cell", True), (4, 2, "half_cell", False),
])
def test_random_ragged_mixed(eik, seed, ndim, boundary, with_U):
    inst = wl.random_small(600 + seed, ndim=ndim, max_side=150 if ndim == 2 else 40,
                           min_side=3, nsrc_max=6, with_U=with_U, hbar_over_h=(1.0, 6.0))
    S, _, _, _ = mixed_solve(eik, inst, boundary=boundary)
    S_ref, _, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx, inst.src_U,
                             boundary=1 if boundary == "drop_edge" else 0)
    assert np.max(np.abs(S - S_ref)) <= S_ABS
    assert np.array_equal(S[sys.src], sys.U)


def test_c2_reduced_mixed(eik):
    inst = wl.config2(n=512)
    S, _, stats, _ = mixed_solve(eik, inst)
    S_ref, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(S - S_ref)) <= S_ABS


def test_c3_reduced_mixed(eik):
    inst = wl.config3(n=48)
    S, _, _, _ = mixed_solve(eik, inst)
    S_ref, _, _, info = cg.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx, tol=1e-13)
    assert np.max(np.abs(S - S_ref)) <= S_ABS


@pytest.mark.parametrize("n,mult,corner", [(400, 2, True), (300, 2, False)])
def test_underflowing_phi(eik, n, mult, corner):
    """hbar = 2h with f up to 1.5: S/hbar reaches a few hundred, so phi
    underflows FP32 far below its range; the oracle solves the diagonally
    similar relative form."""
    rng = np.random.default_rng(n + mult)
    dims = (n, n)
    h = 1.0 / (n - 1)
    f = wl.fourier_field(rng, dims, h)
    src = np.array([0 if corner else n * (n // 2) + n // 2], dtype=np.int64)
    inst = wl.Instance(dims, h, mult * h, f, src, np.zeros(1))
    S, _, stats, _ = mixed_solve(eik, inst)
    sys = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    S_ref = fd.solve_relative(sys)
    assert np.max(S_ref) / inst.hbar > 100
    assert np.max(np.abs(S - S_ref)) <= S_ABS


@pytest.mark.slow
def test_c2_full_size_mixed(eik):
    """Config 2 at 2048^2 in the bench's configuration (tol 1e-6)."""
    inst = wl.config2()
    S, _, stats, _ = mixed_solve(eik, inst, tol=1e-6)
    S_ref, _, _, info = cg.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx,
                                 tol=1e-13)
    assert info["status"] == 0
    assert np.max(np.abs(S - S_ref)) <= S_ABS


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bench_tolerance_meets_S_bound(eik, precision):
    """Both precision modes at the bench tolerance (componentwise 1e-6) meet
    S <= 1e-6 against the direct oracle (config 2 structure at 768^2)."""
    import torch
    inst = wl.config2(n=768)
    opt = eik.make_options(precision=precision, tol=1e-6)
    f = torch.from_numpy(inst.f).cuda()
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, inst.src_idx, None, opt)
    S, _, _ = eik.eik_solve(h)
    eik.eik_destroy(h)
    S_ref, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(S.cpu().numpy().ravel() - S_ref)) <= S_ABS


@pytest.mark.parametrize("k", [43, 132])
def test_level_set_sweep_large_range(eik, k):
    """Config-4 instances with hbar = 2h whose phi spans far more than 2^96
    (S/hbar up to ~300): one global CG, FP32 or FP64 (the oracle's own CG
    stalls on such instances), does not reach them; the mixed path sweeps
    level-set bands of the distance estimate.  Checked against the oracle's
    relative-form direct solve."""
    inst = wl.config4()[k]
    S, _, stats, _ = mixed_solve(eik, inst, tol=1e-7)
    sys = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx, inst.src_U)
    S_ref = fd.solve_relative(sys)
    assert np.max(S_ref) / inst.hbar > 90
    assert np.max(np.abs(S - S_ref)) <= S_ABS
    assert np.array_equal(S[sys.src], sys.U)


@pytest.mark.parametrize("band_bits", [-1, 0, 24])
def test_band_width_does_not_change_the_solution(eik, band_bits):
    """Config 2 structure at 512^2: without sweeps, with the default bands and
    with narrow bands, S meets the same bound against the oracle."""
    inst = wl.config2(n=512)
    S, _, stats, _ = mixed_solve(eik, inst, tol=1e-8, band_bits=band_bits)
    S_ref, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(S - S_ref)) <= S_ABS
    assert stats["res_cw"] <= 1e-8


def test_bounded_wait_timeout_is_reported(eik):
    """Failure detection without a fault: with test_flags bit 0 one warp of
    the first inner iteration never gets its row copy; its bounded wait expires,
    the kernel sets the fault flag, waits (bounded) for its own copies in
    flight and returns; the solve reports EIK_ERR_TIMEOUT and the GPU context
    stays usable for the next solve."""
    import torch
    from paper_1403_1937_gb300 import _lib
    inst = wl.config2(n=256)
    f = torch.from_numpy(inst.f).cuda()
    opt = eik.make_options(precision="mixed", tol=1e-6, test_flags=1)
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, inst.src_idx, None, opt)
    with pytest.raises(_lib.EikError) as ei:
        eik.eik_solve(h)
    assert ei.value.status == _lib.EIK_ERR_TIMEOUT
    assert "timed out" in str(ei.value)
    eik.eik_destroy(h)
    S, _, stats, _ = mixed_solve(eik, inst, tol=1e-8)
    S_ref, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(S - S_ref)) <= S_ABS


@pytest.mark.parametrize("ndim,tile_override", [
    (2, 0), (2, 1), (2, 2), (2, 3), (2, 4), (3, 0), (3, 1), (3, 2), (3, 3), (3, 4)])
def test_kernel_variants_agree_with_oracle(eik, ndim, tile_override):
    """Every inner-CG kernel variant (2D: warps per block and stage depth;
    3D: rows per tile and plane stages) meets the S bound."""
    inst = wl.config2(n=264) if ndim == 2 else wl.config3(n=40)
    import torch
    opt = eik.make_options(precision="mixed", tol=1e-9, tile_override=tile_override)
    f = torch.from_numpy(np.ascontiguousarray(inst.f)).cuda()
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, inst.src_idx, None, opt)
    S, _, stats = eik.eik_solve(h)
    eik.eik_destroy(h)
    S_ref, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(S.cpu().numpy().ravel() - S_ref)) <= S_ABS


@pytest.mark.parametrize("dims,tile_override", [((263, 131), 1), ((263, 131), 4),
                                                ((130, 7), 3), ((41, 23, 19), 1),
                                                ((41, 23, 19), 3), ((131, 5, 9), 2)])
def test_tma_kernels_on_odd_widths(eik, dims, tile_override):
    """The inner-CG kernels on grids whose width is not a multiple of 4 (the
    FP32 arrays get a padded row pitch), with ragged last tiles in every
    direction and tiles wider or taller than the grid."""
    import torch
    rng = np.random.default_rng(sum(dims))
    h = 1.0 / (max(dims) - 1)
    f = wl.fourier_field(rng, dims, h)
    src = wl.random_sources(rng, int(np.prod(dims)), 3)
    inst = wl.Instance(dims, h, 4 * h, f, src, np.zeros(len(src)))
    opt = eik.make_options(precision="mixed", tol=1e-9, tile_override=tile_override)
    hd = eik.eik_create(inst.dims, inst.h, inst.hbar, torch.from_numpy(inst.f).cuda(),
                        inst.src_idx, None, opt)
    S, _, _ = eik.eik_solve(hd)
    eik.eik_destroy(hd)
    S_ref, _, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(S.cpu().numpy().ravel() - S_ref)) <= S_ABS


@pytest.mark.parametrize("dims,src", [
    ((2, 2), [0, 1, 2]),                    # one unknown
    ((3, 3), [0, 2, 6, 8]),                 # corners
    ((5, 4), [7, 8]),                       # adjacent sources
    ((65, 2), list(range(0, 130, 65))),     # slab, x = 0 face
    ((2, 2, 2), [7]),
    ((33, 2, 2), [0, 33, 66, 99]),          # 3D slab
    ((128, 16), [5, 5, 5]),                 # exactly one TMA tile, duplicate source
    ((129, 17), [128 + 129 * 16]),          # one past the tile, far corner source
    ((3, 2), [0, 1, 2, 3, 4, 5]),           # every node a source: no unknowns
])
def test_edge_cases_mixed(eik, dims, src):
    n = int(np.prod(dims))
    inst = wl.Instance(dims, 1.0 / (max(dims) - 1), 0.3 / (max(dims) - 1) * 4,
                       np.random.default_rng(n).uniform(0.5, 2.0, dims[::-1]),
                       np.array(src, dtype=np.int64), np.zeros(len(src)))
    S, _, stats, _ = mixed_solve(eik, inst)
    if len(set(src)) == n:
        assert np.all(S == 0.0)
        return
    S_ref, _, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    assert np.max(np.abs(S - S_ref)) <= S_ABS
    assert np.array_equal(S[sys.src], sys.U)
