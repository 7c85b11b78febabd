"""Batched solves (config 4 structure: uneven 2D instances with their own f,
sources and hbar) vs the oracle per instance, and vs single-instance solves."""
import numpy as np
import pytest

from oracle import fd
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


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_small_c4(eik, precision):
    insts = wl.config4(count=12, side=(48, 200))
    if precision == "fp64":
        # the plain FP64 path needs phi above the float64 range: hbar >= 4h here
        insts = [i for i in insts if i.hbar >= 4 * i.h]
    opt = eik.make_options(precision=precision, tol=1e-7)
    b = eik.eik_create_batch(insts, opt)
    S, stats = eik.eik_solve_batch(b)
    parts = b.split(S.cpu().numpy())
    for inst, Si in zip(insts, parts):
        sys = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
        S_ref = fd.solve_relative(sys)
        assert np.max(np.abs(Si.ravel() - S_ref)) <= 1e-6, inst.name
    assert all(s["inner_iters"] > 0 for s in stats)
    eik.eik_destroy_batch(b)


def test_batch_equals_single_solves(eik):
    """Per-instance batches (each instance on its own stream) run exactly the
    single-solve kernels: bit-identical results."""
    import torch
    insts = wl.config4(count=5, side=(64, 160))
    opt = eik.make_options(precision="mixed", tol=1e-7, batch_pack=-1)
    b = eik.eik_create_batch(insts, opt, workers=3)
    S, _ = eik.eik_solve_batch(b)
    parts = b.split(S.cpu().numpy())
    for inst, Si in zip(insts, parts):
        h = eik.eik_create(inst.dims, inst.h, inst.hbar, torch.from_numpy(inst.f).cuda(),
                           inst.src_idx, None, opt)
        S1, _, _ = eik.eik_solve(h)
        eik.eik_destroy(h)
        assert np.array_equal(S1.cpu().numpy(), Si)
    eik.eik_destroy_batch(b)


def test_batch_errors(eik):
    from paper_1403_1937_gb300 import _lib
    insts = wl.config4(count=3, side=(20, 40))
    insts[1].src_idx = np.array([10 ** 9], dtype=np.int64)   # out of range
    with pytest.raises(_lib.EikError) as ei:
        eik.eik_create_batch(insts)
    assert "instance 1" in str(ei.value)
