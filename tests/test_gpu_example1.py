"""Example 1 of Sec. 5.4 as a workload of the CUDA path: f = exp(r) on
[-0.125, 0.125]^2 with h = 2^-10, one source at the origin, hbar = 0.006,
whose exact eikonal solution is R = exp(r) - 1.

The finite-difference S of the GPU (FP64 and mixed precision, through the C
ABI) must match the oracle's direct solution at the tolerances of the other
parity tests.  Its accuracy against R -- the percentage error Lambda of
Eq. (percentError) and the largest difference -- is then reported beside the
figures the paper prints for its FFT perturbation series and for fast
sweeping (Table eikonalexp1, tests/golden/example1_paper.json).  Those come
from different solvers, so they are context, not parity.  The finite-
difference path with the Dirichlet source S(0) = 0 has Lambda of about 17 %
against the paper's 1.36 %: near the origin R -> 0 while S carries the
logarithmic term of the point source (a few hbar), so the mean relative error
is dominated by the nodes next to the source, and the largest absolute
difference (about 2.7 hbar = 0.016) is eight times the paper's 0.0021.
"""
import json
import os

import numpy as np
import pytest

from oracle import fd
from paper_1403_1937_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "example1_paper.json")


@pytest.fixture(scope="module")
def eik():
    import torch
    from paper_1403_1937_gb300 import build
    build.build()
    from paper_1403_1937_gb300 import eik as e
    assert torch.cuda.is_available()
    return e


def accuracy(S, inst):
    """Lambda (Eq. percentError: mean of |S - R| / R in percent over the nodes
    with R > 0) and max |S - R| against R = exp(r) - 1."""
    n = inst.dims[0]
    x = -0.125 + np.arange(n) * inst.h
    X, Y = np.meshgrid(x, x)
    R = np.exp(np.hypot(X, Y)) - 1
    d = np.abs(S.reshape(n, n) - R)
    m = R > 0
    return 100.0 * float(np.mean(d[m] / R[m])), float(d.max())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_example1_gpu(eik, precision, tol):
    import torch
    gold = json.load(open(GOLDEN))
    inst = wl.example1()
    assert inst.dims == (257, 257) and inst.hbar == gold["setup"]["hbar"]
    S_ref, phi_ref, _ = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    opt = eik.make_options(precision=precision, tol=tol)
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, torch.from_numpy(inst.f).cuda(),
                       inst.src_idx, None, opt)
    S, phi, stats = eik.eik_solve(h, want_phi=True)
    eik.eik_destroy(h)
    S = S.cpu().numpy().ravel()
    assert np.max(np.abs(S - S_ref)) <= 1e-6
    if precision == "fp64":
        assert np.max(np.abs(phi.cpu().numpy().ravel() / phi_ref - 1)) <= 1e-10
    lam, mx = accuracy(S, inst)
    lam_ref, mx_ref = accuracy(S_ref, inst)
    # the GPU reproduces the oracle's accuracy figures
    assert abs(lam - lam_ref) <= 1e-4 * lam_ref and abs(mx - mx_ref) <= 1e-6
    print(f"\nExample 1 ({precision}): Lambda = {lam:.4f} %, max |S - R| = {mx:.5f}; "
          f"paper, FFT perturbation (6 terms): {gold['perturbation_percent_error'][-1]} %, "
          f"{gold['perturbation_max_diff'][-1]}; fast sweeping: "
          f"{gold['fast_sweeping_percent_error']} %")
    # the absolute difference stays within a few hbar (source log term)
    assert mx < 5 * inst.hbar
