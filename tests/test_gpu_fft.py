"""FFT perturbation series (Sec. 5, Table 1) through the C ABI against the
oracle (oracle/fft_series.py) on the same inputs.

Tolerance: the two sides run the same steps with different FP64 transforms
(the oracle numpy's, the library its own radix-2), so each convolution
differs by rounding of order eps log2(P) times the largest value it carries;
phi is compared with an absolute bound eta = 1e-13 max|phi|, and S = -hbar
log phi with hbar eta / phi (plus 1e-12), which is how far the transforms'
rounding lets S be determined at all (the paper's reason for MPFR at small
hbar, Sec. 5, Numerical issues)."""
import json
import os

import numpy as np
import pytest

from oracle import fft_series as fs
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


def check(S, phi, S_ref, phi_ref, hbar):
    eta = 1e-13 * np.max(np.abs(phi_ref))
    assert np.max(np.abs(phi - phi_ref)) <= eta
    ok = phi_ref > 0
    bound = hbar * eta / phi_ref[ok] + 1e-12
    assert np.all(np.abs(S[ok] - S_ref[ok]) <= bound)


@pytest.mark.parametrize("terms", [0, 1, 3, 6])
def test_example1_vs_oracle(eik, terms):
    import torch
    inst = wl.example1()
    n = inst.dims[0]
    S_ref, phi_ref, _, ft_ref = fs.series(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx,
                                          terms)
    S, phi, ft = eik.fft_series(inst.dims, inst.h, inst.hbar, torch.from_numpy(inst.f).cuda(),
                                inst.src_idx, terms)
    assert ft == pytest.approx(ft_ref, rel=1e-15)
    check(S.cpu().numpy(), phi.cpu().numpy(), S_ref, phi_ref, inst.hbar)
    if terms == 6:
        gold = json.load(open(GOLDEN))
        x = -0.125 + np.arange(n) * inst.h
        X, Y = np.meshgrid(x, x)
        R = (np.exp(np.hypot(X, Y)) - 1).ravel()
        m = R > 0
        lam = 100 * np.mean(np.abs(S.cpu().numpy() - R)[m] / R[m])
        lam_ref = 100 * np.mean(np.abs(S_ref - R)[m] / R[m])
        assert abs(lam - lam_ref) <= 1e-6 * lam_ref
        print(f"\nExample 1, FFT series, T = 6: Lambda = {lam:.4f} % (paper: "
              f"{gold['perturbation_percent_error'][-1]} %)")


@pytest.mark.parametrize("f_tilde", [0.0, 1.4])
def test_ragged_grid_many_sources(eik, f_tilde):
    """Non-square grid (both axes not powers of two), several sources,
    Fourier f, with the optimal and with a given f~ (host inputs)."""
    rng = np.random.default_rng(17)
    nx, ny = 151, 90
    h = 1.0 / (nx - 1)
    f = wl.fourier_field(rng, (nx, ny), h)
    src = wl.random_sources(rng, nx * ny, 5)
    hbar = 0.02
    S_ref, phi_ref, _, ft_ref = fs.series(f, (nx, ny), h, hbar, src, 4, ft=f_tilde)
    S, phi, ft = eik.fft_series((nx, ny), h, hbar, f, src, 4, f_tilde=f_tilde)
    assert ft == pytest.approx(ft_ref, rel=1e-15)
    check(np.asarray(S), np.asarray(phi), S_ref, phi_ref, hbar)


def test_constant_f_closed_form(eik):
    """f = f~: the series is phi_0 = sum_k exp(-f~ |x - y_k| / hbar)
    (Eq. STilde with C = 1) whatever the number of terms."""
    nx, ny, h, hbar = 70, 45, 0.01, 0.05
    f = np.full((ny, nx), 0.8)
    src = np.array([3 + nx * 2, 60 + nx * 40, 33 + nx * 20], dtype=np.int64)
    S, phi, ft = eik.fft_series((nx, ny), h, hbar, f, src, 3)
    assert ft == pytest.approx(0.8)
    X, Y = np.meshgrid(np.arange(nx) * h, np.arange(ny) * h)
    ref = sum(np.exp(-0.8 * np.hypot(X - (k % nx) * h, Y - (k // nx) * h) / hbar) for k in src)
    ref = ref.ravel()
    eta = 1e-13 * ref.max()
    assert np.max(np.abs(np.asarray(phi) - ref)) <= eta
    assert np.all(np.abs(np.asarray(S) + hbar * np.log(ref)) <= hbar * eta / ref + 1e-12)


def test_invalid_f_rejected(eik):
    from paper_1403_1937_gb300 import _lib
    f = np.ones((8, 8))
    f[3, 3] = -1.0
    with pytest.raises(_lib.EikError):
        eik.fft_series((8, 8), 0.1, 0.1, f, [0], 2)
