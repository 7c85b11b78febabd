"""Adjoint dL/df through torch.autograd (hand-written adjoint in the CUDA
library) against the FP64 oracle gradient and central finite differences.

Loss (config 5 structure): L = sum over receiver nodes of (S(x_i) - T_i)^2,
T_i = S_ref(x_i) + noise, with S_ref the oracle solution for a separately
seeded reference field.
"""
import numpy as np
import pytest

from oracle import fd
from paper_1403_1937_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    from paper_1403_1937_gb300 import build
    build.build()
    from paper_1403_1937_gb300 import autograd, eik
    assert torch.cuda.is_available()
    return torch, autograd, eik


def c5_case(n=192, k=0):
    inst, recv, f_ref, eps = wl.config5(count=k + 1, n=n, nrecv=512)[k]
    S_ref, _, _ = fd.solve(f_ref, inst.dims, inst.h, inst.hbar, inst.src_idx)
    T = S_ref[recv] + eps
    return inst, recv, T


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autograd_matches_oracle_gradient(mods, precision):
    torch, autograd, eik = mods
    inst, recv, T = c5_case()
    layer = autograd.Eikonal(inst.dims, inst.h, inst.hbar, inst.src_idx,
                             precision=precision, tol=1e-12 if precision == "fp64" else 1e-9)
    f = torch.from_numpy(inst.f).cuda().requires_grad_(True)
    S = layer(f)
    recv_t = torch.from_numpy(recv).cuda()
    T_t = torch.from_numpy(T).cuda()
    L = ((S.reshape(-1)[recv_t] - T_t) ** 2).sum()
    L.backward()
    g = f.grad.cpu().numpy().ravel()
    # oracle: dL/dS = 2 (S - T) on the receivers
    S_o, _, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    dLdS = np.zeros(sys.n)
    dLdS[recv] = 2.0 * (S_o[recv] - T)
    g_ref = fd.grad_f(sys, dLdS)
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) <= (1e-8 if precision == "fp64" else 1e-6) * scale
    assert np.all(g[sys.src] == 0)
    layer.close()


def test_autograd_central_difference(mods):
    torch, autograd, eik = mods
    inst, recv, T = c5_case(n=160, k=0)
    layer = autograd.Eikonal(inst.dims, inst.h, inst.hbar, inst.src_idx, tol=1e-13)
    recv_t = torch.from_numpy(recv).cuda()
    T_t = torch.from_numpy(T).cuda()

    def loss(fv):
        S = layer(fv)
        return ((S.reshape(-1)[recv_t] - T_t) ** 2).sum()

    f = torch.from_numpy(inst.f).cuda().requires_grad_(True)
    L = loss(f)
    L.backward()
    g = f.grad.detach()
    rng = np.random.default_rng(7)
    d = torch.from_numpy(rng.standard_normal(inst.f.shape)).cuda()
    eps = 1e-5
    with torch.no_grad():
        Lp = loss(f.detach() + eps * d).item()
        Lm = loss(f.detach() - eps * d).item()
    fdv = (Lp - Lm) / (2 * eps)
    ad = float((g * d).sum())
    assert abs(ad - fdv) <= 1e-6 * abs(fdv)
    # single-node checks on receivers' neighbourhoods
    gi = g.reshape(-1)
    for node in recv[:8]:
        e = torch.zeros_like(f).reshape(-1)
        e[int(node)] = 1.0
        e = e.reshape(f.shape)
        with torch.no_grad():
            Lp = loss(f.detach() + eps * e).item()
            Lm = loss(f.detach() - eps * e).item()
        fdn = (Lp - Lm) / (2 * eps)
        assert abs(float(gi[int(node)]) - fdn) <= 1e-5 * max(abs(fdn), 1e-8 * abs(fdv))
    layer.close()


def test_backward_after_second_forward_is_rejected(mods):
    torch, autograd, eik = mods
    inst = wl.random_small(31, ndim=2, max_side=30, min_side=20)
    layer = autograd.Eikonal(inst.dims, inst.h, inst.hbar, inst.src_idx)
    f = torch.from_numpy(inst.f).cuda().requires_grad_(True)
    S1 = layer(f)
    S2 = layer(f * 1.01)
    with pytest.raises(RuntimeError):
        S1.sum().backward()
    layer.close()


@pytest.mark.slow
def test_full_size_c5_gradient_vs_oracle(mods):
    """One instance of the differentiation workload at its full size (512^2,
    4096 receivers): forward in mixed precision, hand-written adjoint, against
    the oracle's gradient through the same factorisation."""
    torch, autograd, eik = mods
    inst, recv, f_ref, eps = wl.config5(count=1)[0]
    S_ref, _, _ = fd.solve(f_ref, inst.dims, inst.h, inst.hbar, inst.src_idx)
    T = S_ref[recv] + eps
    layer = autograd.Eikonal(inst.dims, inst.h, inst.hbar, inst.src_idx, precision="mixed",
                             tol=1e-9)
    f = torch.from_numpy(inst.f).cuda().requires_grad_(True)
    S = layer(f)
    recv_t = torch.from_numpy(recv).cuda()
    L = ((S.reshape(-1)[recv_t] - torch.from_numpy(T).cuda()) ** 2).sum()
    L.backward()
    g = f.grad.cpu().numpy().ravel()
    S_o, _, sys = fd.solve(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    dLdS = np.zeros(sys.n)
    dLdS[recv] = 2.0 * (S_o[recv] - T)
    g_ref = fd.grad_f(sys, dLdS)
    assert np.max(np.abs(g - g_ref)) <= 1e-6 * np.max(np.abs(g_ref))
    layer.close()
