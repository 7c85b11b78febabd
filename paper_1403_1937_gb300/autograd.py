"""torch.autograd wrapper: S = Eikonal(f), with the hand-written adjoint.

Forward: eik_set_f + eik_solve.  Backward: eik_grad, one extra solve of the
same symmetric stencil system for the adjoint, giving dL/df (see
``include/eik.h``, eik_grad).  The layer keeps one library handle; the state
kept for the backward pass is that of the last forward, so each backward must
follow its own forward before the layer is called again (checked).
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import eik


class _EikonalFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f: torch.Tensor, layer: "Eikonal"):
        layer._ensure(f)
        eik.eik_set_f(layer.handle, f.detach().contiguous())
        S, _, stats = eik.eik_solve(layer.handle)
        layer.last_stats = stats
        layer._version += 1
        ctx.layer = layer
        ctx.version = layer._version
        return S

    @staticmethod
    def backward(ctx, dS: torch.Tensor):
        layer = ctx.layer
        if layer._version != ctx.version:
            raise RuntimeError("Eikonal layer was called again before this backward; "
                               "the adjoint needs the state of its own forward")
        g, stats = eik.eik_grad(layer.handle, dS.contiguous().to(torch.float64))
        layer.last_grad_stats = stats
        return g, None


class Eikonal:
    """Differentiable solve S(f) for fixed grid, sources, h and hbar.

    ``f`` is a CUDA float64 tensor of shape dims[::-1]; the result has the same
    shape.  ``precision`` is 'fp64' or 'mixed' for the forward solve (the
    adjoint solve is FP64)."""

    def __init__(self, dims: Sequence[int], h: float, hbar: float, src_idx, src_U=None,
                 precision: str = "fp64", tol: float = 1e-12, **opts):
        self.dims = tuple(int(d) for d in dims)
        self.h = float(h)
        self.hbar = float(hbar)
        self.src_idx = src_idx
        self.src_U = src_U
        self.options = eik.make_options(precision=precision, tol=tol, **opts)
        self.handle: Optional[eik.Handle] = None
        self._version = 0
        self.last_stats = None
        self.last_grad_stats = None

    def _ensure(self, f):
        if self.handle is None:
            self.handle = eik.eik_create(self.dims, self.h, self.hbar, f.detach().contiguous(),
                                         self.src_idx, self.src_U, self.options)

    def __call__(self, f: torch.Tensor) -> torch.Tensor:
        return _EikonalFn.apply(f, self)

    def close(self):
        if self.handle is not None:
            eik.eik_destroy(self.handle)
            self.handle = None
