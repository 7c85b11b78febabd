"""Python binding with the names of the C ABI (``include/eik.h``).

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they must be
contiguous float64 (int64 for source indices).  Device tensors are passed to
the library as device pointers, host arrays as host pointers; the library
copies host data itself.  Work is ordered on ``torch.cuda.current_stream()``
unless another stream is given.  This module only marshals arguments; the
solve runs in libeik.so.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence, Tuple

import numpy as np

from . import _lib

try:  # torch provides device memory and streams; optional for host use
    import torch
except Exception:  # pragma: no cover
    torch = None


def _is_torch(a) -> bool:
    return torch is not None and isinstance(a, torch.Tensor)


def _ptr(a, dtype, name: str):
    """(pointer, keepalive) for a contiguous array of ``dtype``."""
    if a is None:
        return None, None
    if _is_torch(a):
        want = torch.float64 if dtype == np.float64 else torch.int64
        if a.dtype != want:
            raise TypeError(f"{name} must be {want}")
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.asarray(a)
    if arr.dtype != dtype:
        raise TypeError(f"{name} must be {np.dtype(dtype).name}")
    if not arr.flags.c_contiguous:
        raise ValueError(f"{name} must be C-contiguous")
    return ctypes.c_void_p(arr.ctypes.data), arr


def _numel(a) -> int:
    return int(a.numel()) if _is_torch(a) else int(np.asarray(a).size)


def _stream_ptr(stream):
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    if torch is not None and torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def make_options(precision: str = "fp64", tol: Optional[float] = None,
                 stop_norm: str = "componentwise", max_iter: Optional[int] = None,
                 boundary: str = "half_cell", inner_tol: float = 0.0,
                 max_outer: int = 0, tile_override: int = 0,
                 band_bits: int = 0, test_flags: int = 0, batch_pack: int = 0,
                 batch_tile_rows: int = 0, precond="jacobi") -> _lib.Options:
    o = _lib.default_options()
    o.precision = {"fp64": _lib.PREC_FP64, "mixed": _lib.PREC_MIXED}[precision]
    if tol is not None:
        o.tol = float(tol)
    o.stop_norm = {"componentwise": _lib.STOP_COMPONENTWISE,
                   "normwise": _lib.STOP_NORMWISE}[stop_norm]
    if max_iter is not None:
        o.max_iter = int(max_iter)
    o.boundary = {"half_cell": _lib.BOUNDARY_HALF_CELL,
                  "drop_edge": _lib.BOUNDARY_DROP_EDGE}[boundary]
    o.inner_tol = float(inner_tol)
    o.max_outer = int(max_outer)
    o.tile_override = int(tile_override)
    o.band_bits = int(band_bits)
    o.test_flags = int(test_flags)
    o.batch_pack = int(batch_pack)
    o.batch_tile_rows = int(batch_tile_rows)
    o.precond = (precond if isinstance(precond, int) else
                 {"jacobi": _lib.PRECOND_JACOBI, "multigrid": _lib.PRECOND_MULTIGRID}[precond])
    return o


class Handle:
    """Owns one ``eik_handle``; see ``eik_create``."""

    def __init__(self, ptr: ctypes.c_void_p, dims: Tuple[int, ...], device: bool):
        self._ptr = ptr
        self.dims = dims
        self.n = int(np.prod(dims))
        self.device = device

    @property
    def ptr(self):
        if not self._ptr:
            raise RuntimeError("handle already destroyed")
        return self._ptr

    def __del__(self):
        try:
            eik_destroy(self)
        except Exception:
            pass


def eik_create(dims: Sequence[int], h: float, hbar: float, f, src_idx, src_U=None,
               options: Optional[_lib.Options] = None, stream=None) -> Handle:
    """Creates a solver (C: ``eik_create``).  ``dims`` is (nx, ny[, nz]);
    ``f`` holds prod(dims) float64 values in C order with x fastest."""
    lib = _lib.load()
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    if _numel(f) != n:
        raise ValueError("f must have prod(dims) elements")
    if not _is_torch(src_idx):
        src_idx = np.ascontiguousarray(np.asarray(src_idx, dtype=np.int64).ravel())
    if src_U is not None and not _is_torch(src_U):
        src_U = np.ascontiguousarray(np.asarray(src_U, dtype=np.float64).ravel())
    fp, fk = _ptr(f, np.float64, "f")
    sp, sk = _ptr(src_idx, np.int64, "src_idx")
    up, uk = _ptr(src_U, np.float64, "src_U")
    if src_U is not None and _numel(src_U) != _numel(src_idx):
        raise ValueError("src_U must match src_idx")
    darr = (ctypes.c_int64 * len(dims))(*dims)
    out = ctypes.c_void_p()
    opt = options if options is not None else _lib.default_options()
    st = lib.eik_create(ctypes.byref(out), len(dims), darr, float(h), float(hbar), fp, sp,
                        up, _numel(src_idx), ctypes.byref(opt), _stream_ptr(stream))
    _lib.check(st)
    return Handle(out, dims, _is_torch(f) and f.is_cuda)


def eik_set_f(handle: Handle, f) -> None:
    """Replaces the forcing field (C: ``eik_set_f``)."""
    if _numel(f) != handle.n:
        raise ValueError("f must have prod(dims) elements")
    fp, fk = _ptr(f, np.float64, "f")
    _lib.check(_lib.load().eik_set_f(handle.ptr, fp))


def _out_like(handle: Handle, out, like_device: bool):
    if out is not None:
        if _numel(out) != handle.n:
            raise ValueError("output must have prod(dims) elements")
        return out
    if like_device and torch is not None:
        return torch.empty(handle.dims[::-1], dtype=torch.float64, device="cuda")
    return np.empty(handle.dims[::-1], dtype=np.float64)


def eik_solve(handle: Handle, S_out=None, phi_out=None, want_phi: bool = False,
              allow_not_converged: bool = False):
    """Solves and returns (S, phi or None, stats dict) (C: ``eik_solve``).
    Outputs are allocated like the inputs (CUDA tensors for a device handle,
    numpy arrays otherwise) unless given."""
    S_out = _out_like(handle, S_out, handle.device)
    if want_phi or phi_out is not None:
        phi_out = _out_like(handle, phi_out, handle.device)
    sp, sk = _ptr(S_out, np.float64, "S_out")
    pp, pk = _ptr(phi_out, np.float64, "phi_out")
    stats = _lib.Stats()
    st = _lib.load().eik_solve(handle.ptr, sp, pp, ctypes.byref(stats))
    allow = (_lib.EIK_OK, _lib.EIK_ERR_NOT_CONVERGED) if allow_not_converged else (_lib.EIK_OK,)
    _lib.check(st, allow)
    d = stats.as_dict()
    d["status"] = st
    return S_out, phi_out, d


def eik_grad(handle: Handle, dLdS, dLdf_out=None):
    """Adjoint gradient dL/df for a loss L(S) of the last solve (C:
    ``eik_grad``).  Returns (dLdf, stats dict)."""
    if _numel(dLdS) != handle.n:
        raise ValueError("dLdS must have prod(dims) elements")
    dLdf_out = _out_like(handle, dLdf_out, _is_torch(dLdS) and dLdS.is_cuda)
    ip, ik = _ptr(dLdS, np.float64, "dLdS")
    op, ok = _ptr(dLdf_out, np.float64, "dLdf")
    stats = _lib.Stats()
    st = _lib.load().eik_grad(handle.ptr, ip, op, ctypes.byref(stats))
    _lib.check(st)
    return dLdf_out, stats.as_dict()


def eik_set_profiling(handle: Handle, enable: bool = True) -> None:
    """Enables per-launch CUDA-event timing of the library's kernels (C:
    ``eik_set_profiling``); graph launches are replaced by timed launches."""
    _lib.check(_lib.load().eik_set_profiling(handle.ptr, int(bool(enable))))


def eik_kernel_stats(handle: Handle):
    """Per-kernel launch counts and timed device milliseconds (C:
    ``eik_kernel_stats``) as a dict name -> (launches, timed, total_ms)."""
    lib = _lib.load()
    cnt = ctypes.c_int()
    _lib.check(lib.eik_kernel_stats(handle.ptr, None, 0, ctypes.byref(cnt)))
    arr = (_lib.KernelStat * max(cnt.value, 1))()
    _lib.check(lib.eik_kernel_stats(handle.ptr, ctypes.cast(arr, ctypes.c_void_p),
                                    cnt.value, ctypes.byref(cnt)))
    return {a.name.decode(): (int(a.launches), int(a.timed_launches), float(a.total_ms))
            for a in arr[:cnt.value]}


def eik_reset_kernel_stats(handle: Handle) -> None:
    _lib.check(_lib.load().eik_reset_kernel_stats(handle.ptr))


def eik_destroy(handle: Handle) -> None:
    """Releases the handle (C: ``eik_destroy``); safe to call twice."""
    if handle is not None and handle._ptr:
        _lib.load().eik_destroy(handle._ptr)
        handle._ptr = None


class Batch:
    """Owns one ``eik_batch`` (see ``eik_create_batch``)."""

    def __init__(self, ptr, dims_list, device: bool):
        self._ptr = ptr
        self.dims = [tuple(d) for d in dims_list]
        self.sizes = [int(np.prod(d)) for d in self.dims]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])
        self.device = device

    @property
    def ptr(self):
        if not self._ptr:
            raise RuntimeError("batch already destroyed")
        return self._ptr

    def split(self, flat):
        return [flat[self.offsets[i]:self.offsets[i + 1]].reshape(self.dims[i][::-1])
                for i in range(len(self.dims))]

    def __del__(self):
        try:
            eik_destroy_batch(self)
        except Exception:
            pass


def eik_create_batch(instances, options: Optional[_lib.Options] = None, stream=None,
                     device: bool = True, workers: int = 0) -> Batch:
    """Creates a batch of independent solves (C: ``eik_create_batch``).
    ``instances`` are objects with dims, h, hbar, f, src_idx, src_U (e.g.
    ``workloads.Instance``).  With ``device`` the concatenated inputs are
    staged in device memory first."""
    lib = _lib.load()
    ndim = len(instances[0].dims)
    if any(len(i.dims) != ndim for i in instances):
        raise ValueError("all instances need the same ndim")
    dims = np.array([list(i.dims) for i in instances], dtype=np.int64).ravel()
    hs = np.array([i.h for i in instances], dtype=np.float64)
    hbars = np.array([i.hbar for i in instances], dtype=np.float64)
    f = np.concatenate([np.ascontiguousarray(i.f, dtype=np.float64).ravel() for i in instances])
    src = np.concatenate([np.asarray(i.src_idx, dtype=np.int64).ravel() for i in instances])
    U = np.concatenate([np.asarray(i.src_U, dtype=np.float64).ravel() for i in instances])
    so = np.concatenate([[0], np.cumsum([len(np.asarray(i.src_idx).ravel())
                                         for i in instances])]).astype(np.int64)
    if device and torch is not None and torch.cuda.is_available():
        f_arg = torch.from_numpy(f).cuda()
    else:
        f_arg = f
    fp, fk = _ptr(f_arg, np.float64, "f")
    out = ctypes.c_void_p()
    opt = options if options is not None else _lib.default_options()
    st = lib.eik_create_batch(
        ctypes.byref(out), len(instances), ndim,
        dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        hs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        hbars.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), fp,
        ctypes.c_void_p(so.ctypes.data), ctypes.c_void_p(src.ctypes.data),
        ctypes.c_void_p(U.ctypes.data), ctypes.byref(opt), _stream_ptr(stream))
    _lib.check(st)
    b = Batch(out, [i.dims for i in instances], device)
    if workers:
        _lib.check(lib.eik_batch_set_concurrency(b.ptr, int(workers)))
    return b


def eik_set_f_batch(batch: Batch, f) -> None:
    fp, fk = _ptr(f, np.float64, "f")
    _lib.check(_lib.load().eik_set_f_batch(batch.ptr, fp))


def eik_solve_batch(batch: Batch, S_out=None, allow_not_converged: bool = False):
    """Solves every instance; returns (S concatenated, list of stats dicts)."""
    if S_out is None:
        if batch.device and torch is not None:
            S_out = torch.empty(batch.n, dtype=torch.float64, device="cuda")
        else:
            S_out = np.empty(batch.n, dtype=np.float64)
    sp, sk = _ptr(S_out, np.float64, "S_out")
    stats = (_lib.Stats * len(batch.dims))()
    st = _lib.load().eik_solve_batch(batch.ptr, sp, ctypes.cast(stats, ctypes.c_void_p))
    allow = (_lib.EIK_OK, _lib.EIK_ERR_NOT_CONVERGED) if allow_not_converged else (_lib.EIK_OK,)
    _lib.check(st, allow)
    return S_out, [s.as_dict() for s in stats]


def eik_grad_batch(batch: Batch, dLdS, dLdf_out=None):
    if dLdf_out is None:
        dLdf_out = (torch.empty_like(dLdS) if _is_torch(dLdS)
                    else np.empty(batch.n, dtype=np.float64))
    ip, ik = _ptr(dLdS, np.float64, "dLdS")
    op, ok = _ptr(dLdf_out, np.float64, "dLdf")
    stats = (_lib.Stats * len(batch.dims))()
    _lib.check(_lib.load().eik_grad_batch(batch.ptr, ip, op, ctypes.cast(stats, ctypes.c_void_p)))
    return dLdf_out, [s.as_dict() for s in stats]


def eik_batch_info(batch: Batch) -> dict:
    """How the batch runs (C: ``eik_batch_info``): packed or not, the packed
    pass's variant and rows per tile, how they were chosen ("fixed",
    "measured", "cached"), the packed pass launches so far, and over the
    solves the node-passes covered and the device time of their graphs."""
    pk, v, ty, how = (ctypes.c_int() for _ in range(4))
    passes, work = ctypes.c_int64(), ctypes.c_int64()
    ms = ctypes.c_double()
    _lib.check(_lib.load().eik_batch_info(batch.ptr, ctypes.byref(pk), ctypes.byref(v),
                                          ctypes.byref(ty), ctypes.byref(how),
                                          ctypes.byref(passes), ctypes.byref(work),
                                          ctypes.byref(ms)))
    return {"packed": bool(pk.value), "variant": v.value, "tile_rows": ty.value,
            "tuned": ("fixed", "measured", "cached")[how.value], "passes": passes.value,
            "node_passes": work.value, "pass_ms": ms.value}


def eik_destroy_batch(batch: Batch) -> None:
    if batch is not None and batch._ptr:
        _lib.load().eik_destroy_batch(batch._ptr)
        batch._ptr = None


def eik_residual_noalloc(dims: Sequence[int], h: float, hbar: float, f, S, src_idx,
                         res_max, boundary: str = "half_cell", stream=None) -> None:
    """Componentwise residual max of S written to the one-element device
    tensor ``res_max``, without any device allocation by the library (C:
    ``eik_residual_noalloc``).  ``f``, ``S``, ``src_idx`` and ``res_max``
    must be CUDA tensors; grids are limited to 2**20 nodes.  The work is
    queued on ``stream`` (default: the current torch stream) and not awaited."""
    dims = tuple(int(d) for d in dims)
    for name, a in (("f", f), ("S", S), ("src_idx", src_idx), ("res_max", res_max)):
        if not (_is_torch(a) and a.is_cuda):
            raise TypeError(f"{name} must be a CUDA tensor")
    fp, fk = _ptr(f, np.float64, "f")
    sp, sk = _ptr(S, np.float64, "S")
    ip, ik = _ptr(src_idx, np.int64, "src_idx")
    rp, rk = _ptr(res_max, np.float64, "res_max")
    darr = (ctypes.c_int64 * len(dims))(*dims)
    b = {"half_cell": _lib.BOUNDARY_HALF_CELL, "drop_edge": _lib.BOUNDARY_DROP_EDGE}[boundary]
    st = _lib.load().eik_residual_noalloc(len(dims), darr, float(h), float(hbar), fp, sp, ip,
                                          _numel(src_idx), b, rp, _stream_ptr(stream))
    if st != _lib.EIK_OK:
        raise _lib.EikError(st, "eik_residual_noalloc failed (grids are limited to 2**20 "
                                "nodes; pointers must be device pointers)")


def grad_S(S, dims: Sequence[int], h: float, stream=None):
    """Nodal gradient of S (C: ``eik_grad_S``): a CUDA float64 tensor of
    shape (ndim, N), component a = dS/dx_a."""
    import torch
    dims = tuple(int(d) for d in dims)
    if not (_is_torch(S) and S.is_cuda):
        raise TypeError("S must be a CUDA tensor")
    n = int(np.prod(dims))
    G = torch.empty((len(dims), n), dtype=torch.float64, device=S.device)
    sp, sk = _ptr(S, np.float64, "S")
    gp, gk = _ptr(G, np.float64, "gradS")
    darr = (ctypes.c_int64 * len(dims))(*dims)
    st = _lib.load().eik_grad_S(len(dims), darr, float(h), sp, gp, _stream_ptr(stream))
    if st != _lib.EIK_OK:
        raise _lib.EikError(st, "eik_grad_S failed")
    return G


def backtrack(G, dims: Sequence[int], h: float, starts, src_idx, step: float,
              max_steps: int, eps: float, stream=None):
    """Optimal paths from the start points (world coordinates, shape
    (P, ndim)) down the gradient G from ``grad_S`` (C: ``eik_backtrack``).
    Returns CUDA tensors (paths (P, max_steps + 1, ndim), lengths (P,),
    status (P,))."""
    import torch
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    dev = G.device
    starts = torch.as_tensor(starts, dtype=torch.float64).reshape(-1, nd).to(dev).contiguous()
    src = torch.as_tensor(np.asarray(src_idx, dtype=np.int64)).to(dev).contiguous()
    P = starts.shape[0]
    paths = torch.empty((P, int(max_steps) + 1, nd), dtype=torch.float64, device=dev)
    lengths = torch.empty(P, dtype=torch.int32, device=dev)
    status = torch.empty(P, dtype=torch.int32, device=dev)
    darr = (ctypes.c_int64 * nd)(*dims)
    gp, gk = _ptr(G, np.float64, "gradS")
    st = _lib.load().eik_backtrack(
        nd, darr, float(h), gp, ctypes.c_void_p(starts.data_ptr()), P, float(step),
        int(max_steps), ctypes.c_void_p(src.data_ptr()), int(src.numel()), float(eps),
        ctypes.c_void_p(paths.data_ptr()), ctypes.c_void_p(lengths.data_ptr()),
        ctypes.c_void_p(status.data_ptr()), _stream_ptr(stream))
    if st != _lib.EIK_OK:
        raise _lib.EikError(st, "eik_backtrack failed")
    return paths, lengths, status


def sfs_forcing(P, f_min: float = 0.0, stream=None):
    """Eikonal forcing of a shape-from-shading image (C: ``eik_sfs_forcing``):
    f = max(sqrt(1/P^2 - 1), f_min) for a CUDA float64 tensor P."""
    import torch
    if not (_is_torch(P) and P.is_cuda):
        raise TypeError("P must be a CUDA tensor")
    f = torch.empty_like(P)
    pp, pk = _ptr(P, np.float64, "P")
    fp, fk = _ptr(f, np.float64, "f")
    st = _lib.load().eik_sfs_forcing(pp, _numel(P), float(f_min), fp, _stream_ptr(stream))
    if st != _lib.EIK_OK:
        raise _lib.EikError(st, "eik_sfs_forcing failed")
    return f


def fft_series(dims: Sequence[int], h: float, hbar: float, f, src_idx, terms: int,
               f_tilde: float = 0.0, stream=None):
    """FFT perturbation series (C: ``eik_fft_series``, Sec. 5 Table 1) on a
    2D grid dims = (nx, ny); f and src_idx host arrays or CUDA tensors.
    Returns (S, phi, f_tilde) with S and phi as CUDA float64 tensors (numpy
    arrays without a GPU-resident input) of nx*ny values, x fastest."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    if _numel(f) != n:
        raise ValueError("f must have prod(dims) elements")
    if not _is_torch(src_idx):
        src_idx = np.ascontiguousarray(np.asarray(src_idx, dtype=np.int64).ravel())
    device = _is_torch(f) and f.is_cuda
    if device:
        import torch
        S = torch.empty(n, dtype=torch.float64, device=f.device)
        phi = torch.empty(n, dtype=torch.float64, device=f.device)
    else:
        f = np.ascontiguousarray(f, dtype=np.float64)
        S = np.empty(n, dtype=np.float64)
        phi = np.empty(n, dtype=np.float64)
    fp, fk = _ptr(f, np.float64, "f")
    sp, sk = _ptr(src_idx, np.int64, "src_idx")
    Sp, Sk = _ptr(S, np.float64, "S")
    pp, pk = _ptr(phi, np.float64, "phi")
    d = (ctypes.c_int64 * 2)(*dims)
    ft = ctypes.c_double()
    st = _lib.load().eik_fft_series(d, float(h), float(hbar), fp, sp, _numel(src_idx),
                                    int(terms), float(f_tilde), Sp, pp, ctypes.byref(ft),
                                    _stream_ptr(stream))
    if st != _lib.EIK_OK:
        raise _lib.EikError(st, "eik_fft_series failed")
    return S, phi, ft.value


def solve(f, h: float, hbar: float, src_idx, src_U=None, precision: str = "fp64",
          tol: Optional[float] = None, want_phi: bool = False, **kw):
    """One-shot convenience: dims are taken from the array shape (numpy order
    (nz,) ny, nx)."""
    shape = tuple(f.shape)
    dims = tuple(reversed(shape))
    opt = make_options(precision=precision, tol=tol, **kw)
    hd = eik_create(dims, h, hbar, f, src_idx, src_U, opt)
    try:
        S, phi, stats = eik_solve(hd, want_phi=want_phi)
    finally:
        eik_destroy(hd)
    return S, phi, stats
