"""Mixed-precision solve with FP64 iterative refinement (bchol_solve_mixed)."""
from __future__ import annotations

import ctypes

import torch

from . import Handle, _band_args, _check, _handle, _require_cuda


def _cols(t: torch.Tensor, n: int):
    if t.dim() == 1:
        if t.shape[0] != n or (n > 1 and t.stride(0) != 1):
            raise ValueError("vector must be contiguous with length n")
        return 1, max(1, n)
    if t.shape[0] != n or (n > 1 and t.stride(0) != 1):
        raise ValueError("matrix must be (n, nrhs) column-major")
    return t.shape[1], (t.stride(1) if t.shape[1] > 1 else max(1, n))


def solve_mixed(ab: torch.Tensor, k: int, b: torch.Tensor, x: torch.Tensor | None = None, max_iter: int = 30,
                tol: float = 1e-13, handle: Handle | None = None):
    """X = A^{-1} B with FP32-accumulated trailing updates and FP64 refinement.

    `ab` (the band of A) and `b` are not modified.  Returns (x, info, iters, resid, corr):
    info is the device int32 info of the factorization; iters the number of
    corrections; resid the final max_c ||b_c - A x_c|| / ||b_c|| (the refinement
    stops once it is <= tol); corr the last relative correction.
    """
    h = _handle(handle)
    ptr, n, ldab = _band_args(ab, k)
    _require_cuda(b, "b")
    nrhs, ldb = _cols(b, n)
    if x is None:
        x = torch.empty_like(b) if b.dim() == 1 else torch.empty(b.shape[1], n, dtype=b.dtype, device=b.device).T
    _require_cuda(x, "x")
    nx, ldx = _cols(x, n)
    if nx != nrhs or b.dtype != torch.float64 or x.dtype != torch.float64:
        raise ValueError("b and x must be float64 with the same number of columns")
    info = torch.zeros(1, dtype=torch.int32, device=ab.device)
    iters, resid, corr = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    h._sync_stream()
    rc = h._lib.bchol_solve_mixed(h.ptr, n, k, nrhs, ptr, ldab, ctypes.c_void_p(b.data_ptr()), ldb,
                                  ctypes.c_void_p(x.data_ptr()), ldx, max_iter, float(tol),
                                  ctypes.c_void_p(info.data_ptr()), ctypes.byref(iters), ctypes.byref(resid),
                                  ctypes.byref(corr))
    if rc not in (0, 1):
        _check("bchol_solve_mixed", rc)
    return x, info, iters.value, resid.value, corr.value
