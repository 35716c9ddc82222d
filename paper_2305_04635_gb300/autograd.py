"""Differentiable banded solve: x = A^{-1} b and log det A with gradients.

The forward pass factors a copy of the band (bchol_factor), solves
(bchol_solve) and forms log det A = 2 sum log L_ii (bchol_logdet).  The
backward pass calls bchol_backward, which forms the band of A^{-1} by
selected inversion on the GPU and returns df/d(band of A) and df/db.  The
gradient is with respect to the STORED band entries: an off-diagonal entry
ab[d, j] stands for both A(j+d, j) and A(j, j+d).
"""
from __future__ import annotations

import ctypes

import torch

from . import BcholError, Handle, _band_args, _check, _handle, factor, get_info, solve


def logdet(L: torch.Tensor, handle: Handle | None = None) -> torch.Tensor:
    """log det A from the factor band L (device scalar, asynchronous)."""
    h = _handle(handle)
    ptr, n, ldab = _band_args(L, 0)
    out = torch.empty((), dtype=torch.float64, device=L.device)
    h._sync_stream()
    _check("bchol_logdet", h._lib.bchol_logdet(h.ptr, n, ptr, ldab, ctypes.c_void_p(out.data_ptr())))
    return out


def backward(L: torch.Tensor, k: int, x: torch.Tensor | None, xbar: torch.Tensor | None, ldbar: float,
             handle: Handle | None = None):
    """(abar, bbar): gradients of f(x, log det A) w.r.t. the stored band of A and b."""
    h = _handle(handle)
    ptr, n, ldab = _band_args(L, k)
    abar = torch.empty(n, k + 1, dtype=torch.float64, device=L.device).T
    bbar = None
    if xbar is not None:
        xbar = xbar.contiguous()
        x = x.contiguous()
        bbar = torch.empty_like(xbar)
    h._sync_stream()
    _check("bchol_backward", h._lib.bchol_backward(
        h.ptr, n, k, ptr, ldab, ctypes.c_void_p(x.data_ptr()) if xbar is not None else None,
        ctypes.c_void_p(xbar.data_ptr()) if xbar is not None else None, float(ldbar),
        ctypes.c_void_p(abar.data_ptr()), k + 1, ctypes.c_void_p(bbar.data_ptr()) if bbar is not None else None))
    return abar, bbar


class BandCholSolve(torch.autograd.Function):
    """(x, logdet) = BandCholSolve.apply(ab, k, b) with ab the (k+1, n) lower band of A."""

    @staticmethod
    def forward(ctx, ab: torch.Tensor, k: int, b: torch.Tensor):
        h = _handle(None)
        L = torch.empty(ab.shape[1], ab.shape[0], dtype=torch.float64, device=ab.device).T
        L.copy_(ab)
        info = factor(L, k, handle=h)
        x = b.detach().clone().contiguous()
        solve(L, k, x, handle=h)
        rc, infos = get_info(info, handle=h)
        if rc != 0:
            raise BcholError("bchol_factor", rc)
        ld = logdet(L, handle=h)
        ctx.save_for_backward(L, x)
        ctx.k = k
        return x, ld

    @staticmethod
    def backward(ctx, xbar, ldbar):
        L, x = ctx.saved_tensors
        ld = 0.0 if ldbar is None else float(ldbar)
        abar, bbar = backward(L, ctx.k, x, None if xbar is None else xbar.contiguous(), ld)
        return abar, None, bbar
