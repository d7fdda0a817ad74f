"""binary64 matrix product through the exact Ozaki-II path, as a
``torch.autograd.Function``.

The forward calls ``ozaki2_dgemm_fwd`` and keeps the returned cache of int8
residue planes; the hand-written backward calls ``ozaki2_dgemm_bwd``, which
computes dA = dC B^T and dB = A^T dC through the same exact path while reusing
the forward's residue planes of B and A instead of recomputing them.  All
arithmetic runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L


class _Cache:
    """Owns one library cache handle (freed when the graph node dies)."""

    def __init__(self, handle: C.c_void_p):
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            L.lib().ozaki2_cache_destroy(self.h)
            self.h = None


def _check_operand(x: torch.Tensor, name: str) -> torch.Tensor:
    if x.dtype != torch.float64 or not x.is_cuda or x.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float64 CUDA tensor")
    return x.contiguous()


class OzakiMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A: torch.Tensor, B: torch.Tensor, opts: L.Opts | None = None):
        A = _check_operand(A, "A")
        B = _check_operand(B, "B")
        M, K = A.shape
        K2, N = B.shape
        if K != K2:
            raise ValueError("inner dimensions differ")
        Cm = torch.empty((M, N), dtype=torch.float64, device=A.device)
        h = C.c_void_p()
        need = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        st = L.lib().ozaki2_dgemm_fwd(M, N, K, A.data_ptr(), K, B.data_ptr(), N, Cm.data_ptr(), N,
                                      C.byref(opts) if opts is not None else None,
                                      C.byref(h) if need else None,
                                      torch.cuda.current_stream(A.device).cuda_stream)
        L.check(st, "ozaki2_dgemm_fwd")
        ctx.cache = _Cache(h) if need else None
        ctx.shape = (M, N, K)
        return Cm

    @staticmethod
    def backward(ctx, dC: torch.Tensor):
        M, N, K = ctx.shape
        dC = dC.to(torch.float64).contiguous()
        dA = torch.empty((M, K), dtype=torch.float64, device=dC.device) if ctx.needs_input_grad[0] else None
        dB = torch.empty((K, N), dtype=torch.float64, device=dC.device) if ctx.needs_input_grad[1] else None
        st = L.lib().ozaki2_dgemm_bwd(ctx.cache.h, dC.data_ptr(), N,
                                      dA.data_ptr() if dA is not None else None, K,
                                      dB.data_ptr() if dB is not None else None, N,
                                      torch.cuda.current_stream(dC.device).cuda_stream)
        L.check(st, "ozaki2_dgemm_bwd")
        return dA, dB, None


def ozaki_matmul(A: torch.Tensor, B: torch.Tensor, **opts) -> torch.Tensor:
    """A @ B for float64 CUDA tensors through the exact Ozaki-II path, rounded
    to nearest-even binary64, differentiable in both arguments."""
    return OzakiMatmul.apply(A, B, L.opts(**opts) if opts else None)
