"""torch.autograd.Function for the rank-k approximation A_k through randUTV.

Forward: ``randutv_lowrank`` (A_k = U_k U_k^T A, the sketch fixed by the
seed).  Backward: ``randutv_lowrank_backward``, the hand-written adjoint,
which recomputes the per-step Householder factors from A and the seed
instead of storing them.  Only A is saved between the two passes.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib


def _colmajor64(x):
    out = _lib.colmajor_empty(x.shape[0], x.shape[1], device=x.device, dtype=torch.float64)
    out.copy_(x)
    return out


class RandUTVLowRank(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, k, b, q, seed):
        if not A.is_cuda or A.dtype != torch.float64:
            raise ValueError("A must be a float64 CUDA tensor")
        m, n = A.shape
        Ac = _colmajor64(A)
        Ak = _lib.colmajor_empty(m, n, device=A.device, dtype=torch.float64)
        _lib._check("randutv_lowrank", _lib.lib().randutv_lowrank(
            m, n, ctypes.c_void_p(Ac.data_ptr()), m, k, b, q, seed,
            ctypes.c_void_p(Ak.data_ptr()), _lib._stream()))
        ctx.save_for_backward(Ac)
        ctx.params = (k, b, q, seed)
        return Ak

    @staticmethod
    def backward(ctx, gAk):
        (Ac,) = ctx.saved_tensors
        k, b, q, seed = ctx.params
        m, n = Ac.shape
        g = _colmajor64(gAk)
        dA = _lib.colmajor_empty(m, n, device=Ac.device, dtype=torch.float64)
        _lib._check("randutv_lowrank_backward", _lib.lib().randutv_lowrank_backward(
            m, n, ctypes.c_void_p(Ac.data_ptr()), m, k, b, q, seed,
            ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(dA.data_ptr()), _lib._stream()))
        return dA, None, None, None, None


def lowrank(A, k, b, q=1, seed=0):
    """A_k = U(:, 0:k) U(:, 0:k)^T A through randUTV (differentiable in A)."""
    return RandUTVLowRank.apply(A, k, b, q, seed)
