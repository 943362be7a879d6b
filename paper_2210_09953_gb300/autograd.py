"""Differentiable RCholeskyQR2 behind torch.autograd.Function.

Forward: rcqr_factor (Alg. 3) -> (Q, R); only R (with the seed and k) is kept
besides the input.  Backward: the factorization is re-run from X and the seed
(which recomputes the sketch, its R and Q exactly as in the forward -- every
kernel is deterministic), then rcqr_qr_adjoint forms

    Xbar = (Qbar + Q copyltu(R Rbar^T - Qbar^T Q)) R^{-T}

on the device (the derivative of the thin QR map that Alg. 3 computes; see
include/rcqr.h).  This module only marshals tensors; every arithmetic step
runs in librcqr.so.
"""
import torch

from . import _binding as rc


def _colmajor(t, dtype):
    out = rc.colmajor(t.shape[0], t.shape[1], dtype, t.device)
    out.copy_(t)
    return out


class RCholeskyQR2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, k, seed):
        Q, R, _, _, status = rc.rcqr_factor(X, k, seed, variant=rc.DIRECT2)
        ctx.save_for_backward(X, R)
        ctx.k, ctx.seed = int(k), int(seed)
        ctx.status = status
        return Q, R

    @staticmethod
    def backward(ctx, Qbar, Rbar):
        X, R = ctx.saved_tensors
        Q, R2, _, _, _ = rc.rcqr_factor(X, ctx.k, ctx.seed, variant=rc.DIRECT2)   # Q recomputed
        qdt = Q.dtype
        m, n = Q.shape
        Qb = _colmajor(Qbar, qdt) if Qbar is not None else rc.colmajor(m, n, qdt, Q.device).zero_()
        Rb = _colmajor(Rbar, torch.float64) if Rbar is not None else rc.colmajor(n, n, torch.float64, Q.device).zero_()
        Xbar = rc.rcqr_qr_adjoint(Q, R, Qb, Rb)
        return Xbar.to(X.dtype), None, None


def rcholqr2(X, k, seed):
    """(Q, R) of RCholeskyQR2 with gradients w.r.t. X (X column-major, see inputs.colmajor_empty)."""
    return RCholeskyQR2.apply(X, k, seed)
