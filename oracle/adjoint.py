"""Reverse-mode derivative of RCholeskyQR2 (oracle; test infrastructure only).

Not in the paper.  In exact arithmetic Alg. 3 returns the thin QR factors of
X with Q orthonormal and diag(R) > 0 -- unique, whatever Theta is (the sketch
only conditions the first pass).  Its derivative is therefore that of the
thin QR map, written here from the matrix-calculus result for X = Q R
(Walter & Lehmann 2018; Seeger et al. 2017):

    M    = R Rbar^T - Qbar^T Q
    Xbar = (Qbar + Q copyltu(M)) R^{-T},    copyltu(M) = tril(M) + tril(M, -1)^T

with Q recomputed from X and R by forward substitution (only R and the seed
are kept from the forward pass).  Pinned in the tests by central finite
differences of the oracle's own rcholqr2 and by torch's QR derivative.
"""
import numpy as np

from . import linalg


def copyltu(M):
    """The symmetric matrix whose lower triangle is that of M."""
    return np.tril(M) + np.tril(M, -1).T


def back_substitution(R, B):
    """Z with R Z = B for upper triangular R (column by column of B, rows from the bottom)."""
    n = R.shape[0]
    Z = np.zeros_like(B, dtype=np.float64)
    for i in range(n - 1, -1, -1):
        Z[i] = (B[i] - R[i, i + 1:] @ Z[i + 1:]) / R[i, i]
    return Z


def qr_adjoint(X, R, Qbar, Rbar):
    """Xbar for the thin QR map X -> (Q, R), Q recomputed as X R^{-1}."""
    X = np.asarray(X, dtype=np.float64)
    return qr_adjoint_factors(linalg.forward_substitution(X, R), R, Qbar, Rbar)


def qr_adjoint_factors(Q, R, Qbar, Rbar):
    """The same Xbar from given factors (Q, R); used where Q came out of a
    lower-precision forward pass and differs from X R^{-1} in FP64."""
    Q = np.asarray(Q, dtype=np.float64)
    M = R @ Rbar.T - Qbar.T @ Q
    Y = Qbar + Q @ copyltu(M)
    return back_substitution(R, Y.T).T


def loss_weights(m, n, seed):
    """Seeded N(0,1) weights W1 (m x n) and W2 (n x n) of loss = sum(W1 * Q) + sum(W2 * R)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, n)), rng.standard_normal((n, n))
