"""The randomized Cholesky QR algorithms in FP64, step by step (oracle; test infrastructure only).

Each driver follows the paper's algorithm in its own order and notation:

* rcholqr    -- Alg. 2 (RCholeskyQR):  P = Theta X;  [S, R] = QR(P);  Q = X R^{-1}.
* rcholqr2   -- Alg. 3 (RCholeskyQR2): Alg. 2, then A = Q^T Q;  R' = chol(A);
                R <- R' R;  Q <- Q R'^{-1}.
* reduced    -- Alg. 5 (reduced RCholeskyQR): P = Theta X, Y = L X;
                [S, R] = QR(P);  Z = Y R^{-1}.
* rrrcholqr  -- Alg. 7 (RRRCholQR) with the column normalisation of Sec. 4:
                D = diag(||X_j||), P = Theta X D^{-1}; [S, R, Pi] = RRQR(P);
                r = min r with ||R22||_F <= tau ||R||_2;
                Q = (X Pi_{:,1:r} D_sel^{-1}) R_{1:r,1:r}^{-1};  R <- R_{1:r,:} Pi^T D Pi.
* rrrcholqr2 -- Alg. 7 followed by one CholeskyQR pass as in Alg. 3 (Sec. 4).

The sketch is the product of the integer levels G (theta.theta_levels) with
X in FP64 (numpy matmul as the library step), scaled afterwards by
c = theta_scale(k); for long X it is formed in row blocks whose FP64 partial
sums are added in order.
"""
import numpy as np

from . import linalg
from . import theta as _theta
from .theta import GAUSSIAN, theta_levels, theta_scale

SKETCH_ROW_BLOCK = 1 << 14


def sketch(X, k, seed, row_offset=0, stream=0, row_block=SKETCH_ROW_BLOCK, dist=GAUSSIAN):
    """P = Theta X (k x n, FP64), Theta rows for global X rows row_offset .. row_offset+m-1 (Alg. 2 step 1)."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    acc = np.zeros((k, n))
    for r0 in range(0, m, row_block):
        r1 = min(m, r0 + row_block)
        G = (theta_levels(seed, k, row_offset + r0, r1 - r0, stream) if dist == GAUSSIAN
             else _theta.levels(seed, k, row_offset + r0, r1 - r0, stream, dist=dist))
        acc += G @ X[r0:r1]
    return (theta_scale(k) if dist == GAUSSIAN else _theta.scale(k, dist)) * acc


def sketch_rows(X, k, seed, rows, row_offset=0, stream=0, row_block=SKETCH_ROW_BLOCK, dist=GAUSSIAN):
    """Selected rows of P = Theta X (one output row at a time for sampled checks of long X)."""
    X = np.asarray(X)
    m, n = X.shape
    acc = np.zeros((len(rows), n))
    for r0 in range(0, m, row_block):
        r1 = min(m, r0 + row_block)
        G = (theta_levels(seed, k, row_offset + r0, r1 - r0, stream, rows=rows) if dist == GAUSSIAN
             else _theta.levels(seed, k, row_offset + r0, r1 - r0, stream, rows=rows, dist=dist))
        acc += G @ np.asarray(X[r0:r1], dtype=np.float64)
    return (theta_scale(k) if dist == GAUSSIAN else _theta.scale(k, dist)) * acc


def column_norms(X):
    """D_j = ||X_(:,j)||_2 (Sec. 4, the normalisation matrix)."""
    X = np.asarray(X, dtype=np.float64)
    return np.sqrt(np.sum(X * X, axis=0))


def rcholqr_from_sketch(X, P):
    """Alg. 2 steps 2-3 for a given sketch P: returns (Q, S, R)."""
    S, R = linalg.householder_qr(P)
    Q = linalg.forward_substitution(X, R)
    return Q, S, R


def rcholqr(X, k, seed, stream=0, dist=GAUSSIAN):
    """Alg. 2: returns (Q, S, R)."""
    P = sketch(X, k, seed, stream=stream, dist=dist)
    return rcholqr_from_sketch(X, P)


def rcholqr_f32(X, k, seed, stream=0):
    """Alg. 2 in the multi-precision form of Sec. 1.3 / Sec. 5: the sketch and the Householder QR
    in FP64 (u_f), the substitution Q = X R^{-1} in float32 (u = 2^-24).  Returns (Q float32, S, R)."""
    P = sketch(X, k, seed, stream=stream)
    S, R = linalg.householder_qr(P)
    return linalg.forward_substitution_f32(X, R), S, R


def cholqr_pass(Q, R):
    """Alg. 3 steps 2-4 applied to (Q, R): returns (Q <- Q R'^{-1}, R <- R' R, R')."""
    A = Q.T @ Q
    Rp = linalg.cholesky(A)
    return linalg.forward_substitution(Q, Rp), Rp @ R, Rp


def rcholqr2(X, k, seed, stream=0, dist=GAUSSIAN):
    """Alg. 3: returns (Q, R, S) -- S is the orthonormal sketch from the first pass."""
    Q, S, R = rcholqr(X, k, seed, stream, dist)
    Q2, R2, _ = cholqr_pass(Q, R)
    return Q2, R2, S


def rcholqr2_implicit(X, k, seed, stream=0, dist=GAUSSIAN):
    """Alg. 3 without step 4 (the remark after Alg. 3): returns (Q1, R, Rp) with Q1 from Alg. 2,
    R = Rp R1 and the orthonormal factor Q = Q1 Rp^{-1} left implicit."""
    Q1, _, R1 = rcholqr(X, k, seed, stream, dist)
    Rp = linalg.cholesky(Q1.T @ Q1)
    return Q1, Rp @ R1, Rp


def implicit_q_times(Q1, Rp, Y):
    """Q Y = Q1 (Rp^{-1} Y): the right product of the implicit Q."""
    return np.asarray(Q1, dtype=np.float64) @ linalg.back_substitution_upper(Rp, np.asarray(Y, dtype=np.float64))


def implicit_qt_times(Q1, Rp, B):
    """Q^T B = Rp^{-T} (Q1^T B): the left product of the implicit Q (Q^T = Rp^{-T} Q1^T),
    Rp^{-T} applied by forward substitution (rows of Rp^T = columns of Rp)."""
    C = np.asarray(Q1, dtype=np.float64).T @ np.asarray(B, dtype=np.float64)
    return linalg.forward_substitution(C.T, Rp).T


def col_rcholqr(X, b, k, seed, rgs=False, stream=0):
    """Alg. 4 (column-oriented RCholeskyQR) on X given as column blocks of width b (the last may be
    narrower): for each block i, in the paper's steps,
        2.  P_i = Theta X_i
        3.  R_{<i,i} = S_{<i}^+ P_i              (least squares; a library routine)
        4.  [S_i, R_ii] = QR(P_i - S_{<i} R_{<i,i})
        5.  Q_i = (X_i - Q_{<i} R_{<i,i}) R_ii^{-1}   (forward substitution)
    rgs=True turns it into the randomized Gram-Schmidt of the remark after Alg. 4: the sketch of
    each computed block replaces S_i, S_i <- Theta Q_i.  Returns (Q, S, R)."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    Q = np.zeros((m, n))
    S = np.zeros((k, n))
    R = np.zeros((n, n))
    for c0 in range(0, n, b):
        c1 = min(n, c0 + b)
        Xi = X[:, c0:c1]
        Pi = sketch(Xi, k, seed, stream=stream)
        if c0 > 0:
            R[:c0, c0:c1] = np.linalg.lstsq(S[:, :c0], Pi, rcond=None)[0]
        Si, Rii = linalg.householder_qr(Pi - S[:, :c0] @ R[:c0, c0:c1])
        S[:, c0:c1] = Si
        R[c0:c1, c0:c1] = Rii
        Q[:, c0:c1] = linalg.forward_substitution(Xi - Q[:, :c0] @ R[:c0, c0:c1], Rii)
        if rgs:
            S[:, c0:c1] = sketch(Q[:, c0:c1], k, seed, stream=stream)
    return Q, S, R


def reduced(X, k, seed, L=None):
    """Alg. 5: returns (Z, S, R); L is an explicit l x m extractor, or None for L = Theta (then Z ~ S)."""
    X = np.asarray(X, dtype=np.float64)
    P = sketch(X, k, seed)
    Y = P if L is None else np.asarray(L, dtype=np.float64) @ X
    S, R = linalg.householder_qr(P)
    Z = linalg.forward_substitution(Y, R)
    return Z, S, R


def rrrcholqr(X, k, seed, tau, stream=0, strong_f=None):
    """Alg. 7 with column normalisation: returns (Q m x r, S k x r, R r x n, perm, r).

    X[:, perm] ~ Q R.  Zero columns of X are left unscaled (D_j = 1 for them).  The RRQR
    of step 2 is column-pivoted Householder QR, followed (strong_f = f) by the strong-RRQR
    swaps of Gu & Eisenstat with parameter f (Sec. 4 and Sec. 6.1 take f = 1.5).
    """
    X = np.asarray(X, dtype=np.float64)
    D = column_norms(X)
    Dsafe = np.where(D > 0, D, 1.0)
    P = sketch(X, k, seed, stream=stream) / Dsafe[None, :]   # P <- P D^{-1}
    if strong_f is None:
        S, R, perm = linalg.qrcp(P)                           # step 2
        r = linalg.truncation_rank(R, tau)                    # step 3
    else:
        S, R, perm, r = linalg.strong_rrqr(P, tau, strong_f)  # steps 2-3
    Xsel = X[:, perm[:r]] / Dsafe[perm[:r]][None, :]          # X Pi_{:,1:r} D_sel^{-1}
    Q = linalg.forward_substitution(Xsel, R[:r, :r])          # step 4
    Rout = R[:r, :] * Dsafe[perm][None, :]                    # step 5 and R <- R Pi^T D Pi
    return Q, S[:, :r], Rout, perm, r


def rrrcholqr2(X, k, seed, tau, stream=0, strong_f=None):
    """Alg. 7 followed by one CholeskyQR pass: returns (Q, R, perm, r)."""
    Q, _, R, perm, r = rrrcholqr(X, k, seed, tau, stream, strong_f)
    if r == 0:
        return Q, R, perm, r
    Q2, R2, _ = cholqr_pass(Q, R)
    return Q2, R2, perm, r


# ---------------------------------------------------------------- metrics (Sec. 6)

def orthogonality(Q):
    """Delta = ||Q^T Q - I||_2."""
    n = Q.shape[1]
    return linalg.spectral_norm(Q.T @ Q - np.eye(n))


def condition_number(A):
    s = np.linalg.svd(A, compute_uv=False)
    return float(s[0] / s[-1]) if s[-1] > 0 else np.inf


def residuals(X, Q, R, perm=None):
    """(||X - Q R||_F / ||X||_F, max_j ||X_j - (QR)_j|| / ||X_j||) on the columns X[:, perm]."""
    X = np.asarray(X, dtype=np.float64)
    if perm is not None:
        X = X[:, perm]
    E = X - Q @ R
    cn = column_norms(X)
    col = column_norms(E) / np.where(cn > 0, cn, 1.0)
    return float(np.linalg.norm(E) / np.linalg.norm(X)), float(np.max(col))


def embedding_epsilon(G_scaled, U):
    """Exact epsilon of Def. 2.1 for Theta (dense, given) on range(U), U orthonormal: max |sigma_i(Theta U)^2 - 1|."""
    s = np.linalg.svd(G_scaled @ U, compute_uv=False)
    return float(np.max(np.abs(s * s - 1.0)))
