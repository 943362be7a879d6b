"""Textbook FP64 kernels the algorithms call (oracle; test infrastructure only).

* householder_qr  -- the QR of the small sketch, Alg. 2 step 2 (the paper's
  choice of Householder reflections, Sec. 3.1).  Unblocked, Golub & Van Loan
  Alg. 5.2.1; signs fixed so that diag(R) > 0, which makes (S, R) unique.
* qrcp            -- the rank-revealing QR of Alg. 7 step 2, realised as
  Businger-Golub column pivoting: at step j the column of largest remaining
  2-norm (recomputed from scratch, ties to the lowest index) is swapped in.
* truncation_rank -- Alg. 7 step 3: min r with ||R[r:, r:]||_F <= tau ||R||_2.
* forward_substitution -- Q = X R^{-1} row by row (Alg. 2 step 3; the
  substitution whose row-wise backward stability Sec. 5.1 invokes).
* cholesky        -- A = R^T R, R upper with positive diagonal (Alg. 3 step 3);
  raises NotSPD(j) on the first non-positive pivot.
"""
import numpy as np


class NotSPD(ArithmeticError):
    """Cholesky met a pivot <= 0 at (0-based) column ``j``."""

    def __init__(self, j):
        super().__init__(f"non-positive Cholesky pivot at column {j}")
        self.j = j


def _house(x):
    """Householder vector v (v[0] = 1 convention not used) and beta with (I - beta v v^T) x = -sign(x0)||x|| e1."""
    alpha = np.linalg.norm(x)
    v = x.copy()
    if alpha == 0.0:
        return v, 0.0, 0.0
    s = 1.0 if x[0] >= 0 else -1.0
    v[0] = x[0] + s * alpha
    vtv = float(v @ v)
    return v, 2.0 / vtv, -s * alpha


def householder_qr(P):
    """[S, R] = QR(P) for a k x n matrix P (k >= n): S k x n orthonormal, R n x n upper, diag(R) > 0.

    The reflectors are applied to the trailing columns one at a time; S is
    formed explicitly by applying them, in reverse order, to the first n
    columns of the identity.  Zero columns give a zero diagonal entry (no sign flip).
    """
    A = np.array(P, dtype=np.float64, copy=True)
    k, n = A.shape
    if k < n:
        raise ValueError("householder_qr needs k >= n")
    vs, betas = [], []
    for j in range(n):
        v, beta, d = _house(A[j:, j])
        if beta != 0.0:
            A[j:, j:] -= beta * np.outer(v, v @ A[j:, j:])
        A[j, j] = d
        A[j + 1:, j] = 0.0
        vs.append(v)
        betas.append(beta)
    R = np.triu(A[:n, :n])
    S = np.zeros((k, n))
    S[:n, :n] = np.eye(n)
    for j in reversed(range(n)):
        v, beta = vs[j], betas[j]
        if beta != 0.0:
            S[j:, :] -= beta * np.outer(v, v @ S[j:, :])
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return S * sgn[None, :], R * sgn[:, None]


def qrcp(P):
    """[S, R, perm] = column-pivoted Householder QR: P[:, perm] = S R, diag(R) >= 0, |R_jj| non-increasing.

    perm[j] is the original column index placed at position j.
    """
    A = np.array(P, dtype=np.float64, copy=True)
    k, n = A.shape
    if k < n:
        raise ValueError("qrcp needs k >= n")
    perm = np.arange(n)
    vs, betas = [], []
    for j in range(n):
        norms = np.sqrt(np.sum(A[j:, j:] ** 2, axis=0))   # recomputed, no downdating
        p = j + int(np.argmax(norms))                      # argmax returns the lowest index on ties
        if p != j:
            A[:, [j, p]] = A[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        v, beta, d = _house(A[j:, j])
        if beta != 0.0:
            A[j:, j:] -= beta * np.outer(v, v @ A[j:, j:])
        A[j, j] = d
        A[j + 1:, j] = 0.0
        vs.append(v)
        betas.append(beta)
    R = np.triu(A[:n, :n])
    S = np.zeros((k, n))
    S[:n, :n] = np.eye(n)
    for j in reversed(range(n)):
        v, beta = vs[j], betas[j]
        if beta != 0.0:
            S[j:, :] -= beta * np.outer(v, v @ S[j:, :])
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return S * sgn[None, :], R * sgn[:, None], perm


def back_substitution_upper(U, B):
    """X with U X = B for upper triangular U (one row of X at a time, from the last)."""
    U = np.asarray(U, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    r = U.shape[0]
    X = np.zeros_like(B)
    for i in reversed(range(r)):
        X[i] = (B[i] - U[i, i + 1:] @ X[i + 1:]) / U[i, i]
    return X


def swap_ratios(R, r):
    """rho_ij of Gu & Eisenstat (1996) for the split of R at rank r: with R11 = R[:r, :r],
    R12 = R[:r, r:], R22 = R[r:, r:],
        rho_ij = (R11^{-1} R12)_ij^2 + (gamma_j(R22) / omega_i(R11))^2,
    gamma_j = the 2-norm of column j of R22, omega_i = 1 / (2-norm of row i of R11^{-1}).
    sqrt(rho_ij) is the factor by which |det R11| grows when column i and column r + j trade
    places (their Lemma 3.1)."""
    R11, R12, R22 = R[:r, :r], R[:r, r:], R[r:, r:]
    W = back_substitution_upper(R11, R12)
    Rinv = back_substitution_upper(R11, np.eye(r))
    inv_omega2 = np.sum(Rinv * Rinv, axis=1)
    gamma2 = np.sum(R22 * R22, axis=0)
    return W * W + inv_omega2[:, None] * gamma2[None, :]


def strong_rrqr_swaps(P, perm, r, f, max_swaps=None):
    """The swaps of strong RRQR (Gu & Eisenstat 1996, Algorithm 4) at a fixed rank r, from the
    column order perm: while some rho_ij > f^2, trade column i of the leading block with
    column r + j (the largest rho_ij, the first one in column-major order on ties) and
    re-factor P[:, perm] by Householder QR.  Each swap multiplies |det R11| by more than f,
    so it ends; max_swaps (default 4 n) bounds it in floating point.
    Returns (S, R, perm, swaps) with P[:, perm] = S R, diag(R) >= 0."""
    P = np.asarray(P, dtype=np.float64)
    n = P.shape[1]
    perm = np.array(perm, copy=True)
    S, R = householder_qr(P[:, perm])
    if r <= 0 or r >= n:
        return S, R, perm, 0
    limit = 4 * n if max_swaps is None else max_swaps
    swaps = 0
    while swaps < limit:
        rho = swap_ratios(R, r)
        flat = rho.ravel(order="F")
        t = int(np.argmax(flat))
        if not flat[t] > f * f:
            break
        i, j = t % r, t // r
        perm[[i, r + j]] = perm[[r + j, i]]
        S, R = householder_qr(P[:, perm])
        swaps += 1
    return S, R, perm, swaps


def strong_rrqr(P, tau, f, rounds=4):
    """Rank-revealing QR for Alg. 7 steps 2-3 with Gu-Eisenstat swaps: QRCP's order, the
    truncation rank r (truncation_rank), strong-RRQR swaps at r, and again while the rank
    of the swapped factor differs (at most `rounds` times).  Returns (S, R, perm, r)."""
    S, R, perm = qrcp(P)
    r = truncation_rank(R, tau)
    for _ in range(rounds):
        S, R, perm, _ = strong_rrqr_swaps(P, perm, r, f)
        r_new = truncation_rank(R, tau)
        if r_new == r:
            break
        r = r_new
    return S, R, perm, r


def spectral_norm(A):
    """||A||_2 (largest singular value; numpy's SVD as a library primitive)."""
    if A.size == 0:
        return 0.0
    return float(np.linalg.svd(A, compute_uv=False)[0])


def truncation_rank(R, tau):
    """Alg. 7 step 3: the least r in 0..n with ||R[r:, r:]||_F <= tau * ||R||_2 (r = n always qualifies)."""
    n = R.shape[1]
    bound = tau * spectral_norm(R)
    for r in range(n + 1):
        if np.sqrt(np.sum(R[r:, r:] ** 2)) <= bound:
            return r
    return n


def forward_substitution(X, R):
    """Q with Q R = X, one column at a time: q_j = (x_j - sum_{i<j} q_i R_ij) / R_jj (rows independent)."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    Q = np.empty((m, n))
    for j in range(n):
        Q[:, j] = (X[:, j] - Q[:, :j] @ R[:j, j]) / R[j, j]
    return Q


def forward_substitution_f32(X, R):
    """forward_substitution in IEEE single precision: X and R rounded to float32 once, then every
    operation of q_j = (x_j - sum_{i<j} q_i R_ij) / R_jj in float32 (numpy float32 arithmetic).

    This is the bulk step of the multi-precision model of Sec. 1.3 and Sec. 5 with the working
    precision u = 2^-24 (the paper's float32 experiments, Sec. 6): the dominant operation in u, the
    sketch and the small factorization (done by the callers) in FP64.
    """
    X = np.asarray(X, dtype=np.float32)
    R = np.asarray(R, dtype=np.float32)
    m, n = X.shape
    Q = np.empty((m, n), dtype=np.float32)
    for j in range(n):
        acc = X[:, j].copy()
        for i in range(j):
            acc -= Q[:, i] * R[i, j]
        Q[:, j] = acc / R[j, j]
    return Q


def cholesky(A):
    """Upper R with R^T R = A (textbook column Cholesky); NotSPD(j) on a pivot <= 0."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    R = np.zeros((n, n))
    for j in range(n):
        d = A[j, j] - R[:j, j] @ R[:j, j]
        if not d > 0.0:
            raise NotSPD(j)
        R[j, j] = np.sqrt(d)
        R[j, j + 1:] = (A[j, j + 1:] - R[:j, j] @ R[:j, j + 1:]) / R[j, j]
    return R


def triangular_inverse(R):
    """R^{-1} for upper triangular R, by substitution against the identity."""
    n = R.shape[0]
    return forward_substitution(np.eye(n), R)
