"""Pins for the oracle's small dense kernels against closed forms, invariants and library routines."""
import itertools

import numpy as np
import pytest
import scipy.linalg

from oracle import linalg

U64 = np.finfo(np.float64).eps / 2


def _sign_fixed_numpy_qr(P):
    Q, R = np.linalg.qr(P)
    s = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * s[None, :], R * s[:, None]


@pytest.mark.parametrize("k,n", [(8, 1), (12, 5), (64, 16), (200, 37)])
def test_householder_invariants_and_library(k, n):
    rng = np.random.default_rng(k * 100 + n)
    P = rng.standard_normal((k, n)) * np.logspace(0, -6, n)[None, :]
    S, R = linalg.householder_qr(P)
    assert np.allclose(np.tril(R, -1), 0)
    assert np.all(np.diag(R) > 0)
    assert np.linalg.norm(S.T @ S - np.eye(n)) < 50 * k * U64
    assert np.linalg.norm(S @ R - P) < 50 * k * U64 * np.linalg.norm(P)
    Sl, Rl = _sign_fixed_numpy_qr(P)                   # LAPACK geqrf, signs fixed the same way
    assert np.max(np.abs(R - Rl) / np.abs(Rl).max(axis=0)[None, :]) < 1e-12
    assert np.max(np.abs(S - Sl)) < 1e-9


def test_householder_single_column_closed_form():
    p = np.array([[3.0], [-4.0], [12.0]])
    S, R = linalg.householder_qr(p)
    assert R[0, 0] == pytest.approx(13.0, rel=1e-15)
    assert np.allclose(S[:, 0], p[:, 0] / 13.0, rtol=0, atol=1e-16)


def test_householder_negative_leading_entry_and_zero_column():
    P = np.array([[-2.0, 0.0], [0.0, 0.0], [0.0, 0.0]])
    S, R = linalg.householder_qr(P)
    assert R[0, 0] == 2.0 and S[0, 0] == -1.0
    assert R[1, 1] == 0.0


def test_qrcp_pivots_and_factorisation():
    rng = np.random.default_rng(5)
    P = rng.standard_normal((40, 9)) * np.array([1, 10, 0.1, 3, 3, 0.5, 7, 2, 1e-3])[None, :]
    S, R, perm = linalg.qrcp(P)
    assert sorted(perm.tolist()) == list(range(9))
    assert np.linalg.norm(P[:, perm] - S @ R) < 1e-13 * np.linalg.norm(P)
    assert np.linalg.norm(S.T @ S - np.eye(9)) < 1e-13
    d = np.abs(np.diag(R))
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-13))        # non-increasing diagonal
    # Brute force: each pivot maximises the norm of the column's residual after
    # projecting out the span of the columns already chosen.
    chosen = []
    for j in range(9):
        if chosen:
            B, _ = np.linalg.qr(P[:, chosen])
            Res = P - B @ (B.T @ P)
        else:
            Res = P
        norms = np.linalg.norm(Res, axis=0)
        norms[chosen] = -1
        assert perm[j] == int(np.argmax(norms))
        chosen.append(perm[j])


def test_qrcp_ties_go_to_lowest_index():
    P = np.eye(4)[:, [0, 1, 2]] * np.array([1.0, 2.0, 2.0])[None, :]
    _, _, perm = linalg.qrcp(np.vstack([P, np.zeros((1, 3))]))
    assert perm.tolist() == [1, 2, 0]


def test_truncation_rank_planted():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((60, 6))
    B = np.hstack([A, A @ rng.standard_normal((6, 4)) + 1e-12 * rng.standard_normal((60, 4))])
    _, R, _ = linalg.qrcp(B)
    assert linalg.truncation_rank(R, 1e-8) == 6
    assert linalg.truncation_rank(R, 1e-16) == 10
    assert linalg.truncation_rank(np.zeros((3, 3)), 1e-8) == 0
    # brute-force definition on a tiny triangle
    R = np.triu(rng.standard_normal((4, 4))) * np.array([1, 1e-3, 1e-9, 1e-12])[:, None]
    tau = 1e-6
    norm2 = np.linalg.norm(R, 2)
    expect = min(r for r in range(5) if np.linalg.norm(R[r:, r:]) <= tau * norm2)
    assert linalg.truncation_rank(R, tau) == expect


def test_forward_substitution_backward_stable_and_library():
    rng = np.random.default_rng(2)
    n = 24
    R = np.triu(rng.standard_normal((n, n))) + 5 * np.eye(n)
    X = rng.standard_normal((300, n))
    Q = linalg.forward_substitution(X, R)
    # Higham Thm 8.5 (cited in Sec. 5.1): |X - Q R| <= 1.1 n u |Q||R| row-wise
    assert np.all(np.abs(X - Q @ R) <= 1.1 * n * U64 * (np.abs(Q) @ np.abs(R)) + 1e-300)
    ref = scipy.linalg.solve_triangular(R.T, X.T, lower=True).T
    assert np.max(np.abs(Q - ref)) < 1e-12 * np.max(np.abs(ref))


def test_cholesky_library_and_failure():
    rng = np.random.default_rng(4)
    G = rng.standard_normal((50, 12))
    A = G.T @ G
    R = linalg.cholesky(A)
    assert np.allclose(np.tril(R, -1), 0) and np.all(np.diag(R) > 0)
    assert np.linalg.norm(R.T @ R - A) < 1e-13 * np.linalg.norm(A)
    assert np.max(np.abs(R - np.linalg.cholesky(A).T)) < 1e-12 * np.abs(R).max()
    B = A.copy()
    B[5, 5] = -1.0
    with pytest.raises(linalg.NotSPD) as e:
        linalg.cholesky(B)
    # pivots 0..4 are those of A; pivot 5 is the first that can fail
    assert e.value.j == 5


def test_triangular_inverse_tiny_bruteforce():
    for vals in itertools.product([1.0, -2.0], [0.5, 3.0], [4.0]):
        R = np.array([[vals[0], 1.0, 2.0], [0.0, vals[1], -1.0], [0.0, 0.0, vals[2]]])
        assert np.allclose(linalg.triangular_inverse(R) @ R, np.eye(3), atol=1e-15)


def test_forward_substitution_f32_backward_error_and_exact_case():
    # Higham Thm 8.5 for the float32 substitution: |X - Q R| <= (n + 2) u32 |Q||R| entrywise (X, R
    # rounded to float32 first); a dropped term, a transposed R or a wrong index breaks it at once
    rng = np.random.default_rng(4)
    m, n = 300, 24
    R = np.triu(rng.standard_normal((n, n))) + 4 * np.eye(n)
    X = rng.standard_normal((m, n))
    Q = linalg.forward_substitution_f32(X, R).astype(np.float64)
    X32, R32 = X.astype(np.float32).astype(np.float64), R.astype(np.float32).astype(np.float64)
    u32 = 2.0 ** -24
    assert np.all(np.abs(X32 - Q @ R32) <= (n + 2) * u32 * (np.abs(Q) @ np.abs(R32)) + 1e-30)
    bad = linalg.forward_substitution_f32(X, R.T.copy()).astype(np.float64)   # transposed operand
    assert not np.all(np.abs(X32 - bad @ R32) <= (n + 2) * u32 * (np.abs(bad) @ np.abs(R32)))
    # small integers, unit upper triangular integer R: every float32 operation is exact
    Ri = np.triu(rng.integers(-3, 4, (8, 8)).astype(np.float64), 1) + np.eye(8)
    Qi = rng.integers(-5, 6, (50, 8)).astype(np.float64)
    assert np.array_equal(linalg.forward_substitution_f32(Qi @ Ri, Ri).astype(np.float64), Qi)


def kahan(n, theta=1.2, pert=1e-10):
    """The Kahan matrix diag(1, s, .., s^{n-1}) (I - c U), U strictly upper all-ones (every
    trailing column norm is s^t at step t), with column j scaled by (1 - pert j) so that
    column pivoting keeps the natural order."""
    c, s = np.cos(theta), np.sin(theta)
    K = np.triu(-c * np.ones((n, n)), 1) + np.eye(n)
    K = np.diag(s ** np.arange(n)) @ K
    return K * (1 - pert * np.arange(n))[None, :]


def test_swap_ratio_is_the_determinant_growth_of_a_swap():
    # Gu & Eisenstat Lemma 3.1: sqrt(rho_ij) = |det R11'| / |det R11| after columns i and r + j
    # trade places; det R11' from numpy's QR of the swapped matrix (a library routine)
    rng = np.random.default_rng(11)
    P = rng.standard_normal((14, 6)) @ np.diag([3, 1, 0.5, 0.2, 1e-2, 1e-3])
    _, R = linalg.householder_qr(P)
    for r in range(1, 6):
        rho = linalg.swap_ratios(R, r)
        d0 = abs(np.prod(np.diag(R)[:r]))
        for i in range(r):
            for j in range(6 - r):
                perm = np.arange(6)
                perm[[i, r + j]] = perm[[r + j, i]]
                _, Rs = np.linalg.qr(P[:, perm])
                d1 = abs(np.prod(np.diag(Rs)[:r]))
                assert abs(np.sqrt(rho[i, j]) - d1 / d0) <= 1e-10 * max(1.0, d1 / d0)


def test_strong_rrqr_fixes_the_kahan_matrix():
    n, r, f = 24, 23, 1.5
    P = np.vstack([kahan(n), np.zeros((8, n))])
    S0, R0, perm0 = linalg.qrcp(P)
    assert perm0.tolist() == list(range(n))                        # no pivoting on Kahan's matrix
    assert np.max(linalg.swap_ratios(R0, r)) > f * f               # ... and it is not a strong RRQR
    S, R, perm, swaps = linalg.strong_rrqr_swaps(P, perm0, r, f)
    assert swaps >= 1
    assert np.max(linalg.swap_ratios(R, r)) <= f * f
    # Gu-Eisenstat Thm 3.2 with q(r, n) = sqrt(1 + f^2 r (n - r))
    sv = np.linalg.svd(P, compute_uv=False)
    q = np.sqrt(1 + f * f * r * (n - r))
    assert np.linalg.svd(R[:r, :r], compute_uv=False).min() >= sv[r - 1] / q * (1 - 1e-10)
    assert np.linalg.norm(R[r:, r:], 2) <= sv[r] * q * (1 + 1e-10)
    # a valid QR of the permuted matrix
    assert np.allclose(S @ R, P[:, perm], atol=1e-13)
    assert np.linalg.norm(S.T @ S - np.eye(n)) <= 1e-13
    assert np.all(np.diag(R) >= 0) and np.array_equal(R, np.triu(R))
    assert sorted(perm.tolist()) == list(range(n))


def test_strong_rrqr_rank_and_local_maximality():
    rng = np.random.default_rng(5)
    m, n, r = 60, 9, 5
    B = rng.standard_normal((m, r))
    P = np.hstack([B, B @ rng.standard_normal((r, n - r)) + 1e-9 * rng.standard_normal((m, n - r))])
    P = P[:, rng.permutation(n)]
    S, R, perm, rk = linalg.strong_rrqr(P, 1e-6, 1.5)
    assert rk == r
    # no single swap grows |det R11| by more than f (brute force over all swaps)
    d0 = abs(np.prod(np.diag(R)[:r]))
    for i in range(r):
        for j in range(n - r):
            pp = perm.copy()
            pp[[i, r + j]] = pp[[r + j, i]]
            _, Rs = np.linalg.qr(P[:, pp])
            assert abs(np.prod(np.diag(Rs)[:r])) <= 1.5 * d0 * (1 + 1e-9)
