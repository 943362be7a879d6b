"""Pins for the oracle's algorithms (Alg. 2, 3, 5, 7) against special cases and Sec. 5 bounds."""
import math

import numpy as np
import pytest

from oracle import linalg, rcqr, theta

U64 = np.finfo(np.float64).eps / 2


def svd_matrix(m, n, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.logspace(0, -math.log10(cond), n) if n > 1 else np.ones(1)
    return (U * s[None, :]) @ V.T, U


def rcholqr_violations(X, U, k, seed, kappa, Q, S, R):
    """Violated statements of Thm. 5.2 for Alg. 2 output (empty list when all hold)."""
    m, n = X.shape
    bad = []
    Th = theta.theta(seed, k, 0, m)
    eps = rcqr.embedding_epsilon(Th, U)
    s = np.linalg.svd(Q, compute_uv=False)
    slack = 4 * U64 * n ** 1.5 * kappa
    if not s.min() >= (1 + eps) ** -0.5 - slack:
        bad.append("sigma_min")
    if eps < 1 and not s.max() <= (1 - eps) ** -0.5 + slack:
        bad.append("sigma_max")
    dX = Q @ R - X
    if not np.all(np.linalg.norm(dX, axis=0) <= 2.1 * U64 * n * np.linalg.norm(X, axis=0)):
        bad.append("main1")
    if not np.linalg.norm(S - Th @ Q) <= 6.1 * U64 * n ** 1.5 * kappa:
        bad.append("main3")
    # Householder in uniform FP64 (not the u_f << u of Assumptions 5.1): O(sqrt(k) n u)
    if not np.linalg.norm(S.T @ S - np.eye(n)) <= 10 * math.sqrt(S.shape[0]) * n * U64:
        bad.append("S orthonormal")
    return bad


@pytest.mark.parametrize("kappa", [1e4, 1e8, 1e12])
def test_rcholqr_theorem_5_2(kappa):
    m, n, k = 3000, 12, 192          # k = 16 n: eps < 1 so both sides of (main2) are finite
    X, U = svd_matrix(m, n, kappa, 1)
    Q, S, R = rcqr.rcholqr(X, k, 77)
    assert rcholqr_violations(X, U, k, 77, kappa, Q, S, R) == []


def test_planted_mistakes_are_caught(monkeypatch):
    m, n, k, kappa = 2000, 8, 128, 1e6
    X, U = svd_matrix(m, n, kappa, 2)
    good = rcqr.rcholqr(X, k, 5)
    assert rcholqr_violations(X, U, k, 5, kappa, *good) == []
    # wrong scale of Theta (drop the 1/sqrt(k v)): sigma(Q) leaves the Thm. 5.2 interval
    monkeypatch.setattr(rcqr, "theta_scale", lambda kk: 1.3 / math.sqrt(kk * theta.table_variance()))
    assert rcholqr_violations(X, U, k, 5, kappa, *rcqr.rcholqr(X, k, 5))
    monkeypatch.undo()
    # transposed operand in the substitution
    real_fs = linalg.forward_substitution
    monkeypatch.setattr(linalg, "forward_substitution", lambda A, R: real_fs(A, R.T))
    assert rcholqr_violations(X, U, k, 5, kappa, *rcqr.rcholqr(X, k, 5))
    monkeypatch.undo()
    # dropped term in the substitution (the last off-diagonal contribution)
    def fs_dropped(A, R):
        Q = np.empty_like(A)
        for j in range(A.shape[1]):
            Q[:, j] = (A[:, j] - Q[:, :max(j - 1, 0)] @ R[:max(j - 1, 0), j]) / R[j, j]
        return Q
    monkeypatch.setattr(linalg, "forward_substitution", fs_dropped)
    assert rcholqr_violations(X, U, k, 5, kappa, *rcqr.rcholqr(X, k, 5))
    monkeypatch.undo()
    # sign error in a reflector update
    real_hqr = linalg.householder_qr
    monkeypatch.setattr(linalg, "householder_qr", lambda P: (lambda S, R: (S, -R))(*real_hqr(P)))
    assert rcholqr_violations(X, U, k, 5, kappa, *rcqr.rcholqr(X, k, 5))


def test_identity_sketch_reduces_to_householder_qr():
    # Theta = I (k = m): Alg. 2 becomes Householder QR of X itself
    X, _ = svd_matrix(50, 7, 1e3, 3)
    Q, S, R = rcqr.rcholqr_from_sketch(X, X)
    Ql, Rl = np.linalg.qr(X)
    sg = np.where(np.diag(Rl) < 0, -1.0, 1.0)
    assert np.max(np.abs(R - Rl * sg[:, None])) < 1e-13
    assert np.max(np.abs(Q - Ql * sg[None, :])) < 1e-12
    assert np.max(np.abs(S - Q)) < 1e-12


def test_single_column_closed_form():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((777, 1))
    Q, S, R = rcqr.rcholqr(x, 16, 3)
    P = theta.theta(3, 16, 0, 777) @ x
    assert R[0, 0] == pytest.approx(np.linalg.norm(P), rel=1e-14)
    assert np.allclose(Q, x / np.linalg.norm(P), rtol=1e-14, atol=0)


def test_sketch_exact_on_integers_bruteforce():
    rng = np.random.default_rng(9)
    m, n, k, seed = 300, 3, 16, 1234
    X = rng.integers(-128, 128, size=(m, n))
    G = theta.quantile_table().astype(np.int64)[theta.theta_bytes(seed, k, 0, m)]
    exact = [[sum(int(G[i, r]) * int(X[r, j]) for r in range(m)) for j in range(n)] for i in range(k)]
    P = rcqr.sketch(X.astype(np.float64), k, seed)
    assert np.array_equal(P, theta.theta_scale(k) * np.array(exact, dtype=np.float64))


def test_sketch_is_additive_over_row_shards():
    X, _ = svd_matrix(5000, 6, 1e2, 4)
    P = rcqr.sketch(X, 32, 42)
    P2 = rcqr.sketch(X[:1234], 32, 42) + rcqr.sketch(X[1234:], 32, 42, row_offset=1234)
    assert np.max(np.abs(P - P2)) < 1e-13 * np.max(np.abs(P))


@pytest.mark.parametrize("kappa", [1e4, 1e12])
def test_rcholqr2_orthonormal_and_matches_householder_R(kappa):
    m, n, k = 4000, 16, 64
    X, _ = svd_matrix(m, n, kappa, 5)
    Q, R, S = rcqr.rcholqr2(X, k, 11)
    assert rcqr.orthogonality(Q) < 10 * n * U64
    res_f, res_c = rcqr.residuals(X, Q, R)
    assert res_f < 10 * n * U64 and res_c < 10 * n * U64
    _, Rh = np.linalg.qr(X)
    Rh *= np.where(np.diag(Rh) < 0, -1.0, 1.0)[:, None]
    # the R of an orthonormal-Q factorization is unique: pass 2 recovers Householder's R
    assert np.max(np.abs(R - Rh) / np.abs(Rh).max(axis=0)[None, :]) < 10 * n * U64 * (1 + kappa * U64 * 1e3)


def test_reduced_with_theta_returns_sketch_of_Q():
    m, n, k, kappa = 3000, 10, 160, 1e6
    X, U = svd_matrix(m, n, kappa, 6)
    Z, S, R = rcqr.reduced(X, k, 21)
    Q, S1, R1 = rcqr.rcholqr(X, k, 21)
    assert np.array_equal(S, S1) and np.array_equal(R, R1)
    # Z = P R^{-1} is the sketch of Q; it equals S up to Thm. 5.4-size rounding
    assert np.linalg.norm(Z - S) <= 6.1 * U64 * n ** 1.5 * kappa
    Th = theta.theta(21, k, 0, m)
    assert np.linalg.norm(Z - Th @ Q) <= 6.1 * U64 * n ** 1.5 * kappa


def test_reduced_with_explicit_extractor_rows():
    m, n, k, l, kappa = 2000, 8, 128, 5, 1e5
    X, _ = svd_matrix(m, n, kappa, 7)
    L = np.random.default_rng(1).standard_normal((l, m))
    Z, S, R = rcqr.reduced(X, k, 3, L=L)
    Q, _, _ = rcqr.rcholqr(X, k, 3)
    # Thm. 5.4 first bound: ||Z_i - L_i Q|| <= 3.5 u n^{3/2} kappa ||L_i||
    err = np.linalg.norm(Z - L @ Q, axis=1)
    assert np.all(err <= 3.5 * U64 * n ** 1.5 * kappa * np.linalg.norm(L, axis=1))


def test_rrrcholqr_planted_rank_and_theorem_5_7():
    rng = np.random.default_rng(12)
    m, n, r, k = 3000, 16, 8, 64
    B = rng.standard_normal((m, r)) * rng.uniform(0.1, 10, size=r)[None, :]
    X = np.hstack([B, B @ rng.standard_normal((r, n - r)) + 1e-12 * rng.standard_normal((m, n - r))])
    tau = 1e-8
    Q, S, R, perm, rr = rcqr.rrrcholqr(X, k, 5, tau)
    assert rr == r
    assert sorted(perm.tolist()) == list(range(n))
    # Thm. 5.7: column-normalised residual <= 2 tau (up to rounding), Q well conditioned
    D = rcqr.column_norms(X)
    E = (X[:, perm] - Q @ R) / D[perm][None, :]
    assert np.linalg.norm(E) <= 2 * tau + 1e-13
    Th = theta.theta(5, k, 0, m)
    Uq, _ = np.linalg.qr(Q)
    eps = rcqr.embedding_epsilon(Th, Uq)
    s = np.linalg.svd(Q, compute_uv=False)
    assert s.min() >= (1 + eps) ** -0.5 - 0.016
    if eps < 1:
        assert s.max() <= (1 - eps) ** -0.5 + 0.016
    assert np.linalg.norm(S - Th @ Q) <= 0.061
    Q2, R2, perm2, r2 = rcqr.rrrcholqr2(X, k, 5, tau)
    assert r2 == r and np.array_equal(perm2, perm)
    assert rcqr.orthogonality(Q2) < 100 * U64 * n


def test_rrrcholqr_full_rank_is_permuted_rcholqr():
    X, _ = svd_matrix(1500, 6, 1e3, 13)
    Q, S, R, perm, r = rcqr.rrrcholqr(X, 48, 9, 1e-15)
    assert r == 6
    res_f, res_c = rcqr.residuals(X, Q, R, perm)
    assert res_c < 50 * U64 * 6


def test_cholqr_pass_reports_indefinite_gram():
    Q = np.ones((4, 2))                                   # Gram [[4,4],[4,4]]: second pivot is exactly 0
    with pytest.raises(linalg.NotSPD) as e:
        rcqr.cholqr_pass(Q, np.eye(2))
    assert e.value.j == 1


@pytest.mark.parametrize("row_offset", [0, 5, 17, 12345])
def test_sketch_rows_selects_rows_of_the_sketch(row_offset):
    """sketch_rows (the checker of the full-size GPU tests) equals the selected rows of sketch,
    bit for bit on integer X (every partial sum exact), for offsets that are not multiples of the
    16-row Philox counter block and for row blocks that split X unevenly."""
    rng = np.random.default_rng(row_offset + 3)
    m, n, k = 1000, 5, 40
    X = rng.integers(-128, 128, (m, n)).astype(np.float64)
    rows = np.array([39, 0, 17, 8, 9, 38])
    full = rcqr.sketch(X, k, 0xC0FFEE, row_offset=row_offset, row_block=333)
    sel = rcqr.sketch_rows(X, k, 0xC0FFEE, rows, row_offset=row_offset, row_block=157)
    assert np.array_equal(sel, full[rows])
    # and a wrong offset is caught (Theta's columns are tied to the global row index)
    off_by_one = rcqr.sketch_rows(X, k, 0xC0FFEE, rows, row_offset=row_offset + 1, row_block=157)
    assert not np.array_equal(off_by_one, full[rows])


def test_rcholqr_f32_well_conditioned_q():
    """Alg. 2 with a float32 substitution: Q has the backward error of the float32 substitution and
    stays well conditioned while u32 * cond stays small (Thm. 5.2 with u = 2^-24)."""
    m, n, k, kappa = 4000, 16, 256, 1e3        # k = 16 n: eps < 1, both sides of (main2) finite
    X, U = svd_matrix(m, n, kappa, 9)
    Q, S, R = rcqr.rcholqr_f32(X, k, 21)
    Th = theta.theta(21, k, 0, m)
    eps = rcqr.embedding_epsilon(Th, U)
    s = np.linalg.svd(Q.astype(np.float64), compute_uv=False)
    slack = 4 * 2.0 ** -24 * n ** 1.5 * kappa
    assert eps < 1
    assert (1 + eps) ** -0.5 - slack <= s.min() and s.max() <= (1 - eps) ** -0.5 + slack
    assert np.linalg.norm(S - Th @ Q.astype(np.float64)) <= 6.1 * 2.0 ** -24 * n ** 1.5 * kappa


def test_rademacher_sketch_exact_on_integers_bruteforce():
    rng = np.random.default_rng(19)
    m, n, k, seed, off = 333, 3, 24, 4321, 90
    X = rng.integers(-128, 128, size=(m, n))
    Sg = theta.rademacher_signs(seed, k, off, m).astype(np.int64)
    exact = [[sum(int(Sg[i, r]) * int(X[r, j]) for r in range(m)) for j in range(n)] for i in range(k)]
    P = rcqr.sketch(X.astype(np.float64), k, seed, row_offset=off, dist=theta.RADEMACHER)
    assert np.array_equal(P, (1.0 / np.sqrt(k)) * np.array(exact, dtype=np.float64))


def test_srht_sketch_exact_on_integers_bruteforce():
    # the SRHT through the same row-blocked sketch: sqrt(k) P is the integer product S H D X
    rng = np.random.default_rng(23)
    m, n, k, seed, off = 301, 3, 20, 98765, 45
    X = rng.integers(-128, 128, size=(m, n))
    Sg = theta.srht_signs(seed, k, off, m).astype(np.int64)
    exact = [[sum(int(Sg[i, r]) * int(X[r, j]) for r in range(m)) for j in range(n)] for i in range(k)]
    P = rcqr.sketch(X.astype(np.float64), k, seed, row_offset=off, dist=theta.SRHT, row_block=64)
    assert np.array_equal(P, (1.0 / np.sqrt(k)) * np.array(exact, dtype=np.float64))


def test_rcholqr2_with_srht_theta():
    # an SRHT embedding serves Alg. 3 like the Gaussian one (Sec. 2; the paper's figures use it)
    m, n, k, kappa = 3000, 10, 80, 1e6
    X, _ = svd_matrix(m, n, kappa, 29)
    Q, R, _ = rcqr.rcholqr2(X, k, 9, dist=theta.SRHT)
    _, Rh = linalg.householder_qr(X)
    assert rcqr.orthogonality(Q) <= 100 * n * U64
    assert np.max(np.abs(R - Rh) / np.abs(Rh).max(axis=0)[None, :]) <= 10 * n * U64 * kappa


def test_rcholqr2_with_rademacher_theta():
    # a Rademacher embedding serves Alg. 3 like the Gaussian one: R equals Householder R of X
    m, n, k, kappa = 3000, 10, 80, 1e6
    X, _ = svd_matrix(m, n, kappa, 23)
    Q, R, _ = rcqr.rcholqr2(X, k, 8, dist=theta.RADEMACHER)
    _, Rh = linalg.householder_qr(X)
    assert rcqr.orthogonality(Q) <= 100 * n * U64
    assert np.max(np.abs(R - Rh) / np.abs(Rh).max(axis=0)[None, :]) <= 10 * n * U64 * kappa


def test_implicit_rcholqr2_is_the_explicit_one():
    # Alg. 3 without step 4: Q1 Rp^{-1} is the Q of Alg. 3 (the same substitution), R the same R,
    # and the two products of the implicit Q agree with the explicit Q
    m, n, k, kappa = 2500, 9, 72, 1e7
    X, _ = svd_matrix(m, n, kappa, 31)
    Q, R, _ = rcqr.rcholqr2(X, k, 17)
    Q1, R2, Rp = rcqr.rcholqr2_implicit(X, k, 17)
    assert np.array_equal(R2, R)
    assert np.array_equal(linalg.forward_substitution(Q1, Rp), Q)
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((n, 4))
    B = rng.standard_normal((m, 3))
    assert np.linalg.norm(rcqr.implicit_q_times(Q1, Rp, Y) - Q @ Y) <= 1e-12 * np.linalg.norm(Y)
    assert np.linalg.norm(rcqr.implicit_qt_times(Q1, Rp, B) - Q.T @ B) <= 1e-12 * np.linalg.norm(B)
    # a transposed Rp in the left product is caught
    bad = linalg.forward_substitution((Q1.T @ B).T, Rp.T.copy()).T
    assert np.linalg.norm(bad - Q.T @ B) > 1e-6 * np.linalg.norm(B)


def test_column_oriented_rcholqr_one_block_is_rcholqr():
    # Alg. 4 with a single block is Alg. 2 step by step
    m, n, k = 2000, 8, 64
    X, _ = svd_matrix(m, n, 1e5, 41)
    Q, S, R = rcqr.col_rcholqr(X, n, k, 9)
    Q2, S2, R2 = rcqr.rcholqr(X, k, 9)
    assert np.array_equal(R, R2) and np.array_equal(S, S2) and np.array_equal(Q, Q2)


@pytest.mark.parametrize("rgs", [False, True])
@pytest.mark.parametrize("kappa", [1e3, 1e9])
def test_column_oriented_rcholqr_matches_thm_5_2(rgs, kappa):
    # "numerically equivalent to Alg. 2": block by block, the same Thm. 5.2 statements hold
    m, n, k, b = 3000, 12, 192, 4
    X, U = svd_matrix(m, n, kappa, 43)
    Q, S, R = rcqr.col_rcholqr(X, b, k, 77, rgs=rgs)
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    assert np.all(np.linalg.norm(Q @ R - X, axis=0) <= 2.1 * U64 * n * np.linalg.norm(X, axis=0) * 10)
    Th = theta.theta(77, k, 0, m)
    eps = rcqr.embedding_epsilon(Th, U)
    s = np.linalg.svd(Q, compute_uv=False)
    slack = 4 * U64 * n ** 1.5 * kappa
    assert s.min() >= (1 + eps) ** -0.5 - slack and s.max() <= (1 - eps) ** -0.5 + slack
    # the same R as Alg. 2 up to its forward error (the blocks are solved in the same order)
    _, _, R2 = rcqr.rcholqr(X, k, 77)
    assert np.max(np.abs(R - R2) / np.abs(R2).max(axis=0)[None, :]) <= 10 * n * U64 * kappa + 1e-13
    if rgs:
        assert np.linalg.norm(S - Th @ Q) <= 1e-12 * np.sqrt(n)        # S is the sketch of Q
    else:
        # S orthonormal up to the loss of the one-projection (least-squares) step, O(n u kappa)
        assert np.linalg.norm(S.T @ S - np.eye(n)) <= 100 * n * U64 * kappa
