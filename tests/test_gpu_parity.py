"""GPU parity: every stage of the CUDA path against the CPU FP64 oracle on the same seeded inputs.

Tolerances (stated per result; u = 2^-53):
* sketch P, column-wise relative (SKETCH_TOL): FP64 X 1e-12; FP32 X 1e-11
  (the tensor-core sketch keeps 3 exact 7-bit slices and rounds the last two
  in one fp32 accumulator, ~2^-39 of each 1024-row block's largest |x|);
  BF16 X 1e-6 (3 slices: 21 bits below the block's largest |x|).  All three
  are far below Assumptions 5.1's 0.1 u n^{-1/2} for the storage precision.
  Integer X: bit-exact.
* small QR / QRCP / Cholesky: R, S relative to column norms <= max(1e-12, 10 n u cond).
* forward substitution: Q column-relative <= max(1e-12, 10 n u cond(R)) in FP64;
  FP32 output: additionally 2^-23 (one rounding to float).
* Gram: relative 1e-13 (FP64 sums of exact products).
All sizes span several tiles and a ragged tail.
"""
import math

import numpy as np
import pytest
import torch

from oracle import linalg as olin
from oracle import rcqr as orc

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
SKETCH_TOL = {"f64": 1e-12, "f32": 1e-11, "bf16": 1e-6}


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2210_09953_gb300 import _binding
    return _binding


@pytest.fixture(scope="module")
def inputs():
    from paper_2210_09953_gb300 import inputs as inp
    return inp


DEV = "cuda"
DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def host64(t):
    """float64 numpy copy of a (column-major) device tensor."""
    return t.detach().to("cpu", torch.float64).numpy()


def colrel(A, B):
    den = np.linalg.norm(B, axis=0)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.linalg.norm(A - B, axis=0) / den))


# ----------------------------------------------------------------------------- sketch

@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n,k,off", [(1000, 1, 8, 0), (5037, 7, 64, 0), (20000, 64, 256, 37),
                                       (3001, 130, 264, 5)])
def test_sketch_parity(rc, inputs, prec, m, n, k, off):
    X = inputs.svd_matrix(m, n, 1e6, 11 + m, dtype=prec, device=DEV)
    cn = torch.empty(n, dtype=torch.float64, device=DEV)
    P = rc.rcqr_sketch(X, k, 0xABC + n, row_offset=off, colnorm2=cn)
    torch.cuda.synchronize()
    Xh = host64(X)
    Po = orc.sketch(Xh, k, 0xABC + n, row_offset=off)
    assert colrel(host64(P), Po) <= SKETCH_TOL[prec]
    assert np.max(np.abs(host64(cn) - np.sum(Xh * Xh, axis=0)) / np.sum(Xh * Xh, axis=0)) <= 1e-13


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_sketch_integer_input_is_bit_exact(rc, inputs, prec):
    m, n, k = 50021, 33, 72                 # |sum| < 2^14 * 2^16: every partial sum exact in FP64
    X = inputs.integer_matrix(m, n, 5, dtype=prec, device=DEV)
    P = rc.rcqr_sketch(X, k, 987654321)
    torch.cuda.synchronize()
    Po = orc.sketch(host64(X), k, 987654321)
    assert np.array_equal(host64(P), Po)


def test_sketch_shards_add_up(rc, inputs):
    m, n, k, a = 30000, 16, 64, 12345
    X = inputs.svd_matrix(m, n, 1e3, 3, dtype="f64", device=DEV)
    P = host64(rc.rcqr_sketch(X, k, 42))
    P1 = host64(rc.rcqr_sketch(X[:a], k, 42, row_offset=0))
    P2 = host64(rc.rcqr_sketch(X[a:], k, 42, row_offset=a))
    assert colrel(P1 + P2, P) <= 1e-13


def test_sketch_ld_larger_than_m(rc, inputs):
    X = inputs.svd_matrix(1000, 9, 1e2, 8, dtype="f32", device=DEV, ld=1024)
    assert X.stride() == (1, 1024)
    P = rc.rcqr_sketch(X, 32, 7)
    assert colrel(host64(P), orc.sketch(host64(X), 32, 7)) <= SKETCH_TOL["f32"]


# ----------------------------------------------------------------------------- small kernels

@pytest.mark.parametrize("k,n,cond", [(8, 1, 1.0), (64, 16, 1e4), (256, 64, 1e8), (520, 130, 1e10),
                                      (2048, 256, 1e3)])
def test_small_qr_parity(rc, inputs, k, n, cond):
    P = inputs.svd_matrix(k, n, cond, 17 + n, dtype="f64", device=DEV)
    S, R = rc.rcqr_small_qr(P)
    torch.cuda.synchronize()
    So, Ro = olin.householder_qr(host64(P))
    tol = max(1e-12, 10 * n * U * cond)
    assert colrel(host64(R), Ro) <= tol
    assert colrel(host64(S), So) <= tol
    Sg = host64(S)
    assert np.linalg.norm(Sg.T @ Sg - np.eye(n)) <= 100 * math.sqrt(k) * n * U
    assert np.all(np.diag(host64(R)) >= 0)


@pytest.mark.parametrize("k,n,cond", [(8, 1, 1.0), (72, 16, 1e4), (256, 64, 1e8), (520, 130, 1e10),
                                      (263, 7, 1e12), (2048, 256, 1e3), (300, 100, 1e6), (128, 128, 1e4),
                                      (512, 65, 1e8), (2000, 40, 1e8)])
def test_small_r_tree_parity(rc, inputs, k, n, cond):
    # R without S: the cluster kernel (k <= 512, n <= 128: columns spread over eight CTAs)
    # or the TSQR tree (leaf Householder QRs, then folds of stacked triangles)
    P = inputs.svd_matrix(k, n, cond, 19 + n, dtype="f64", device=DEV)
    R = rc.rcqr_small_qr(P, want_S=False)
    torch.cuda.synchronize()
    _, Ro = olin.householder_qr(host64(P))
    assert colrel(host64(R), Ro) <= max(1e-12, 10 * n * U * cond)
    assert np.all(np.diag(host64(R)) >= 0) and np.all(np.tril(host64(R), -1) == 0)


def test_qrcp_parity_planted_rank(rc, inputs):
    m, n, r, k = 4000, 24, 12, 96
    X = inputs.rank_deficient(m, n, r, 21, noise=1e-12, dtype="f64", device=DEV)
    cn = torch.empty(n, dtype=torch.float64, device=DEV)
    P = rc.rcqr_sketch(X, k, 5, colnorm2=cn)
    R, perm, rank, status = rc.rcqr_qrcp(P, 1e-8, colnorm2=cn)
    torch.cuda.synchronize()
    Ph, D = host64(P), np.sqrt(host64(cn))
    So, Ro, permo = olin.qrcp(Ph / D[None, :])
    ro = olin.truncation_rank(Ro, 1e-8)
    assert int(rank[0]) == ro == r
    assert perm.cpu().numpy().tolist() == permo.tolist()
    Rexp = np.zeros_like(Ro)
    Rexp[:ro] = Ro[:ro] * D[permo][None, :]
    assert colrel(host64(R)[:ro], Rexp[:ro]) <= 1e-10
    assert np.all(host64(R)[ro:] == 0)
    assert int(status[0]) == 0


def test_qrcp_zero_sketch_reports_rank0(rc):
    P = torch.zeros((64, 8), dtype=torch.float64, device=DEV).t().contiguous().t()
    R, perm, rank, status = rc.rcqr_qrcp(P, 1e-8)
    torch.cuda.synchronize()
    assert int(rank[0]) == 0 and int(status[0]) == -3


@pytest.mark.parametrize("n", [40, 128, 150])     # R' in shared memory up to n = 141, else in place
def test_chol_update_parity_and_failure(rc, inputs, n):
    G = inputs.gaussian_colmajor(500, n, 3, device=DEV)
    A = (G.t() @ G).t().contiguous().t()           # column-major SPD
    R0 = torch.triu(torch.randn(n, n, dtype=torch.float64, device=DEV)).t().contiguous().t()
    R = R0.clone()
    Rp, status = rc.rcqr_chol_update(A, R)
    torch.cuda.synchronize()
    Rpo = olin.cholesky(host64(A))
    assert int(status[0]) == 0
    assert colrel(host64(Rp), Rpo) <= 1e-13
    assert colrel(host64(R), Rpo @ host64(R0)) <= 1e-13
    B = A.clone()
    B[7, 7] = -1.0
    R2 = R0.clone()
    _, status = rc.rcqr_chol_update(B, R2)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [-2, 7]
    assert torch.equal(R2, R0)                      # R untouched on failure


# ----------------------------------------------------------------------------- bulk kernels

@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n,cond", [(1000, 1, 1.0), (4099, 17, 1e4), (20011, 64, 1e8), (3000, 200, 1e3),
                                      (2001, 100, 1e4), (5003, 256, 1e3)])
def test_trsm_parity(rc, inputs, prec, m, n, cond):
    X = inputs.svd_matrix(m, n, cond, 31 + n, dtype=prec, device=DEV)
    Rm = inputs.svd_matrix(4 * n, n, cond, 77, dtype="f64", device="cpu").numpy()
    _, Ro = olin.householder_qr(Rm)                 # an upper triangular R with cond ~ cond
    R = torch.from_numpy(Ro).to(DEV).t().contiguous().t()
    Q = rc.rcqr_trsm(X, R)
    torch.cuda.synchronize()
    Xh = host64(X)
    Qo = olin.forward_substitution(Xh, Ro)
    Qg = host64(Q)
    if prec == "f64":
        assert colrel(Qg, Qo) <= max(1e-12, 10 * n * U * cond)
    else:
        # FP32 substitution (the mixed path's working precision u = 2^-24): row-wise
        # backward error |X - Q R| <= (n + 3) u |Q||R| (Higham Thm 8.5, plus R and Q
        # rounded to float), hence a forward error <= (n + 3) u cond(R) column-wise.
        u32 = 2.0 ** -24
        E = np.abs(Xh - Qg @ Ro)
        assert np.all(E <= 2 * (n + 3) * u32 * (np.abs(Qg) @ np.abs(Ro)) + 1e-300)
        assert colrel(Qg, Qo) <= 2 * (n + 3) * u32 * cond + 2 * u32


def test_trsm_permuted_rank(rc, inputs):
    m, n, r = 5000, 12, 7
    X = inputs.svd_matrix(m, n, 1e2, 4, dtype="f64", device=DEV)
    perm = torch.tensor([3, 0, 11, 5, 6, 1, 9, 2, 4, 7, 8, 10], dtype=torch.int32, device=DEV)
    rank = torch.tensor([r], dtype=torch.int64, device=DEV)
    Ro = np.triu(np.random.default_rng(0).standard_normal((n, n))) + 3 * np.eye(n)
    R = torch.from_numpy(Ro).to(DEV).t().contiguous().t()
    Q = host64(rc.rcqr_trsm(X, R, perm=perm, rank=rank))
    Xh = host64(X)[:, perm.cpu().numpy()[:r]]
    Qo = olin.forward_substitution(Xh, Ro[:r, :r])
    assert colrel(Q[:, :r], Qo) <= 1e-12
    assert np.all(Q[:, r:] == 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("m,n", [(1000, 1), (7777, 33), (40000, 64), (3000, 256)])
def test_gram_parity(rc, inputs, prec, m, n):
    Q = inputs.gaussian_colmajor(m, n, 9, dtype=prec, device=DEV)
    A = rc.rcqr_gram(Q)
    torch.cuda.synchronize()
    Qh = host64(Q)
    Ao = Qh.T @ Qh
    if prec == "f64":
        assert np.max(np.abs(host64(A) - Ao)) <= 1e-13 * np.max(np.abs(Ao))
    else:
        # FP32 products summed in FP32 over 64-row chunks (<= 66 roundings each), the chunk
        # sums compensated: |dA| <= 66 u32 (|Q|^T |Q|) entrywise
        scale = np.abs(Qh).T @ np.abs(Qh)
        assert np.all(np.abs(host64(A) - Ao) <= 66 * 2.0 ** -24 * scale)


# ----------------------------------------------------------------------------- end to end

@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("m,n,k,cond", [(4096, 32, 128, 1e8), (20011, 64, 256, 1e4), (3001, 8, 16, 1e12)])
def test_factor_direct_parity(rc, inputs, prec, variant, m, n, k, cond):
    X = inputs.svd_matrix(m, n, cond, 1001 + n, dtype=prec, device=DEV)
    seed = 0x5EED0000 + n
    Q, R, _, rank, status = rc.rcqr_factor(X, k, seed, variant=variant)
    torch.cuda.synchronize()
    assert int(status[0]) == 0 and int(rank[0]) == n
    Xh = host64(X)
    if variant == 0:
        Qo, So, Ro = orc.rcholqr(Xh, k, seed)
    else:
        Qo, Ro, So = orc.rcholqr2(Xh, k, seed)
    Qg, Rg = host64(Q), host64(R)
    # stored X's condition number (rounding to f32/bf16 changes it)
    kap = orc.condition_number(Xh)
    ub = U if prec == "f64" else 2.0 ** -24          # unit roundoff of the bulk steps
    # backward error: X = Q R up to the bulk precision, at every condition number (Thm 5.2 (main1))
    assert np.linalg.norm(Qg @ Rg - Xh) / np.linalg.norm(Xh) <= max(1e-12, 10 * n * ub)
    if variant == 1 and prec == "f64":
        assert orc.orthogonality(Qg) <= max(1e-12, 100 * n * ub)
    # forward errors: R comes from the sketch (FP64-level) in pass 1; in pass 2 and in Q the
    # bulk precision enters amplified by cond -- checked where that product is small
    tol_r = max(1e-12, 10 * n * U * kap) + 10 * math.sqrt(n) * kap * (0 if prec == "f64" else SKETCH_TOL[prec])
    if variant == 1 and prec != "f64":
        tol_r += 10 * n * ub * kap
    if tol_r < 1e-2:
        assert colrel(Rg, Ro) <= tol_r
        if variant == 0:
            assert colrel(Qg, Qo) <= tol_r + 10 * n * ub * kap + 2 * ub
        elif prec != "f64":
            assert orc.orthogonality(Qg) <= 100 * n * ub


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("n", [32, 96])
def test_factor_rank_revealing_parity(rc, inputs, prec, variant, n):
    # n = 96 on the mixed path: the wide tensor-core substitution with the permutation and
    # the rank, and for RR2 the tensor-core Gram and the pass-2 product (zero beyond the rank)
    m, r, k = 20000, n // 2, 4 * n
    X = inputs.rank_deficient(m, n, r, 77, noise=1e-12, dtype=prec, device=DEV)
    tau = 1e-10 if prec == "f64" else 1e-5
    seed = 99
    Q, R, perm, rank, status = rc.rcqr_factor(X, k, seed, variant=variant, tau=tau)
    torch.cuda.synchronize()
    Xh = host64(X)
    if variant == 2:
        Qo, So, Ro, permo, ro = orc.rrrcholqr(Xh, k, seed, tau)
    else:
        Qo, Ro, permo, ro = orc.rrrcholqr2(Xh, k, seed, tau)
    assert int(status[0]) == 0
    assert int(rank[0]) == ro == r
    # the kept columns are decided by clear norm gaps; beyond the rank the remaining column
    # norms are noise of the size of the rounding (1e-12 relative), where the order of
    # near-ties may differ: compared as a set there
    pg = perm.cpu().numpy()
    assert pg[:r].tolist() == permo[:r].tolist()
    assert sorted(pg.tolist()) == list(range(n))
    Qg, Rg = host64(Q), host64(R)
    assert np.all(Qg[:, r:] == 0) and np.all(Rg[r:] == 0)
    uq = U if prec == "f64" else 2.0 ** -24
    D = np.linalg.norm(Xh, axis=0)
    E = (Xh[:, pg] - Qg[:, :r] @ Rg[:r]) / D[pg][None, :]
    assert np.linalg.norm(E) <= 2 * tau + 100 * uq
    # the two factorizations' products, each with its columns put back in X's order
    Pg, Po = np.empty_like(Xh), np.empty_like(Xh)
    Pg[:, pg] = Qg[:, :r] @ Rg[:r]
    Po[:, permo] = Qo @ Ro
    assert colrel(Pg, Po) <= max(1e-10, 100 * uq)
    if variant == 3:
        assert orc.orthogonality(Qg[:, :r]) <= max(1e-12, 100 * r * uq)


def test_factor_reports_indefinite_gram(rc, inputs):
    # two identical columns: the first pass divides by a zero pivot of R, the Gram is not SPD
    m, n = 2000, 4
    X = inputs.gaussian_colmajor(m, n, 2, device=DEV)
    X[:, 3] = X[:, 2]
    Q, R, _, rank, status = rc.rcqr_factor(X, 16, 1, variant=1)
    torch.cuda.synchronize()
    assert int(status[0]) in (-2, 0)    # ENOTSPD unless rounding keeps the copy independent
    if int(status[0]) == -2:
        assert 0 <= int(status[1]) < n


@pytest.mark.parametrize("use_L", [False, True])
def test_reduced_parity(rc, inputs, use_L):
    m, n, k, l = 10007, 16, 64, 5
    X = inputs.svd_matrix(m, n, 1e6, 5, dtype="f64", device=DEV)
    L = inputs.gaussian_colmajor(l, m, 8, device=DEV) if use_L else None
    Z, S, R, status = rc.rcqr_reduced(X, k, 3, L=L)
    torch.cuda.synchronize()
    Zo, So, Ro = orc.reduced(host64(X), k, 3, L=host64(L) if use_L else None)
    tol = max(1e-12, 10 * n * U * 1e6)
    assert colrel(host64(R), Ro) <= tol
    assert colrel(host64(S), So) <= tol
    assert np.max(np.abs(host64(Z) - Zo)) <= tol * max(1.0, np.max(np.abs(Zo)))


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("m,n", [(70001, 64), (5000, 17), (300, 48)])
def test_trsm_gram_fused_matches_separate_steps(rc, inputs, prec, m, n):
    """The fused pass: Q within the FP32 substitution's backward error (bit-identical to rcqr_trsm
    where both use the SIMT substitution, n <= 32), A within the compensated-Gram bound of the
    oracle Gram of that Q."""
    X = inputs.svd_matrix(m, n, 1e6, 900 + n, dtype=prec, device=DEV)
    k = (4 * n + 7) // 8 * 8
    R0 = rc.rcqr_small_qr(rc.rcqr_sketch(X, k, 77), want_S=False)
    Q, A = rc.rcqr_trsm_gram(X, R0)
    Qs = rc.rcqr_trsm(X, R0)
    torch.cuda.synchronize()
    if n <= 32:
        assert torch.equal(Q, Qs)
    Qh = host64(Q)
    Ro = host64(R0)
    E = np.abs(host64(X) - Qh @ Ro)
    assert np.all(E <= 2 * (n + 3) * 2.0 ** -24 * (np.abs(Qh) @ np.abs(Ro)) + 1e-300)
    Ao = Qh.T @ Qh
    scale = np.abs(Qh).T @ np.abs(Qh)
    assert np.all(np.abs(host64(A) - Ao) <= 66 * 2.0 ** -24 * scale)


def test_trsm_gram_rejects_fp64_and_wide(rc, inputs):
    X = inputs.svd_matrix(1000, 8, 10.0, 3, dtype="f64", device=DEV)
    R = inputs.to_colmajor(torch.eye(8, dtype=torch.float64, device=DEV))
    with pytest.raises(rc.RcqrError):
        rc.rcqr_trsm_gram(X, R, Q=rc.colmajor(1000, 8, torch.float32, DEV))
