"""GPU parity of the tensor-core blocked substitution fused with the Gram matrix (rcqr_trsm_gram,
32 < n <= 64, FP32 / BF16 X), and of the FP32 SIMT substitution (rcqr_trsm) beside it, against the
oracle.

Tolerances (u = 2^-24, the mixed path's working precision):
* Q = X R^{-1}: the row-wise backward error of an FP32 substitution, |X - Q R| <=
  2 (n + 3) u |Q||R| entrywise (Higham Thm. 8.5; the off-diagonal blocks' products are
  exact three-piece bf16 splits summed in FP32, so they keep that bound), and the forward
  error against the FP64 oracle substitution, column-wise <= 2 (n + 3) u cond(R) + 2 u.
* A = Q^T Q from the fused pass: |A - Q^T Q| <= 66 u (|Q|^T |Q|) entrywise, Q^T Q in FP64
  from the returned Q (the bound the compensated FP32 Gram states).
Shapes: a single partial tile (m < 128), exact multiples of the 128-row tile, ragged tails,
n = 33 (one used column in the last 16-column block), n = 48, 64, a permuted rank-deficient
call (the rank-revealing form of Alg. 7 step 4) and Q in place of X (Alg. 3 step 4).
The last test checks the second pass's product with the explicit inverse (bound stated
there) for 16 < n <= 128.
"""
import numpy as np
import pytest
import torch

from oracle import linalg as olin

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
DEV = "cuda"


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


def host64(t):
    return t.detach().to("cpu", torch.float64).numpy()


def colrel(A, B):
    den = np.linalg.norm(B, axis=0)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.linalg.norm(A - B, axis=0) / den))


def upper_r(n, cond, seed):
    from paper_2210_09953_gb300 import inputs as inp
    Rm = inp.svd_matrix(4 * n, n, cond, seed, dtype="f64", device="cpu").numpy()
    _, Ro = olin.householder_qr(Rm)
    return Ro


def check_substitution(Xh, Qg, Ro, n, cond):
    E = np.abs(Xh - Qg @ Ro)
    assert np.all(E <= 2 * (n + 3) * U32 * (np.abs(Qg) @ np.abs(Ro)) + 1e-300)
    Qo = olin.forward_substitution(Xh, Ro)
    assert colrel(Qg, Qo) <= 2 * (n + 3) * U32 * cond + 2 * U32


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,cond", [(77, 40, 1e3), (128, 64, 1e2), (5000, 33, 1e4), (70001, 64, 1e6),
                                      (32768, 48, 1e8), (100003, 57, 1e2)])
def test_tc_substitution_and_fused_gram(rc, inputs, prec, m, n, cond):
    X = inputs.svd_matrix(m, n, cond, 500 + n, dtype=prec, device=DEV)
    Ro = upper_r(n, cond, 90 + n)
    R = torch.from_numpy(Ro).to(DEV).t().contiguous().t()
    Q = rc.rcqr_trsm(X, R)
    Qf, A = rc.rcqr_trsm_gram(X, R)
    torch.cuda.synchronize()
    Xh, Qg = host64(X), host64(Qf)
    check_substitution(Xh, Qg, Ro, n, cond)           # tensor-core blocked substitution
    check_substitution(Xh, host64(Q), Ro, n, cond)    # SIMT substitution
    Ao = Qg.T @ Qg
    scale = np.abs(Qg).T @ np.abs(Qg)
    assert np.all(np.abs(host64(A) - Ao) <= 66 * U32 * scale)
    assert np.array_equal(host64(A), host64(A).T)


def test_tc_substitution_permuted_rank(rc, inputs):
    m, n, r = 20000, 64, 37
    X = inputs.svd_matrix(m, n, 1e2, 6, dtype="f32", device=DEV)
    perm_h = np.random.default_rng(1).permutation(n).astype(np.int32)
    perm = torch.from_numpy(perm_h).to(DEV)
    rank = torch.tensor([r], dtype=torch.int64, device=DEV)
    Ro = np.triu(np.random.default_rng(0).standard_normal((n, n))) + 8 * np.eye(n)
    R = torch.from_numpy(Ro).to(DEV).t().contiguous().t()
    Qs = host64(rc.rcqr_trsm(X, R, perm=perm, rank=rank))
    Qf, A = rc.rcqr_trsm_gram(X, R, perm=perm, rank=rank)
    torch.cuda.synchronize()
    Q = host64(Qf)
    Xs = host64(X)[:, perm_h[:r]]
    R11 = Ro[:r, :r].astype(np.float32).astype(np.float64)
    check_substitution(Xs, Q[:, :r], R11, r, np.linalg.cond(R11))
    check_substitution(Xs, Qs[:, :r], R11, r, np.linalg.cond(R11))
    assert np.all(Q[:, r:] == 0) and np.all(Qs[:, r:] == 0)
    Ag = host64(A)
    assert np.all(Ag[r:, :] == 0) and np.all(Ag[:, r:] == 0)


def test_tc_substitution_in_place(rc, inputs):
    # Alg. 3 step 4: Q <- Q R'^{-1} with Q overwritten row by row
    m, n = 50001, 64
    X = inputs.svd_matrix(m, n, 1e3, 12, dtype="f32", device=DEV)
    Ro = upper_r(n, 10.0, 13)
    R = torch.from_numpy(Ro).to(DEV).t().contiguous().t()
    Xh = host64(X)
    Qs = host64(rc.rcqr_trsm(X.clone(), R))
    Y = X.clone()
    rc.rcqr_trsm(Y, R, Q=Y)
    torch.cuda.synchronize()
    assert np.array_equal(host64(Y), Qs)
    check_substitution(Xh, Qs, Ro, n, 10.0)


# ----------------------------------------------------------------------------- pass 2 by the explicit inverse
# Alg. 3 step 4 on the mixed path, Q <- Q1 W with W = R'^{-1} (FP64) as a tensor-core
# product whose leading term is exact (gemm_tc.cu).  Q1 and R' come from
# rcqr_factor_implicit, which runs the same kernels as rcqr_factor up to Alg. 3 step 3.
# Bound, entrywise: every entry of Q1 and of W is represented to 2^-22 of itself (an
# 8-bit digit and two FP16 pieces after scaling by 2^(14 - e) per row of Q1 / column of
# W), except that the last piece has an absolute resolution of 2^-24 scaled units
# (FP16 subnormals), 2^-38 of the row's or column's largest entry; the one product
# dropped is below 2^-22 of |q||w|, and the result is rounded to FP32 once:
#   |Q - Q1 W| <= 2^-20 (|Q1| |W|) + 2^-36 (rowsum |Q1| colmax |W| + rowmax |Q1| colsum |W|)
#                 + 2 u |Q|,  u = 2^-24.

@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,k,cond", [(30011, 64, 256, 1e8), (20000, 100, 400, 1e8), (9001, 128, 512, 1e12),
                                        (1000, 40, 160, 1e4), (257, 17, 72, 1e6)])
def test_pass2_product_with_explicit_inverse(rc, inputs, prec, m, n, k, cond):
    X = inputs.svd_matrix(m, n, cond, 700 + n, dtype=prec, device=DEV)
    Q1, R1, Rp, st1 = rc.rcqr_factor_implicit(X, k, 31)
    Q, R, _, _, st2 = rc.rcqr_factor(X, k, 31, variant=rc.DIRECT2)
    torch.cuda.synchronize()
    assert int(st1[0]) == 0 and int(st2[0]) == 0
    Q1h, Rph, Qh = host64(Q1), host64(Rp), host64(Q)
    W = olin.triangular_inverse(Rph)
    E = np.abs(Qh - Q1h @ W)
    aQ, aW = np.abs(Q1h), np.abs(W)
    tiny = aQ.sum(1, keepdims=True) * aW.max(0, keepdims=True) + aQ.max(1, keepdims=True) * aW.sum(0, keepdims=True)
    assert np.all(E <= 2.0 ** -20 * (aQ @ aW) + 2.0 ** -36 * tiny + 2 * U32 * np.abs(Qh))
    from oracle import rcqr as orc
    assert orc.orthogonality(Qh) <= 1e-6


# ----------------------------------------------------------------------------- tensor-core Gram, 64 < n <= 128
# A = Q^T Q (Alg. 3 step 2) on the tensor cores (gemm_tc.cu): per tile and column an 8-bit
# digit and two FP16 pieces (each entry to 2^-22 of itself), the digit products exact, the
# next products in FP32 over at most eight 16-row steps (2^-21 of at most 2^-7 of the
# leading term), per-tile Kahan sums, FP64 across CTAs; the dropped products are below
# 2^-26.  Bound, entrywise: |A - Q^T Q| <= 2^-19 (|Q|^T |Q|).

@pytest.mark.parametrize("m,n", [(100, 65), (70001, 100), (128 * 300, 128), (9999, 128)])
def test_gram_tensor_core(rc, inputs, m, n):
    g = torch.Generator(device="cpu").manual_seed(1000 + n)
    Qh = torch.randn((m, n), dtype=torch.float64, generator=g).numpy()
    Qh *= 10.0 ** (np.arange(n) / 25.0)[None, :]                 # columns of different scales
    Qh[: m // 3] *= 1e-3                                        # and rows of different scales
    Qh[:, n // 2] = 0.0                                          # one zero column
    Q32 = Qh.astype(np.float32)
    Q = torch.from_numpy(Q32).to(DEV).t().contiguous().t()
    A = host64(rc.rcqr_gram(Q))
    torch.cuda.synchronize()
    Qd = Q32.astype(np.float64)
    Ao = Qd.T @ Qd
    assert np.array_equal(A, A.T)
    assert np.all(np.abs(A - Ao) <= 2.0 ** -19 * (np.abs(Qd).T @ np.abs(Qd)))


# ----------------------------------------------------------------------------- blocked substitution, 64 < n <= 128
# rcqr_trsm for 64 < n <= 128 runs the eight-block tensor-core substitution (trsm_tcw.cu):
# the same FP32 backward and forward bounds as the 64-column kernel above.

@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,cond", [(77, 65, 1e3), (128 * 97, 128, 1e6), (70001, 100, 1e8), (30000, 120, 1e2)])
def test_tc_wide_substitution(rc, inputs, prec, m, n, cond):
    X = inputs.svd_matrix(m, n, cond, 900 + n, dtype=prec, device=DEV)
    Ro = upper_r(n, cond, 190 + n)
    R = torch.from_numpy(Ro).to(DEV).t().contiguous().t()
    Q = rc.rcqr_trsm(X, R)
    torch.cuda.synchronize()
    check_substitution(host64(X), host64(Q), Ro, n, cond)


def test_tc_wide_substitution_permuted_rank_and_in_place(rc, inputs):
    m, n, r = 20000, 128, 83
    X = inputs.svd_matrix(m, n, 1e2, 16, dtype="f32", device=DEV)
    perm_h = np.random.default_rng(2).permutation(n).astype(np.int32)
    perm = torch.from_numpy(perm_h).to(DEV)
    rank = torch.tensor([r], dtype=torch.int64, device=DEV)
    Ro = np.triu(np.random.default_rng(3).standard_normal((n, n))) + 12 * np.eye(n)
    R = torch.from_numpy(Ro).to(DEV).t().contiguous().t()
    Q = host64(rc.rcqr_trsm(X, R, perm=perm, rank=rank))
    torch.cuda.synchronize()
    Xs = host64(X)[:, perm_h[:r]]
    R11 = Ro[:r, :r].astype(np.float32).astype(np.float64)
    check_substitution(Xs, Q[:, :r], R11, r, np.linalg.cond(R11))
    assert np.all(Q[:, r:] == 0)
    # Q in place of X (Alg. 3 step 4 form), bit-equal to the out-of-place call
    Ro2 = upper_r(n, 10.0, 17)
    R2 = torch.from_numpy(Ro2).to(DEV).t().contiguous().t()
    Qs = host64(rc.rcqr_trsm(X.clone(), R2))
    Y = X.clone()
    rc.rcqr_trsm(Y, R2, Q=Y)
    torch.cuda.synchronize()
    assert np.array_equal(host64(Y), Qs)
