"""GPU parity of column-oriented RCholeskyQR (Alg. 4) and its randomized Gram-Schmidt form (the
remark after Alg. 4) against oracle.rcqr.col_rcholqr.

Tolerances: FP64 X, per column relative max(1e-12, 10 n u kappa) for R, S and Q (the forward
error of the method; blocks are independent least-squares + QR steps in FP64 on both sides).
FP32 X: ||X - QR|| <= 10 n u32 ||X||, R as the mixed RCholeskyQR tests (the sketch is exact
to 1e-11, the small steps are FP64).  The block-by-block call (rcqr_colblock_step) on blocks
generated from the previous Q (the Krylov use of Sec. 3.2 and Sec. 6.2) matches the oracle run afterwards
on the generated X.
"""
import math

import numpy as np
import pytest
import torch

from oracle import rcqr as orc

pytestmark = pytest.mark.gpu
DEV = "cuda"
U = 2.0 ** -53
U32 = 2.0 ** -24


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


@pytest.mark.parametrize("rgs", [False, True])
@pytest.mark.parametrize("m,n,b,k,cond", [(6007, 24, 8, 96, 1e6), (20011, 64, 16, 256, 1e4), (3001, 40, 40, 128, 1e8),
                                          (5003, 50, 16, 200, 1e3)])
def test_colwise_fp64_parity(rc, inputs, rgs, m, n, b, k, cond):
    X = inputs.svd_matrix(m, n, cond, 1601 + n, dtype="f64", device=DEV)
    Q, S, R, status = rc.rcqr_factor_colwise(X, k, 0xC01, b, rgs=rgs)
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    Xh = host64(X)
    Qo, So, Ro = orc.col_rcholqr(Xh, b, k, 0xC01, rgs=rgs)
    kap = orc.condition_number(Xh)
    tol = max(1e-12, 10 * n * U * kap)
    Rg = host64(R)
    assert np.array_equal(Rg, np.triu(Rg)) and np.all(np.diag(Rg) > 0)
    assert colrel(Rg, Ro) <= tol
    assert colrel(host64(S), So) <= tol
    assert colrel(host64(Q), Qo) <= tol
    assert np.linalg.norm(host64(Q) @ Rg - Xh) / np.linalg.norm(Xh) <= 1e-12


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_colwise_mixed_precision(rc, inputs, prec):
    m, n, b, k, cond = 20011, 64, 16, 256, 1e4
    X = inputs.svd_matrix(m, n, cond, 1701, dtype=prec, device=DEV)
    Q, S, R, status = rc.rcqr_factor_colwise(X, k, 0xC02, b)
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    Xh = host64(X)
    _, _, Ro = orc.col_rcholqr(Xh, b, k, 0xC02)
    kap = orc.condition_number(Xh)
    Qg, Rg = host64(Q), host64(R)
    assert np.linalg.norm(Qg @ Rg - Xh) / np.linalg.norm(Xh) <= 10 * n * U32
    tol_r = max(1e-12, 10 * n * U * kap) + 10 * math.sqrt(n) * kap * (1e-11 if prec == "f32" else 1e-6)
    assert colrel(Rg, Ro) <= tol_r + 10 * n * U32 * kap


def test_colblock_steps_on_generated_blocks(rc, inputs):
    # a Krylov-like build: X_1 given, X_{i+1} = D Q_i (D diagonal), one rcqr_colblock_step per block
    m, n, b, k = 8009, 32, 8, 128
    d = torch.linspace(1.0, 3.0, m, dtype=torch.float64, device=DEV)
    Q = rc.colmajor(m, n, torch.float64, DEV)
    S = rc.colmajor(k, n, torch.float64, DEV)
    R = torch.zeros((n, n), dtype=torch.float64, device=DEV).t()
    Xfull = rc.colmajor(m, n, torch.float64, DEV)
    Xfull[:, :b] = inputs.svd_matrix(m, b, 10.0, 1801, dtype="f64", device=DEV)
    for i0 in range(0, n, b):
        if i0 > 0:
            Xfull[:, i0:i0 + b] = d[:, None] * Q[:, i0 - b:i0]
        Xi = Xfull[:, i0:i0 + b]
        st = rc.rcqr_colblock_step(Xi, k, 0xC03, i0, Q, S, R)
        torch.cuda.synchronize()
        assert int(st[0]) == 0
    Xh = host64(Xfull)
    Qo, So, Ro = orc.col_rcholqr(Xh, b, k, 0xC03)
    kap = orc.condition_number(Xh)
    tol = max(1e-12, 10 * n * U * kap)
    assert colrel(host64(R), Ro) <= tol
    assert colrel(host64(Q), Qo) <= tol
