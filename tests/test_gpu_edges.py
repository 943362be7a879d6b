"""GPU parity at the edges of the method and of the number formats, against the CPU oracle.

* Sketch (Alg. 2 step 1) of X whose rows span 1e-15 .. 1e15 within every column (the
  row-scaled test family of Sec. 6.1), and of X with an all-zero column and columns of
  subnormal numbers only.  Tolerance for the scaled rows, column-wise relative: every X
  entry more than a few binades below its 2048-row block's largest one (1024 for FP64 X)
  is rounded once, at 2^-b of that largest entry (b = 36 FP32, 22 BF16, 55 FP64: the
  exact digit slices and the rounded last slice), so
  ||dP_j|| <= (1 + eps) sqrt(rows per block) 2^-b ||X_j||; the tests use 4 sqrt(BR) 2^-b.
* Alg. 2 on the mixed path (FP32 / BF16 X, FP32 substitution) at cond 1e8 and 1e12,
  where the FP64 forward-error checks of test_gpu_parity are vacuous: cond(Q) and
  ||S - Theta Q||_F within 10x of the oracle run in the same multi-precision model
  (oracle.rcqr.rcholqr_f32: sketch and QR in FP64, substitution in float32), and
  sigma(Q) inside the Thm. 5.2 interval (with the exact eps of the drawn Theta and u =
  2^-24) wherever that interval is not vacuous.
* Alg. 3 on the mixed path: ||Q^T Q - I|| <= 1e-6 at every condition number tested, for
  n = 64, 100 and 128 (the second pass by the tensor-core product with R'^{-1}).
* Alg. 5 with FP32 / BF16 X (the sketch exact to SKETCH_TOL, the rest FP64): Z and R
  against the FP64 oracle on the stored X, and Thm. 5.4 (rmain1) for Z against L Q.
* A zero column of X: R_jj = 0, Q's column j and the Gram of Alg. 3 step 2 are NaN, so
  the Cholesky pivot j is not positive: rcqr_factor must report {RCQR_ENOTSPD, j}, as
  the oracle's cholesky raises NotSPD(j).  (An exact duplicate of a column does not
  force this: rounding in the Householder QR leaves R_jj ~ u ||x_j|| instead of 0.)
* A bounded wait of the tensor-core sketch that runs out (a limit of one poll):
  dev_status = RCQR_ETIMEOUT, NaN results, and the next call with the default limit
  is correct again (the context stays usable).
"""
import math

import numpy as np
import pytest
import torch

from oracle import linalg as olin
from oracle import rcqr as orc
from oracle import theta as oth

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
U32 = 2.0 ** -24
SKETCH_TOL = {"f64": 1e-12, "f32": 1e-11, "bf16": 1e-6}
DEV = "cuda"
DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


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


def to_dev(Xh, prec):
    """Column-major device copy of a host float64 matrix, rounded to the storage type."""
    t = torch.from_numpy(np.asfortranarray(Xh)).to(DT[prec])
    return t.t().contiguous().t().to(DEV)


# ----------------------------------------------------------------------------- sketch edges

@pytest.mark.parametrize("prec,bits,br", [("f64", 55, 1024), ("f32", 36, 2048), ("bf16", 22, 2048)])
def test_sketch_rows_spanning_thirty_orders(rc, inputs, prec, bits, br):
    m, n, k = 40000, 12, 96
    X = host64(inputs.svd_matrix(m, n, 1e4, 61, dtype="f64", device="cpu"))
    scale = 10.0 ** np.random.default_rng(62).uniform(-15, 15, m)
    Xd = to_dev(X * scale[:, None], prec)
    P = rc.rcqr_sketch(Xd, k, 0x5CA1E)
    torch.cuda.synchronize()
    Po = orc.sketch(host64(Xd), k, 0x5CA1E)
    tol = max(SKETCH_TOL[prec], 4 * math.sqrt(br) * 2.0 ** -bits)
    assert colrel(host64(P), Po) <= tol


@pytest.mark.parametrize("prec,tiny", [("f64", 1e-309), ("f32", 1e-40), ("bf16", 1e-39)])
def test_sketch_zero_and_subnormal_columns(rc, inputs, prec, tiny):
    m, n, k = 9000, 6, 48
    rng = np.random.default_rng(7)
    X = host64(inputs.svd_matrix(m, n, 1e2, 63, dtype="f64", device="cpu"))
    X[:, 1] = 0.0                                         # all-zero column
    X[:, 2] = tiny * rng.uniform(-1, 1, m)                # subnormal numbers only
    X[: m // 2, 4] = tiny * rng.uniform(-1, 1, m // 2)    # subnormal rows above normal ones
    Xd = to_dev(X, prec)
    Xs = host64(Xd)
    finfo = {"f64": np.finfo(np.float64).tiny, "f32": float(np.finfo(np.float32).tiny),
             "bf16": float(np.finfo(np.float32).tiny)}[prec]
    assert np.all(np.abs(Xs[:, 2]) < finfo) and np.any(Xs[:, 2] != 0)   # really subnormal, not flushed
    cn = torch.empty(n, dtype=torch.float64, device=DEV)
    P = rc.rcqr_sketch(Xd, k, 0xD0D0, colnorm2=cn)
    torch.cuda.synchronize()
    Po = orc.sketch(Xs, k, 0xD0D0)
    Pg = host64(P)
    assert np.all(Pg[:, 1] == 0.0)
    assert colrel(Pg, Po) <= SKETCH_TOL[prec]
    ref = np.sum(Xs * Xs, axis=0)
    normal = ref > 1e-290
    assert np.all(np.abs(host64(cn)[normal] - ref[normal]) <= 1e-13 * ref[normal])
    assert host64(cn)[1] == 0.0


# ----------------------------------------------------------------------------- mixed Alg. 2 / 3

@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("cond", [1e8, 1e12])
def test_mixed_rcholqr_conditioning_against_f32_oracle(rc, inputs, prec, cond):
    m, n, k = 20011, 64, 256
    X = inputs.svd_matrix(m, n, cond, 1301, dtype=prec, device=DEV)
    seed = 0x5EED0000 + 7
    Q, R, _, rank, status = rc.rcqr_factor(X, k, seed, variant=rc.DIRECT)
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    Xh = host64(X)
    Qo, So, Ro = orc.rcholqr_f32(Xh, k, seed)
    Qg = host64(Q)
    Qo = Qo.astype(np.float64)
    cg, co = orc.condition_number(Qg), orc.condition_number(Qo)
    assert cg <= 10 * co
    dsg = np.linalg.norm(So - orc.sketch(Qg, k, seed))
    dso = np.linalg.norm(So - orc.sketch(Qo, k, seed))
    assert dsg <= 10 * dso + 1e-12
    # Thm. 5.2 (main2) with the exact eps of this Theta on range(X), u = 2^-24 and the stored
    # condition number, where the interval says something
    kap = orc.condition_number(Xh)
    slack = 4 * U32 * n ** 1.5 * kap
    if slack < 0.5:
        Uf, _ = np.linalg.qr(Xh)
        eps = orc.embedding_epsilon(oth.theta(seed, k, 0, m), Uf)
        s = np.linalg.svd(Qg, compute_uv=False)
        assert s.min() >= (1 + eps) ** -0.5 - slack
        if eps < 1:
            assert s.max() <= (1 - eps) ** -0.5 + slack
    # backward error at any condition number: the float32 substitution's row-wise bound
    # |X - Q R| <= (n + 3) u |Q||R| (Higham Thm. 8.5, R rounded to float), doubled for the
    # rounding of the comparison itself
    Rg = host64(R)
    assert np.all(np.abs(Xh - Qg @ Rg) <= 2 * (n + 3) * U32 * (np.abs(Qg) @ np.abs(Rg)) + 1e-300)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("cond", [1e4, 1e8, 1e12])
@pytest.mark.parametrize("n", [64, 100, 128])
def test_mixed_rcholqr2_orthogonality(rc, inputs, prec, cond, n):
    m, k = 30011, 4 * n
    X = inputs.svd_matrix(m, n, cond, 1401, dtype=prec, device=DEV)
    Q, R, _, _, status = rc.rcqr_factor(X, k, 0x5EED0002, variant=rc.DIRECT2)
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    Qg, Xh = host64(Q), host64(X)
    assert orc.orthogonality(Qg) <= 1e-6
    assert np.linalg.norm(Qg @ host64(R) - Xh) / np.linalg.norm(Xh) <= 10 * n * U32


# ----------------------------------------------------------------------------- reduced, mixed storage

@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("use_L", [False, True])
def test_reduced_mixed_storage(rc, inputs, prec, use_L):
    m, n, k, l = 30007, 16, 64, 5
    X = inputs.svd_matrix(m, n, 1e6, 55, dtype=prec, device=DEV)
    L = inputs.gaussian_colmajor(l, m, 8, device=DEV) if use_L else None
    Z, S, R, status = rc.rcqr_reduced(X, k, 3, L=L)
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    Xh = host64(X)
    Lh = host64(L) if use_L else None
    Zo, So, Ro = orc.reduced(Xh, k, 3, L=Lh)
    kap = orc.condition_number(Xh)
    tol = max(1e-12, 10 * n * U * kap) + 10 * math.sqrt(n) * kap * SKETCH_TOL[prec]
    assert colrel(host64(R), Ro) <= tol
    assert colrel(host64(S), So) <= tol
    Zg = host64(Z)
    if not use_L:
        assert np.array_equal(Zg, host64(S))        # Z = P R^{-1} = S: the same substitution
    # Thm. 5.4 (rmain1): ||Z_i - L_i Q|| <= 3.5 u n^{3/2} kappa ||L_i|| with Q = X R^{-1} (u = 2^-53:
    # every step after the sketch is FP64) plus the sketch's own error carried through R^{-1}
    Rg = host64(R)
    Qx = olin.forward_substitution(Xh, Rg)
    Lm = Lh if use_L else oth.theta(3, k, 0, m)
    bound = (3.5 * U * n ** 1.5 * kap + 10 * math.sqrt(n) * kap * SKETCH_TOL[prec]) * np.linalg.norm(Lm, axis=1)
    assert np.all(np.linalg.norm(Zg - Lm @ Qx, axis=1) <= bound + 1e-300)


# ----------------------------------------------------------------------------- device status

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_factor_zero_column_reports_enotspd(rc, inputs, prec):
    m, n, j = 5000, 8, 3
    X = host64(inputs.svd_matrix(m, n, 1e2, 71, dtype="f64", device="cpu"))
    X[:, j] = 0.0
    Xd = to_dev(X, prec)
    Q, R, _, _, status = rc.rcqr_factor(Xd, 32, 11, variant=rc.DIRECT2)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [-2, j]
    with np.errstate(all="ignore"), pytest.raises(olin.NotSPD) as info:
        orc.rcholqr2(host64(Xd), 32, 11)
    assert info.value.j == j


def test_sketch_wait_that_runs_out_reports_etimeout(rc, inputs):
    m, n, k = 100000, 64, 256
    X = inputs.svd_matrix(m, n, 1e3, 81, dtype="f32", device=DEV)
    prev = rc.rcqr_set_wait_polls(1)
    try:
        Q, R, _, _, status = rc.rcqr_factor(X, k, 5, variant=rc.DIRECT)
        torch.cuda.synchronize()
    finally:
        rc.rcqr_set_wait_polls(prev)
    assert status.cpu().tolist() == [-5, -1]
    assert bool(torch.isnan(R).any())
    # the default limit again: the same call is correct, the context is intact
    Q, R, _, _, status = rc.rcqr_factor(X, k, 5, variant=rc.DIRECT)
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    _, _, Ro = orc.rcholqr(host64(X), k, 5)
    assert colrel(host64(R), Ro) <= 1e-6
