"""Parity and properties at the full sizes of the workload configurations.

* 4,194,304 x 64, cond 1e8, k = 256 (the benchmark's launch configuration):
  FP32-stored X on the mixed path and FP64 X on the FP64 path, RCholeskyQR2.
  The FP64 path is compared with the CPU oracle run on the whole matrix
  (R column-wise, sampled rows of Q).  The mixed path is checked by what holds
  at any condition number: ||Q^T Q - I|| <= 1e-6 (the stated target),
  ||X - QR|| / ||X|| <= 10 n u32, and sampled rows of the sketch against the
  oracle.  cond 1e4 and 1e12 are checked by the same properties.
* 16,777,216 x 128, k = 512, FP32 and BF16 storage, cond 1e4 and 1e8: the same
  properties and sampled sketch rows.
* 512 rank-deficient FP32 problems, m uniform in [16384, 262144], n in
  {16, 32, 64, 96}, rank n/2, k = 4n, tau = 1e-5, batched RR and RR2: every
  problem's status, rank and residual; the oracle on a sample of problems.

Sampled sketch rows are compared entrywise against the oracle's rows with the
bound |dP_ij| <= tol ||X_j||_2 (Theta is an isometry on range(X), so ||P_j|| is
of the order of ||X_j||); tol is the sketch tolerance of the parity tests.
Norms over long matrices are accumulated on the device in FP64 chunks.
"""
import math

import numpy as np
import pytest
import torch

from oracle import rcqr as orc

pytestmark = pytest.mark.gpu

U64, U32 = 2.0 ** -53, 2.0 ** -24
SKETCH_TOL = {"f64": 1e-12, "f32": 1e-11, "bf16": 1e-6}
CHUNK = 1 << 21


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2210_09953_gb300 import _binding
    return _binding


def host64(t):
    return t.detach().to("cpu", torch.float64).numpy()


def gram64(Q):
    n = Q.shape[1]
    G = torch.zeros((n, n), dtype=torch.float64, device=Q.device)
    for c in range(0, Q.shape[0], CHUNK):
        q = Q[c:c + CHUNK].double()
        G += q.T @ q
    return G


def orthogonality(Q):
    G = gram64(Q).cpu()
    return float(torch.linalg.matrix_norm(G - torch.eye(G.shape[0], dtype=G.dtype), ord=2))


def residual(X, Q, R):
    num = den = 0.0
    for c in range(0, X.shape[0], CHUNK):
        x = X[c:c + CHUNK].double()
        d = x - Q[c:c + CHUNK].double() @ R
        num += float((d * d).sum())
        den += float((x * x).sum())
    return math.sqrt(num / den)


def col_norms(X):
    s = torch.zeros(X.shape[1], dtype=torch.float64, device=X.device)
    for c in range(0, X.shape[0], CHUNK):
        s += (X[c:c + CHUNK].double() ** 2).sum(dim=0)
    return s.sqrt().cpu().numpy()


def check_sketch_rows(rc, X, k, seed, prec, rows):
    P = rc.rcqr_sketch(X, k, seed)
    torch.cuda.synchronize()
    Xh = X.detach().cpu().float().numpy() if X.dtype != torch.float64 else X.detach().cpu().numpy()
    Po = orc.sketch_rows(Xh, k, seed, rows)
    Pg = host64(P)[rows]
    bound = SKETCH_TOL[prec] * col_norms(X)[None, :]
    assert np.all(np.abs(Pg - Po) <= bound)


def check_factor_properties(X, Q, R, status, rank, n, u_res, orth_tol):
    assert int(status[0]) == 0 and int(rank[0]) == n
    Rh = host64(R)
    assert np.all(np.tril(Rh, -1) == 0) and np.all(np.diag(Rh) > 0)
    assert orthogonality(Q) <= orth_tol
    assert residual(X, Q, R) <= 10 * n * u_res


# ----------------------------------------------------------------------------- 4M x 64

@pytest.mark.parametrize("cond", [1e8, 1e4, 1e12])
def test_benchmark_workload_mixed_path(rc, cond):
    from paper_2210_09953_gb300 import inputs
    m, n, k, seed = 4194304, 64, 256, 0x5EED0002
    X = inputs.svd_matrix(m, n, cond, 1002, dtype="f32", device="cuda")
    ws = torch.empty(rc.rcqr_workspace_size(m, n, k, rc.DIRECT2, rc.F32) + 256, dtype=torch.uint8, device="cuda")
    Q, R, _, rank, status = rc.rcqr_factor(X, k, seed, variant=rc.DIRECT2, workspace=ws)
    torch.cuda.synchronize()
    check_factor_properties(X, Q, R, status, rank, n, U32, 1e-6)
    if cond == 1e8:
        check_sketch_rows(rc, X, k, seed, "f32", [0, 97, k - 1])


def test_benchmark_workload_fp64_path_against_full_oracle(rc):
    from paper_2210_09953_gb300 import inputs
    m, n, k, seed = 4194304, 64, 256, 0x5EED0002
    X = inputs.svd_matrix(m, n, 1e8, 1002, dtype="f64", device="cuda")
    Q, R, _, rank, status = rc.rcqr_factor(X, k, seed, variant=rc.DIRECT2)
    torch.cuda.synchronize()
    check_factor_properties(X, Q, R, status, rank, n, U64, 100 * n * U64)
    Xh = host64(X)
    Qo, Ro, _ = orc.rcholqr2(Xh, k, seed)
    kap = np.linalg.cond(Ro)
    tol = max(1e-12, 10 * n * U64 * kap)
    Rg = host64(R)
    assert np.max(np.linalg.norm(Rg - Ro, axis=0) / np.linalg.norm(Ro, axis=0)) <= tol
    rows = np.random.default_rng(5).choice(m, 64, replace=False)
    Qs = host64(Q[torch.from_numpy(rows).cuda()])
    assert np.max(np.abs(Qs - Qo[rows])) <= tol * np.max(np.abs(Qo))


# ----------------------------------------------------------------------------- 16M x 128

@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("cond", [1e4, 1e8])
def test_mixed_precision_16M_by_128(rc, prec, cond):
    from paper_2210_09953_gb300 import inputs
    m, n, k, seed = 16777216, 128, 512, 0x5EED0003
    X = inputs.svd_matrix(m, n, cond, 1003, dtype=prec, device="cuda")
    Q, R, _, rank, status = rc.rcqr_factor(X, k, seed, variant=rc.DIRECT2)
    torch.cuda.synchronize()
    # BF16 values are exact in FP32, so Q R reproduces X to the FP32 working precision
    check_factor_properties(X, Q, R, status, rank, n, U32, 1e-6)
    if cond == 1e8:
        check_sketch_rows(rc, X, k, seed, prec, [0, k - 1])
    del Q, R, X
    torch.cuda.empty_cache()


# ----------------------------------------------------------------------------- 512 batched

@pytest.mark.parametrize("variant", [2, 3])
def test_batched_512_rank_deficient(rc, variant):
    from paper_2210_09953_gb300 import inputs
    shapes = inputs.batched_shapes(512, 1004)
    Xs = [inputs.rank_deficient(mm, nn, nn // 2, 4000 + i, noise=1e-12, dtype="f32", device="cuda")
          for i, (mm, nn) in enumerate(shapes)]
    ks = [4 * nn for _, nn in shapes]
    tau, seed = 1e-5, 0x5EED0004
    b = rc.rcqr_factor_batched(Xs, ks, seed, variant=variant, tau=tau)
    torch.cuda.synchronize()
    assert np.all(b.status.cpu().numpy()[:, 0] == 0)
    for i, X in enumerate(Xs):
        n = X.shape[1]
        r = int(b.ranks[i][0])
        assert r == n // 2
        perm = b.perms[i].long()
        D = X.double().norm(dim=0)[perm]
        E = (X.double()[:, perm] - b.Qs[i][:, :r].double() @ b.Rs[i][:r]) / D[None, :]
        assert float(E.norm()) <= 2 * tau + 1e-4
        if variant == 3:
            assert orthogonality(b.Qs[i][:, :r]) <= 100 * r * U32
    for i in (0, 101, 257, 511):
        Xh = host64(Xs[i])
        if variant == 2:
            _, _, _, permo, ro = orc.rrrcholqr(Xh, ks[i], seed, tau, stream=i)
        else:
            _, _, permo, ro = orc.rrrcholqr2(Xh, ks[i], seed, tau, stream=i)
        assert int(b.ranks[i][0]) == ro
        assert b.perms[i].cpu().numpy().tolist() == permo.tolist()
