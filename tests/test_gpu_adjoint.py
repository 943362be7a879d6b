"""The hand-written adjoint of RCholeskyQR2 on the GPU.

* FP64, 2048 x 16: the autograd gradient of loss = sum(W1 * Q) + sum(W2 * R)
  against central finite differences of the GPU loss itself (relative 1e-6),
  and against the CPU FP64 oracle adjoint (relative 1e-9).
* FP32 at the size of the differentiable configuration (1,048,576 x 256,
  cond 1e6, k = 1024): against the CPU FP64 adjoint evaluated on the same
  factors Q (the FP32 Q of the forward pass, which differs from X R^{-1} in
  FP64 by up to u cond(R)), R, Qbar, Rbar.  The FP32 rows (u = 2^-24) solve
  x R^T = y after y = qbar + q C, so the check is backward: the residual
  Xbar R^T - Y_oracle, formed in FP64, is within
  10 (n + 2) u (|Qbar| + |Q| |C| + |Xbar| |R^T|) in Frobenius norm -- the
  standard componentwise bounds of a dot product and of a triangular solve
  (Higham, Thm 8.5).  |Xbar| |R^T| is the dominant term: Xbar is large in the
  directions of R's small singular values.  (A forward bound,
  (n + 2) u cond(R) ~ 1.5e-2 here, says little.)
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2210_09953_gb300 import autograd
    return autograd


def host64(t):
    return t.detach().to("cpu", torch.float64).numpy()


def test_adjoint_fp64_finite_differences(ag):
    from paper_2210_09953_gb300 import inputs
    m, n, k, seed = 2048, 16, 64, 0xD1FF
    X = inputs.svd_matrix(m, n, 1e3, 5, dtype="f64", device="cuda")
    W1n, W2n = oadj.loss_weights(m, n, 7)
    W1 = torch.from_numpy(W1n).cuda()
    W2 = torch.from_numpy(W2n).cuda()

    def loss(Xv):
        Q, R = ag.rcholqr2(Xv, k, seed)
        return torch.sum(W1 * Q) + torch.sum(W2 * R)

    Xg = X.clone().requires_grad_(True)
    loss(Xg).backward()
    G = host64(Xg.grad)
    rng = np.random.default_rng(1)
    with torch.no_grad():
        for _ in range(3):
            D = rng.standard_normal((m, n))
            h = 1e-6 * float(torch.linalg.norm(X)) / np.linalg.norm(D)
            Dt = inputs.to_colmajor(torch.from_numpy(D).cuda())
            fd = (float(loss(X + h * Dt)) - float(loss(X - h * Dt))) / (2 * h)
            assert abs(np.sum(G * D) - fd) <= 1e-6 * max(1.0, abs(fd))
    # the CPU FP64 adjoint on the same factors
    _, R = ag.rcholqr2(X, k, seed)
    Go = oadj.qr_adjoint(host64(X), host64(R), W1n, np.triu(W2n))
    assert np.max(np.abs(G - Go)) <= 1e-9 * np.max(np.abs(Go))


def test_adjoint_fp32_full_size_against_cpu_fp64(ag):
    from paper_2210_09953_gb300 import inputs
    m, n, k, seed = 1 << 20, 256, 1024, 0xAD30
    X = inputs.svd_matrix(m, n, 1e6, 1005, dtype="f32", device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(41)
    W1 = torch.randn((m, n), dtype=torch.float32, device="cuda", generator=g)
    W2 = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    Xg = X.clone().requires_grad_(True)
    Q, R = ag.rcholqr2(Xg, k, seed)
    (torch.sum(W1 * Q) + torch.sum(W2 * R)).backward()
    torch.cuda.synchronize()
    G = host64(Xg.grad)
    Rh = host64(R)
    Qh, W1h, W2h = host64(Q), host64(W1), np.triu(host64(W2))
    Go = oadj.qr_adjoint_factors(Qh, Rh, W1h, W2h)
    u = 2.0 ** -24
    Yg, Yo = G @ Rh.T, Go @ Rh.T
    C = oadj.copyltu(Rh @ W2h.T - W1h.T @ Qh)
    scale = (np.linalg.norm(W1h) + np.linalg.norm(np.abs(Qh) @ np.abs(C))
             + np.linalg.norm(np.abs(G) @ np.abs(Rh).T))
    assert np.linalg.norm(Yg - Yo) <= 10 * (n + 2) * u * scale
    assert np.all(np.isfinite(G))
