"""Pins for the oracle's reverse-mode derivative of RCholeskyQR2."""
import numpy as np
import pytest
import torch

from oracle import adjoint, rcqr


def svd_matrix(m, n, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (U * np.logspace(0, -np.log10(cond), n)[None, :]) @ V.T


def loss(X, k, seed, W1, W2):
    Q, R, _ = rcqr.rcholqr2(X, k, seed)
    return float(np.sum(W1 * Q) + np.sum(W2 * R))


@pytest.mark.parametrize("cond", [1.0 + 1e-9, 1e3])
def test_adjoint_matches_central_differences(cond):
    m, n, k, seed = 300, 6, 48, 5
    X = svd_matrix(m, n, cond, 1)
    W1, W2 = adjoint.loss_weights(m, n, 2)
    Q, R, _ = rcqr.rcholqr2(X, k, seed)
    G = adjoint.qr_adjoint(X, R, W1, np.triu(W2))
    rng = np.random.default_rng(3)
    for _ in range(3):
        D = rng.standard_normal((m, n))
        h = 1e-6 * np.linalg.norm(X) / np.linalg.norm(D)
        fd = (loss(X + h * D, k, seed, W1, W2) - loss(X - h * D, k, seed, W1, W2)) / (2 * h)
        assert abs(np.sum(G * D) - fd) <= 1e-6 * max(1.0, abs(fd))


def test_adjoint_matches_torch_qr_derivative():
    # torch's derivative of its (LAPACK) thin QR, signs fixed to diag(R) > 0 -- an independent routine
    m, n = 200, 5
    X = svd_matrix(m, n, 1e2, 4)
    W1, W2 = adjoint.loss_weights(m, n, 6)
    Xt = torch.tensor(X, requires_grad=True)
    Qt, Rt = torch.linalg.qr(Xt, mode="reduced")
    s = torch.sign(torch.diagonal(Rt)).detach()
    Qt, Rt = Qt * s[None, :], Rt * s[:, None]
    (torch.sum(torch.tensor(W1) * Qt) + torch.sum(torch.tensor(W2) * Rt)).backward()
    _, R, _ = rcqr.rcholqr2(X, 40, 9)
    G = adjoint.qr_adjoint(X, R, W1, np.triu(W2))
    assert np.max(np.abs(G - Xt.grad.numpy())) <= 1e-9 * np.max(np.abs(G))


def test_planted_mistake_in_adjoint_is_caught(monkeypatch):
    m, n = 200, 5
    X = svd_matrix(m, n, 10.0, 8)
    W1, W2 = adjoint.loss_weights(m, n, 1)
    _, R, _ = rcqr.rcholqr2(X, 40, 9)
    good = adjoint.qr_adjoint(X, R, W1, np.triu(W2))
    monkeypatch.setattr(adjoint, "copyltu", lambda M: np.triu(M) + np.triu(M, 1).T)   # wrong triangle
    bad = adjoint.qr_adjoint(X, R, W1, np.triu(W2))
    assert np.max(np.abs(bad - good)) > 1e-3 * np.max(np.abs(good))


def test_back_substitution_closed_form():
    R = np.array([[2.0, 1.0], [0.0, 4.0]])
    B = np.array([[5.0], [8.0]])
    assert np.allclose(adjoint.back_substitution(R, B), [[1.5], [2.0]], rtol=0, atol=1e-15)
