"""GPU parity of the strong rank-revealing QR (Gu & Eisenstat swaps with f, after column
pivoting) and of the RRRCholQR variants that use it (Alg. 7 with the RRQR of Sec. 4 / 6.1),
against oracle.linalg.strong_rrqr and oracle.rcqr.rrrcholqr(strong_f=1.5).

Exact: the permutation and the rank (the test inputs keep the chosen swap well ahead of the
next candidate, so both sides pick the same one).  Values: R column-relative <= 1e-10 (FP64
small kernels on the same sketch).  Invariants of the GPU result itself: every swap ratio
rho_ij <= f^2 (recomputed by the oracle from the GPU's R) and Gu-Eisenstat Thm 3.2.
"""
import numpy as np
import pytest
import torch

from oracle import linalg as olin
from oracle import rcqr as orc

pytestmark = pytest.mark.gpu
DEV = "cuda"
F = 1.5


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


def kahan(n, theta=1.2, pert=1e-10):
    c, s = np.cos(theta), np.sin(theta)
    K = np.triu(-c * np.ones((n, n)), 1) + np.eye(n)
    K = np.diag(s ** np.arange(n)) @ K
    return K * (1 - pert * np.arange(n))[None, :]


def to_dev(A):
    return torch.from_numpy(np.asfortranarray(A)).t().contiguous().t().to(DEV)


@pytest.mark.parametrize("n", [16, 24, 40])
def test_srrqr_kahan_matrix(rc, n):
    P = np.vstack([kahan(n), np.zeros((8, n))])
    _, R0, _ = olin.qrcp(P)
    tau = abs(R0[-1, -1]) / olin.spectral_norm(R0) * 1.01          # the truncation rank n - 1
    So, Ro, permo, ro = olin.strong_rrqr(P, tau, F)
    assert ro == n - 1
    R, perm, rank, status = rc.rcqr_srrqr(to_dev(P), tau, F)
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    assert int(rank[0]) == ro
    assert perm.cpu().numpy().tolist() == permo.tolist()
    Rg = host64(R)
    assert colrel(Rg[:ro], Ro[:ro]) <= 1e-10
    # the strong-RRQR property of the GPU's own factor (D = I here), and Gu-Eisenstat Thm 3.2
    _, Rfull = olin.householder_qr(P[:, perm.cpu().numpy()])
    assert np.max(olin.swap_ratios(Rfull, ro)) <= F * F * (1 + 1e-8)
    sv = np.linalg.svd(P, compute_uv=False)
    q = np.sqrt(1 + F * F * ro * (n - ro))
    assert np.linalg.svd(Rfull[:ro, :ro], compute_uv=False).min() >= sv[ro - 1] / q * (1 - 1e-9)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("variant", [4, 5])
def test_factor_strong_rank_revealing(rc, inputs, prec, variant):
    m, n, r, k = 20000, 48, 24, 192
    X = inputs.rank_deficient(m, n, r, 78, noise=1e-12, dtype=prec, device=DEV)
    tau = 1e-10 if prec == "f64" else 1e-5
    seed = 314
    Q, R, perm, rank, status = rc.rcqr_factor(X, k, seed, variant=variant, tau=tau)
    torch.cuda.synchronize()
    Xh = host64(X)
    if variant == 4:
        Qo, So, Ro, permo, ro = orc.rrrcholqr(Xh, k, seed, tau, strong_f=F)
    else:
        Qo, Ro, permo, ro = orc.rrrcholqr2(Xh, k, seed, tau, strong_f=F)
    assert int(status[0]) == 0
    assert int(rank[0]) == ro == r
    # the kept columns are unique; the order of the discarded ones is decided by noise-level
    # norms (near-ties), so only their set is compared
    pg = perm.cpu().numpy()
    assert pg[:r].tolist() == permo[:r].tolist()
    assert sorted(pg[r:].tolist()) == sorted(permo[r:].tolist())
    Qg, Rg = host64(Q), host64(R)
    assert np.all(Qg[:, r:] == 0) and np.all(Rg[r:] == 0)
    uq = 2.0 ** -53 if prec == "f64" else 2.0 ** -24
    D = np.linalg.norm(Xh, axis=0)
    E = (Xh[:, pg] - Qg[:, :r] @ Rg[:r]) / D[pg][None, :]
    assert np.linalg.norm(E) <= 2 * tau + 100 * uq
    # Q R in the original column order against the oracle's
    Yg, Yo = np.zeros_like(Xh), np.zeros_like(Xh)
    Yg[:, pg] = Qg[:, :r] @ Rg[:r]
    Yo[:, permo] = Qo @ Ro
    assert colrel(Yg, Yo) <= max(1e-10, 100 * uq)
    if variant == 5:
        assert orc.orthogonality(Qg[:, :r]) <= max(1e-12, 100 * r * uq)


def test_srrqr_full_rank_equals_qrcp(rc, inputs):
    # a well-conditioned sketch has rank n: no swap, the QRCP result itself
    P = inputs.svd_matrix(256, 32, 1e2, 5, dtype="f64", device=DEV)
    R1, p1, r1, _ = rc.rcqr_srrqr(P, 1e-12, F)
    R2, p2, r2, _ = rc.rcqr_qrcp(P, 1e-12)
    torch.cuda.synchronize()
    assert int(r1[0]) == int(r2[0]) == 32
    assert torch.equal(p1, p2) and torch.equal(R1, R2)
