"""Seeded synthetic inputs shaped like the paper's test matrices (Sec. 6).

This module generates data only; it holds none of the factorization's
arithmetic and is shared by the tests, the benchmark and the oracle checks.
Every matrix is column-major (Fortran order) as the library expects: a torch
tensor X of logical shape (m, n) is stored as the transpose of a contiguous
(n, m) tensor, so ``X.stride() == (1, ld)``.

* ``svd_matrix``   -- X = U diag(sigma) V^T with U (m x n) and V (n x n) the
  orthonormalised factors of seeded Gaussians and sigma log-spaced from 1 to
  1/cond (the first test family of Sec. 6.1 and the runtime family of Sec. 6.3).
* ``rank_deficient`` -- n/2 independent columns, the remaining columns random
  combinations of them plus a tiny Gaussian perturbation (numerical rank r).
* ``integer_matrix`` -- small integers, for sketches that are exact in FP64.
"""
import torch

_DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def colmajor_empty(m, n, dtype, device, ld=None):
    """An (m, n) column-major tensor view with leading dimension ld >= m."""
    ld = m if ld is None else ld
    base = torch.empty((n, ld), dtype=dtype, device=device)
    return base.t()[:m, :]


def to_colmajor(A, dtype=None, ld=None):
    """Copy an (m, n) tensor into column-major storage (optionally with ld > m)."""
    m, n = A.shape
    out = colmajor_empty(m, n, dtype or A.dtype, A.device, ld)
    out.copy_(A)
    return out


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def orthonormal(m, n, seed, device="cpu"):
    """Orthonormal m x n matrix from a seeded standard Gaussian, FP64.

    Small or square matrices: the Q factor of LAPACK's QR on the host.  Tall
    ones (m > 8192, m >= 4n): the orthogonal polar factor of G / sqrt(m) by
    Newton-Schulz iterations U <- U (3 I - U^T U) / 2, plain matrix products on
    the device (the singular values of G / sqrt(m) lie in 1 +- ~sqrt(n/m), well
    inside the iteration's convergence region (0, sqrt 3)).
    """
    G = torch.randn((m, n), dtype=torch.float64, device=device, generator=_gen(seed, device))
    if m <= 8192 or m < 4 * n:
        Q, _ = torch.linalg.qr(G.cpu(), mode="reduced")
        return Q.to(device)
    U = G / (m ** 0.5)
    eye = torch.eye(n, dtype=torch.float64, device=device)
    for _ in range(40):
        A = U.t() @ U
        if float(torch.max(torch.abs(A - eye))) < 1e-15:
            break
        U = U @ (1.5 * eye - 0.5 * A)
    return U


def svd_matrix(m, n, cond, seed, dtype="f64", device="cpu", ld=None, return_factors=False):
    """X = U diag(sigma) V^T, sigma_i = cond^{-(i-1)/(n-1)}, rounded to ``dtype``; column-major."""
    U = orthonormal(m, n, seed, device)
    V = orthonormal(n, n, seed + 7919, device)
    if n > 1:
        expo = torch.arange(n, dtype=torch.float64, device=device) / (n - 1)
        sigma = torch.pow(torch.tensor(float(cond), dtype=torch.float64, device=device), -expo)
    else:
        sigma = torch.ones(1, dtype=torch.float64, device=device)
    X = (U * sigma[None, :]) @ V.t()
    Xs = to_colmajor(X, _DT[dtype], ld)
    if return_factors:
        return Xs, U, sigma, V
    return Xs


def rank_deficient(m, n, r, seed, noise=1e-12, dtype="f32", device="cpu", ld=None):
    """First r columns Gaussian; the other n-r are Gaussian combinations of them plus noise*N(0,1)."""
    g = _gen(seed, device)
    B = torch.randn((m, r), dtype=torch.float64, device=device, generator=g)
    C = torch.randn((r, n - r), dtype=torch.float64, device=device, generator=g) / max(r, 1) ** 0.5
    E = torch.randn((m, n - r), dtype=torch.float64, device=device, generator=g)
    X = torch.cat([B, B @ C + noise * E], dim=1)
    return to_colmajor(X, _DT[dtype], ld)


def integer_matrix(m, n, seed, lo=-128, hi=127, dtype="f64", device="cpu", ld=None):
    """Uniform integers in [lo, hi] (exactly representable in every storage type used)."""
    X = torch.randint(lo, hi + 1, (m, n), generator=_gen(seed, "cpu"), dtype=torch.int64)
    return to_colmajor(X.to(torch.float64).to(device), _DT[dtype], ld)


def gaussian_colmajor(m, n, seed, dtype="f64", device="cpu", ld=None):
    G = torch.randn((m, n), dtype=torch.float64, device=device, generator=_gen(seed, device))
    return to_colmajor(G, _DT[dtype], ld)


def batched_shapes(count, seed, m_lo=16384, m_hi=262144, n_choices=(16, 32, 64, 96)):
    """Seeded (m_i, n_i) pairs: m uniform integer in [m_lo, m_hi], n uniform over n_choices."""
    g = _gen(seed, "cpu")
    ms = torch.randint(m_lo, m_hi + 1, (count,), generator=g).tolist()
    ns = torch.randint(0, len(n_choices), (count,), generator=g).tolist()
    return [(int(mm), int(n_choices[j])) for mm, j in zip(ms, ns)]


def e2_matrix(m, n, dtype="f64", device="cpu", ld=None):
    """The second test matrix of Sec. 6.1: X_ij = sin(10 (x_i + y_j)) / (cos(100 (y_j - x_i)) + 1.1)
    on the uniform unit grid x_i = i / (m - 1), y_j = j / (n - 1), built in FP64 and rounded to
    ``dtype``; column-major.  Its singular values decay rapidly (numerically low rank)."""
    x = torch.arange(m, dtype=torch.float64, device=device) / max(m - 1, 1)
    y = torch.arange(n, dtype=torch.float64, device=device) / max(n - 1, 1)
    X = torch.sin(10 * (x[:, None] + y[None, :])) / (torch.cos(100 * (y[None, :] - x[:, None])) + 1.1)
    return to_colmajor(X, _DT[dtype], ld)
