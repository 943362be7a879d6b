"""GPU parity of the sketch with the SRHT embedding (Sec. 2: sqrt(1/k) S H D, random signs,
Hadamard rows sampled uniformly) against the oracle (oracle.theta.srht_signs,
oracle.rcqr.sketch(dist="srht")).

* Integer X: bit-exact (every partial sum is an integer below 2^53), including row offsets
  that are not multiples of the 128-row Philox block and one beyond 2^32 (the Hadamard
  index is the 64-bit global row).
* Other X: column-wise relative SKETCH_TOL, the tolerance of the Gaussian sketch (the same
  exact digit slices; the +-1 entries only shrink the products).
* Row shards add up to the whole; RCholeskyQR2 driven by it matches the oracle run with the
  same embedding.
"""
import numpy as np
import pytest
import torch

from oracle import rcqr as orc
from oracle import theta as oth

pytestmark = pytest.mark.gpu
DEV = "cuda"
SKETCH_TOL = {"f64": 1e-12, "f32": 1e-11, "bf16": 1e-6}
SRHT = oth.SRHT
U = 2.0 ** -53


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


@pytest.mark.parametrize("prec,off", [("f64", 0), ("f32", 77), ("bf16", 77), ("f32", (1 << 33) + 5)])
def test_srht_sketch_integer_input_is_bit_exact(rc, inputs, prec, off):
    m, n, k = 40021, 19, 64
    X = inputs.integer_matrix(m, n, 6, dtype=prec, device=DEV)
    P = rc.rcqr_sketch(X, k, 0xFACE, row_offset=off, theta=rc.THETA_SRHT)
    torch.cuda.synchronize()
    Po = orc.sketch(host64(X), k, 0xFACE, row_offset=off, dist=SRHT)
    assert np.array_equal(host64(P), Po)


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n,k", [(1000, 1, 8), (20000, 64, 256), (3001, 130, 264)])
def test_srht_sketch_parity(rc, inputs, prec, m, n, k):
    X = inputs.svd_matrix(m, n, 1e6, 41 + m, dtype=prec, device=DEV)
    P = rc.rcqr_sketch(X, k, 0xD00D + n, theta=rc.THETA_SRHT)
    torch.cuda.synchronize()
    Po = orc.sketch(host64(X), k, 0xD00D + n, dist=SRHT)
    assert colrel(host64(P), Po) <= SKETCH_TOL[prec]


def test_srht_sketch_shards_add_up(rc, inputs):
    m, n, k, a = 30000, 16, 64, 12345
    X = inputs.svd_matrix(m, n, 1e3, 5, dtype="f64", device=DEV)
    P = host64(rc.rcqr_sketch(X, k, 43, theta=rc.THETA_SRHT))
    P1 = host64(rc.rcqr_sketch(X[:a], k, 43, row_offset=0, theta=rc.THETA_SRHT))
    P2 = host64(rc.rcqr_sketch(X[a:], k, 43, row_offset=a, theta=rc.THETA_SRHT))
    assert colrel(P1 + P2, P) <= 1e-13


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rcholqr2_with_srht_theta(rc, inputs, prec):
    m, n, k, cond = 20011, 64, 256, 1e6
    X = inputs.svd_matrix(m, n, cond, 1203, dtype=prec, device=DEV)
    Q, R, _, _, status = rc.rcqr_factor(X, k, 78, variant=rc.DIRECT2, theta=rc.THETA_SRHT)
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    Xh = host64(X)
    Qo, Ro, _ = orc.rcholqr2(Xh, k, 78, dist=SRHT)
    Qg, Rg = host64(Q), host64(R)
    ub = U if prec == "f64" else 2.0 ** -24
    assert np.linalg.norm(Qg @ Rg - Xh) / np.linalg.norm(Xh) <= max(1e-12, 10 * n * ub)
    assert orc.orthogonality(Qg) <= (max(1e-12, 100 * n * ub) if prec == "f64" else 1e-6)
    if prec == "f64":
        kap = orc.condition_number(Xh)
        assert colrel(Rg, Ro) <= max(1e-12, 10 * n * U * kap)
