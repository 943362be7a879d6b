"""Pins for the oracle's Philox generator and Theta realisation (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import philox, theta


def _kat_rows(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            vals = [int(x, 16) for x in line.split()]
            rows.append((vals[:4], vals[4:6], vals[6:]))
    return rows


def test_philox_known_answers(golden_dir):
    rows = _kat_rows(golden_dir)
    assert len(rows) == 3
    for ctr, key, expect in rows:
        out = philox.philox4x32_10(*ctr, *key)
        assert [int(w) for w in out] == expect


def test_philox_vectorised_matches_scalar_calls():
    c0 = np.arange(50, dtype=np.uint64) * np.uint64(2654435761)
    out = philox.philox4x32_10(c0, 3, 7, 11, 0xDEADBEEF, 0x12345678)
    for j in (0, 17, 49):
        single = philox.philox4x32_10(int(c0[j]) & 0xFFFFFFFF, 3, 7, 11, 0xDEADBEEF, 0x12345678)
        assert [int(w[j]) for w in out] == [int(w) for w in single]


def test_table_is_the_scaled_normal_quantile_grid():
    T = theta.quantile_table()
    assert T.shape == (256,)
    assert np.all(T == np.round(T))
    assert T.max() == 127 and T.min() == -127
    assert np.all(np.diff(T) >= 0)                      # monotone (inverse CDF)
    assert np.all(T[::-1] == -T)                        # antisymmetric: Phi^{-1}(1-p) = -Phi^{-1}(p)
    # Each level is the nearest integer to 44*Phi^{-1}(p_t): check with the normal CDF via math.erfc
    # (an independent routine): Phi((T-1/2)/44) <= p_t <= Phi((T+1/2)/44).
    Phi = lambda x: 0.5 * math.erfc(-x / math.sqrt(2.0))
    for t in range(256):
        p = (t + 0.5) / 256
        assert Phi((T[t] - 0.5) / 44.0) <= p <= Phi((T[t] + 0.5) / 44.0)


def test_scale_gives_unit_second_moment():
    T = theta.quantile_table()
    v = theta.table_variance()
    assert v == float(np.sum(T.astype(np.int64) ** 2)) / 256     # exact integer sum
    for k in (1, 128, 256, 1000):
        c = theta.theta_scale(k)
        assert abs(k * c * c * v - 1.0) < 4e-16                  # E[Theta^T Theta] = I
    assert abs(v / 44.0 ** 2 - 1.0) < 0.01                       # close to N(0,1) scaled by 44


def test_bytes_mapping_and_offsets():
    B = theta.theta_bytes(99, 5, 0, 100)
    # a window with a row offset is the same slice of the full stream
    assert np.array_equal(theta.theta_bytes(99, 5, 37, 40), B[:, 37:77])
    # stream and seed change the bytes
    assert not np.array_equal(theta.theta_bytes(99, 5, 0, 100, stream=1), B)
    assert not np.array_equal(theta.theta_bytes(100, 5, 0, 100), B)
    # entry (i, r) is byte r%16 of the Philox block floor(r/16) for row i
    i, r = 3, 53
    w = philox.philox4x32_10(r // 16, 0, i, 0, 99, 0)
    assert B[i, r] == (int(w[(r % 16) // 4]) >> (8 * (r % 4))) & 0xFF
    # 64-bit seed and row index split into two 32-bit words
    seed = (5 << 32) | 9
    r = (3 << 36) + 21
    w = philox.philox4x32_10((r // 16) & 0xFFFFFFFF, (r // 16) >> 32, 2, 0, 9, 5)
    assert theta.theta_bytes(seed, 3, r, 1)[2, 0] == (int(w[(r % 16) // 4]) >> (8 * (r % 4))) & 0xFF


def test_bytes_are_uniform_and_levels_centred():
    B = theta.theta_bytes(2024, 64, 0, 4096)
    counts = np.bincount(B.ravel(), minlength=256)
    expect = B.size / 256
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    assert chi2 < 400                                   # 255 dof: mean 255, sd ~22.6
    G = theta.quantile_table()[B]
    assert abs(G.mean()) < 4 * 44 / math.sqrt(B.size)
    # unit second moment of Theta columns on average: E||Theta e_r||^2 = 1
    Th = theta.theta_scale(64) * G
    col2 = np.sum(Th * Th, axis=0)
    assert abs(col2.mean() - 1.0) < 0.02


@pytest.mark.parametrize("k,n", [(128, 8), (256, 16)])
def test_theta_is_a_subspace_embedding(k, n):
    # Cor. 2.2 / Def. 2.1: Theta U has singular values in [sqrt(1-eps), sqrt(1+eps)] with eps < 1
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((2048, n)))
    Th = theta.theta(7, k, 0, 2048)
    s = np.linalg.svd(Th @ U, compute_uv=False)
    # Gaussian-like OSE: singular values near 1 +- sqrt(n/k)
    assert s.max() < 1 + 2 * math.sqrt(n / k) and s.min() > 1 - 2 * math.sqrt(n / k)


def test_rademacher_signs_follow_the_bit_definition():
    # an independent per-entry recomputation: one scalar Philox call per entry, bit picked with
    # Python integers (entry (i, r): bit r mod 128 of the call at counter (r // 128, i))
    from oracle.philox import philox4x32_10
    seed, k, off, m, stream = 0x1234567890ABCDEF, 5, 77, 300, 3
    S = theta.rademacher_signs(seed, k, off, m, stream)
    for i in (0, 4):
        for r in (off, off + 50, off + 51, off + 299):
            q = r // 128
            w = philox4x32_10(np.uint64(q & 0xFFFFFFFF), np.uint64(q >> 32), np.uint64(i), np.uint64(stream),
                              seed & 0xFFFFFFFF, seed >> 32)
            b = r % 128
            bit = (int(w[b // 32]) >> (b % 32)) & 1
            assert S[i, r - off] == 1.0 - 2.0 * bit
    # rows= selects rows, offsets shift columns consistently
    assert np.array_equal(theta.rademacher_signs(seed, k, off, m, stream, rows=[4, 1]), S[[4, 1]])
    assert np.array_equal(theta.rademacher_signs(seed, k, off + 10, 20, stream), S[:, 10:30])


def test_rademacher_theta_unit_columns_and_balance():
    Th = theta.dense(99, 64, 0, 4096, dist=theta.RADEMACHER)
    assert np.allclose(np.sum(Th * Th, axis=0), 1.0, rtol=0, atol=1e-15)    # unit columns exactly
    s = np.sign(Th)
    assert abs(np.mean(s)) < 0.02                                            # +-1 balanced
    assert abs(np.mean(s[:, :-1] * s[:, 1:])) < 0.02                         # no pairing of neighbours


def _scalar_bit(seed, q, row, stream, b):
    """Bit b (0..127) of the Philox4x32-10 output at counter (q lo, q hi, row, stream)."""
    from oracle.philox import philox4x32_10
    w = philox4x32_10(np.uint64(q & 0xFFFFFFFF), np.uint64(q >> 32), np.uint64(row), np.uint64(stream),
                      seed & 0xFFFFFFFF, seed >> 32)
    return (int(w[b // 32]) >> (b % 32)) & 1


def test_srht_is_random_signs_times_sampled_sylvester_hadamard_rows():
    # Theta(i, r) sqrt(k) = d_r H(h_i, r): H from scipy's Sylvester construction (independent of
    # the oracle's popcount), d_r and h_i recomputed entry by entry from scalar Philox calls
    from scipy.linalg import hadamard
    from oracle.philox import philox4x32_10
    seed, k, off, m, stream = 0x0DDC0FFEE1234567, 7, 77, 300, 2
    S = theta.srht_signs(seed, k, off, m, stream)
    H = hadamard(1024)                       # rows off .. off+m-1 < 1024: only h mod 1024 matters
    for i in range(k):
        w = philox4x32_10(np.uint64(i), np.uint64(0), np.uint64(0xFFFFFFFE), np.uint64(stream),
                          seed & 0xFFFFFFFF, seed >> 32)
        h = int(w[0]) | (int(w[1]) << 32)
        for r in range(off, off + m, 7):
            d = 1 - 2 * _scalar_bit(seed, r // 128, 0xFFFFFFFF, stream, r % 128)
            assert S[i, r - off] == d * H[h % 1024, r]
    assert np.array_equal(theta.srht_signs(seed, k, off, m, stream, rows=[5, 0]), S[[5, 0]])
    assert np.array_equal(theta.srht_signs(seed, k, off + 10, 20, stream), S[:, 10:30])


def test_srht_rows_are_exactly_orthogonal_over_aligned_blocks():
    # Over the 2^p aligned rows r = q 2^p + j of X the signs cancel in Theta Theta^T and the
    # Hadamard rows are orthogonal: k (Theta Theta^T)(i, j) = 0 unless h_i = h_j (mod 2^p), and
    # then +-2^p with the sign (-1)^popcount((h_i XOR h_j) AND q 2^p) -- exactly
    seed, k, p, q = 4242, 40, 9, 3
    L = theta.levels(seed, k, q * 2 ** p, 2 ** p, dist=theta.SRHT)      # sqrt(k) Theta: +-1
    h = [int(v) for v in theta.srht_rows(seed, k)]
    G = L @ L.T
    for a in range(k):
        for b in range(k):
            same = (h[a] - h[b]) % 2 ** p == 0
            sign = -1.0 if bin((h[a] ^ h[b]) & (q * 2 ** p)).count("1") % 2 else 1.0
            assert G[a, b] == (sign * 2 ** p if same else 0.0)
    assert np.sum(G != 0) > k                                         # some rows do coincide mod 2^p
    # unit columns exactly; E[Theta^T Theta] = I (off-diagonal ~ 1/sqrt(k) for many rows)
    Th = theta.dense(seed, 4096, 5, 48, dist=theta.SRHT)
    C = Th.T @ Th
    assert np.allclose(np.diag(C), 1.0, rtol=0, atol=1e-15)
    assert np.max(np.abs(C - np.eye(48))) < 6.0 / math.sqrt(4096)
