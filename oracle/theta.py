"""The sketching matrix Theta (Sec. 2, rescaled Gaussian OSE), realised from Philox bytes.

The paper asks for a k x m oblivious subspace embedding drawn from a seeded
generator so that it is never stored (Sec. 2, Sec. 3.1), with i.i.d. zero-mean
entries of variance 1/k.  The realisation used here (a reading; the paper
fixes no bit stream):

* Entry (i, r) -- row i < k of Theta, global row r of X -- takes byte
  (r mod 16) of the Philox4x32-10 output for
      counter = (floor(r/16) mod 2^32, floor(r/16) div 2^32, i, stream),
      key     = (seed mod 2^32, seed div 2^32),
  byte b of the 128-bit output being bits 8*(b mod 4) .. 8*(b mod 4)+7 of
  word floor(b/4).
* That byte t in [0, 256) selects the level
      T[t] = round(44 * Phi^{-1}((t + 1/2) / 256)),
  an integer in [-127, 127]: the 256-point quantile discretisation of N(0, 1)
  scaled by 44 (a sub-Gaussian, zero-mean, antisymmetric distribution).
* Theta(i, r) = T[t] / sqrt(k * v) with v = (1/256) * sum_t T[t]^2, so
  E[Theta^T Theta] = I exactly.

Phi^{-1} here is scipy's ``ndtri`` (a library primitive); the library builds
its own table with its own inverse-CDF code and the tests compare the two
tables entry by entry.

The Rademacher embedding (Sec. 2 lists it beside the Gaussian one) uses one
bit per entry:
* entry (i, r) takes bit (r mod 128) of the Philox4x32-10 output for
      counter = (floor(r/128) mod 2^32, floor(r/128) div 2^32, i, stream),
  bit b being bit (b mod 32) of word floor(b/32);
* Theta(i, r) = (1 - 2 bit) / sqrt(k): +-1/sqrt(k), so E[Theta^T Theta] = I and
  every column of Theta has unit norm exactly.

The subsampled randomized Hadamard transform (SRHT, Sec. 2: random signs, a
Hadamard matrix over X's rows padded with zeros to a power of two, uniform row
sampling, the factor sqrt(1/k)) is written out as its definition
Theta = sqrt(1/k) S H D (a reading; the paper fixes no bit stream and no order):
* D = diag(d_r): d_r = 1 - 2 bit, bit (r mod 128) of the Philox4x32-10 output for
      counter = (floor(r/128) mod 2^32, floor(r/128) div 2^32, 2^32 - 1, stream)
  (the Rademacher bit stream at the row index 2^32 - 1, which no Theta row takes);
* H is the Sylvester-Hadamard matrix of order 2^64 (X padded with zero rows):
  H(h, r) = (-1)^popcount(h AND r);
* S samples k rows of H uniformly, with replacement: Theta row i takes Hadamard row
      h_i = w0 + 2^32 w1,  (w0, w1) the first two words of the Philox output for
      counter = (i, 0, 2^32 - 2, stream);
* Theta(i, r) = d_r (-1)^popcount(h_i AND r) / sqrt(k).  Every column has unit norm
  exactly and E[Theta^T Theta] = I.  Over any 2^p aligned rows of X, two rows of
  Theta whose h differ modulo 2^p are orthogonal, and two whose h agree are equal
  up to sign.
"""
import numpy as np
from scipy.special import ndtri

from .philox import philox4x32_10

TABLE_SCALE = 44.0
LEVELS = 256


def quantile_table():
    """The 256 integer levels T[t] (float64 holding integers)."""
    t = np.arange(LEVELS, dtype=np.float64)
    x = TABLE_SCALE * ndtri((t + 0.5) / LEVELS)
    # round half away from zero; no level lies within 1e-3 of a half-integer
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def table_variance():
    """v = mean of T^2 (exact in FP64: an integer sum divided by 256)."""
    T = quantile_table()
    return float(np.sum(T * T)) / LEVELS


def theta_scale(k):
    """c = 1/sqrt(k v): Theta = c * (integer levels)."""
    return 1.0 / np.sqrt(float(k) * table_variance())


def theta_bytes(seed, k, row_offset, m, stream=0, rows=None):
    """The k x m array of Philox bytes t(i, r) for rows r = row_offset .. row_offset+m-1.

    ``rows`` (optional) selects Theta's rows i (default 0..k-1); the result then
    has one line per selected row.
    """
    sel = np.arange(k) if rows is None else np.asarray(rows)
    if m == 0:
        return np.zeros((len(sel), 0), dtype=np.int64)
    k = len(sel)
    q0 = row_offset // 16
    q1 = (row_offset + m - 1) // 16
    q = np.arange(q0, q1 + 1, dtype=np.uint64)[None, :]          # one Philox call per 16 rows
    i = sel.astype(np.uint64)[:, None]
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    words = philox4x32_10(q & np.uint64(0xFFFFFFFF), q >> np.uint64(32),
                          i, np.uint64(stream), seed & 0xFFFFFFFF, seed >> 32)
    out = np.empty((k, q.shape[1], 16), dtype=np.int64)
    for b in range(16):                                          # byte b of the 128-bit output
        out[:, :, b] = ((words[b >> 2] >> np.uint64(8 * (b & 3))) & np.uint64(0xFF)).astype(np.int64)
    out = out.reshape(k, -1)
    start = row_offset - 16 * q0
    return out[:, start:start + m]


def theta_levels(seed, k, row_offset, m, stream=0, rows=None):
    """Integer levels G(i, r) = T[t(i, r)] as float64 (Theta = theta_scale(k) * G)."""
    return quantile_table()[theta_bytes(seed, k, row_offset, m, stream, rows)]


def theta(seed, k, row_offset, m, stream=0):
    """Dense Theta[:, row_offset:row_offset+m] in FP64 (for small m only)."""
    return theta_scale(k) * theta_levels(seed, k, row_offset, m, stream)


GAUSSIAN, RADEMACHER = "gaussian", "rademacher"


def rademacher_signs(seed, k, row_offset, m, stream=0, rows=None):
    """The k x m array of +-1 (float64) for rows r = row_offset .. row_offset+m-1 (one bit each)."""
    sel = np.arange(k) if rows is None else np.asarray(rows)
    if m == 0:
        return np.zeros((len(sel), 0))
    q0 = row_offset // 128
    q1 = (row_offset + m - 1) // 128
    q = np.arange(q0, q1 + 1, dtype=np.uint64)[None, :]          # one Philox call per 128 rows
    i = sel.astype(np.uint64)[:, None]
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    words = philox4x32_10(q & np.uint64(0xFFFFFFFF), q >> np.uint64(32),
                          i, np.uint64(stream), seed & 0xFFFFFFFF, seed >> 32)
    bits = np.empty((len(sel), q.shape[1], 128), dtype=np.int64)
    for b in range(128):
        bits[:, :, b] = ((words[b >> 5] >> np.uint64(b & 31)) & np.uint64(1)).astype(np.int64)
    bits = bits.reshape(len(sel), -1)
    start = row_offset - 128 * q0
    return 1.0 - 2.0 * bits[:, start:start + m]


SRHT = "srht"
SRHT_SIGN_ROW = 0xFFFFFFFF       # the counter word of the SRHT's sign stream D
SRHT_ROW_TAG = 0xFFFFFFFE        # the counter word of its row sampling S


def srht_rows(seed, k, stream=0, rows=None):
    """The sampled Hadamard row h_i (uint64) of every Theta row i (S of the SRHT)."""
    sel = np.arange(k) if rows is None else np.asarray(rows)
    i = sel.astype(np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    w = philox4x32_10(i, np.uint64(0), np.uint64(SRHT_ROW_TAG), np.uint64(stream),
                      seed & 0xFFFFFFFF, seed >> 32)
    return w[0].astype(np.uint64) | (w[1].astype(np.uint64) << np.uint64(32))


def parity64(v):
    """popcount(v) mod 2 of uint64 values, by folding."""
    v = np.asarray(v, dtype=np.uint64).copy()
    for s in (32, 16, 8, 4, 2, 1):
        v ^= v >> np.uint64(s)
    return (v & np.uint64(1)).astype(np.int64)


def srht_signs(seed, k, row_offset, m, stream=0, rows=None):
    """The k x m array of +-1 (float64) of the SRHT, d_r (-1)^popcount(h_i AND r), for
    rows r = row_offset .. row_offset+m-1 of X."""
    sel = np.arange(k) if rows is None else np.asarray(rows)
    if m == 0:
        return np.zeros((len(sel), 0))
    d = rademacher_signs(seed, 1, row_offset, m, stream, rows=[SRHT_SIGN_ROW])[0]
    h = srht_rows(seed, k, stream, sel)
    r = np.arange(row_offset, row_offset + m, dtype=np.uint64)
    par = parity64(h[:, None] & r[None, :])
    return d[None, :] * (1.0 - 2.0 * par)


def levels(seed, k, row_offset, m, stream=0, rows=None, dist=GAUSSIAN):
    """Theta / scale(k, dist): the integer levels (Gaussian table) or the signs (Rademacher, SRHT)."""
    if dist == RADEMACHER:
        return rademacher_signs(seed, k, row_offset, m, stream, rows)
    if dist == SRHT:
        return srht_signs(seed, k, row_offset, m, stream, rows)
    return theta_levels(seed, k, row_offset, m, stream, rows)


def scale(k, dist=GAUSSIAN):
    """Theta = scale(k, dist) * levels(...): 1/sqrt(k v) (Gaussian table) or 1/sqrt(k)."""
    return 1.0 / np.sqrt(float(k)) if dist in (RADEMACHER, SRHT) else theta_scale(k)


def dense(seed, k, row_offset, m, stream=0, dist=GAUSSIAN):
    """Dense Theta[:, row_offset:row_offset+m] in FP64 for either distribution (small m only)."""
    return scale(k, dist) * levels(seed, k, row_offset, m, stream, dist=dist)
