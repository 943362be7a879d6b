"""The C ABI: the library loads, exports every entry point include/rcqr.h declares,
agrees with the oracle on the Theta table, and rejects bad arguments on the host
(no kernel is launched for an invalid call, so these run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rcqr.h")


@pytest.fixture(scope="module")
def rc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2210_09953_gb300 import _binding
    return _binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rcqr_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rcqr_factor", "rcqr_sketch", "rcqr_reduced", "rcqr_small_qr", "rcqr_qrcp",
                     "rcqr_trsm", "rcqr_gram", "rcqr_chol_update", "rcqr_workspace_size"):
        assert required in names


def test_library_exports_every_declared_symbol(rc):
    for name in declared_functions():
        assert hasattr(rc.lib, name), name


def test_theta_table_and_scale_match_oracle(rc):
    from oracle import theta
    assert np.array_equal(np.array(rc.rcqr_theta_table(), dtype=np.float64), theta.quantile_table())
    for k in (8, 128, 256, 512, 1024, 2048):
        assert rc.rcqr_theta_scale(k) == theta.theta_scale(k)


def test_status_strings(rc):
    for code in range(-7, 1):
        assert rc.status_string(code).startswith("RCQR_")


def test_workspace_size_rules(rc):
    assert rc.rcqr_workspace_size(4096, 32, 128, 1, 0) > 0
    assert rc.rcqr_workspace_size(4096, 32, 130, 1, 0) == 0     # k not a multiple of 8
    assert rc.rcqr_workspace_size(4096, 32, 16, 1, 0) == 0      # k < n
    assert rc.rcqr_workspace_size(4096, 300, 512, 1, 0) == 0    # n > 256
    assert rc.rcqr_workspace_size(4096, 32, 128, 7, 0) == 0     # bad variant
    assert rc.rcqr_workspace_size(4096, 32, 128, 1, 9) == 0     # bad precision


def test_invalid_arguments_return_einval_without_device(rc):
    L = rc.lib
    fake = ctypes.c_void_p(0x1000)       # never dereferenced: the checks fail first
    ws = ctypes.c_void_p(0x100000)
    # null X
    assert L.rcqr_factor(None, 100, 4, 100, 0, 16, 1, 1, 0.0, fake, 100, fake, 4, None, None, ws, 1 << 30,
                         fake, None) == -1
    # ld < m
    assert L.rcqr_factor(fake, 100, 4, 99, 0, 16, 1, 1, 0.0, fake, 100, fake, 4, None, None, ws, 1 << 30,
                         fake, None) == -1
    # k < n
    assert L.rcqr_factor(fake, 100, 32, 100, 0, 16, 1, 1, 0.0, fake, 100, fake, 32, None, None, ws, 1 << 30,
                         fake, None) == -1
    # RR without perm
    assert L.rcqr_factor(fake, 100, 4, 100, 0, 16, 1, 2, 1e-8, fake, 100, fake, 4, None, None, ws, 1 << 30,
                         fake, None) == -1
    # workspace too small / misaligned
    assert L.rcqr_factor(fake, 100, 4, 100, 0, 16, 1, 1, 0.0, fake, 100, fake, 4, None, None, ws, 16,
                         fake, None) == -6
    assert L.rcqr_factor(fake, 100, 4, 100, 0, 16, 1, 1, 0.0, fake, 100, fake, 4, None, None,
                         ctypes.c_void_p(0x100001), 1 << 30, fake, None) == -6
    # Q aliasing X with a different element type (BF16 in, float out)
    assert L.rcqr_factor(fake, 100, 4, 100, 2, 16, 1, 1, 0.0, fake, 100, fake, 4, None, None, ws, 1 << 30,
                         fake, None) == -1
    # sketch: negative row offset, reduced: l != k with L = Theta
    assert L.rcqr_sketch(fake, 100, 4, 100, 0, 16, 1, -1, fake, 16, None, ws, 1 << 30, None) == -1
    assert L.rcqr_reduced(fake, 100, 4, 100, 0, 16, 1, None, 8, 0, fake, 16, None, 0, fake, 4, ws, 1 << 30,
                          None, None) == -1
    assert L.rcqr_trsm(fake, 100, 300, 100, 0, fake, 300, None, None, fake, 100, None, 0, None) == -1
    assert L.rcqr_gram(fake, 100, 4, 50, 0, None, fake, 4, ws, 1 << 30, None) == -1
    assert L.rcqr_chol_update(None, 4, 4, None, fake, 4, fake, 4, None, None) == -1
    # Theta distributions: Gaussian, Rademacher and SRHT (0, 1, 2) pass the argument check and
    # fail on the workspace size instead; anything else is EINVAL
    for theta in (0, 1, 2):
        assert L.rcqr_sketch_theta(fake, 100, 4, 100, 0, 16, 1, theta, 0, fake, 16, None, ws, 16, None) == -6
    for theta in (-1, 3):
        assert L.rcqr_sketch_theta(fake, 100, 4, 100, 0, 16, 1, theta, 0, fake, 16, None, ws, 1 << 30, None) == -1


def test_reduced_workspace_counts_the_extractor(rc):
    # an explicit L needs room for Y = L X (l x n doubles) on top of the L = Theta case
    base = rc.rcqr_reduced_workspace_size(1 << 20, 64, 256, 0, 1)
    with_l = rc.rcqr_reduced_workspace_size(1 << 20, 64, 256, 2000, 1)
    assert base > 0 and with_l >= base + 2000 * 64 * 8
    assert rc.rcqr_reduced_workspace_size(1 << 20, 64, 256, 4000, 1) == 0     # l > 2048
    # the size check comes first: too small a workspace is refused before anything is queued
    fake = ctypes.c_void_p(0x1000)
    L = rc.lib
    small = rc.rcqr_reduced_workspace_size(100, 4, 16, 0, 0)
    assert rc.rcqr_reduced_workspace_size(100, 4, 16, 2000, 0) > small
    assert L.rcqr_reduced(fake, 100, 4, 100, 0, 16, 1, fake, 2000, 2000, fake, 2000, None, 0, fake, 4,
                          ctypes.c_void_p(0x100000), small, None, None) == -6


def test_wait_poll_bound_round_trip(rc):
    prev = rc.rcqr_set_wait_polls(7)
    try:
        assert prev == 1 << 22
        assert rc.rcqr_set_wait_polls(0) == 7        # 0 restores the default
        assert rc.rcqr_set_wait_polls(0) == 1 << 22
    finally:
        rc.rcqr_set_wait_polls(0)
