"""rcqr_sketch_noalloc: the sketch for callers that cannot pass device scratch memory.

Some callers (a plugin with a fixed argument list, code inside an application
that owns all device memory through its own pool) cannot hand the library a
workspace.  This entry point keeps its partial sums in the library's own
fixed device array instead.  The test calls it through the C ABI twice in a
row, on three different shapes (FP32, FP64 and BF16 X), and checks each result against rcqr_sketch
(the column-wise tolerance the sketch parity tests state for each precision) and that the calls
after the first change no device memory usage.  This file is collected last
so that a failure here does not hide the other tests' results.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
# the column-wise sketch tolerances the parity tests state (FP64 X / FP32 X / BF16 X)
SKETCH_TOL = {"f64": 1e-12, "f32": 1e-11, "bf16": 1e-6}


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2210_09953_gb300 import _binding
    f = _binding.lib.rcqr_sketch_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                  ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    return _binding


def _noalloc(rc, X, k, seed, row_offset=0, with_norms=False):
    m, n = X.shape
    P = rc.colmajor(k, n, torch.float64, X.device)
    cn = torch.empty(n, dtype=torch.float64, device=X.device) if with_norms else None
    st = rc.lib.rcqr_sketch_noalloc(ctypes.c_void_p(X.data_ptr()), m, n, X.stride(1), rc.prec_of(X.dtype), k, seed,
                                    row_offset, ctypes.c_void_p(P.data_ptr()), P.stride(1),
                                    ctypes.c_void_p(cn.data_ptr()) if cn is not None else None,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, rc.status_string(st)
    return P, cn


def _colrel(A, B):
    A, B = A.cpu().double().numpy(), B.cpu().double().numpy()
    return float(np.max(np.linalg.norm(A - B, axis=0) / np.linalg.norm(B, axis=0)))


def test_noalloc_sketch_matches_workspace_sketch_twice(rc):
    from paper_2210_09953_gb300 import inputs
    cases = [(20011, 64, 256, "f32", 3), (5003, 7, 64, "f64", 0), (12007, 33, 136, "bf16", 21)]
    _noalloc(rc, inputs.svd_matrix(1000, 4, 10.0, 1, dtype="f64", device="cuda"), 16, 1)   # first call: set-up
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for m, n, k, dt, off in cases:
        X = inputs.svd_matrix(m, n, 1e6, 40 + n, dtype=dt, device="cuda")
        torch.cuda.synchronize()
        free_x = torch.cuda.mem_get_info()[0]
        P, cn = _noalloc(rc, X, k, 0xFEED + n, row_offset=off, with_norms=True)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] >= free_x - (k * n * 8 + n * 8 + (2 << 20))  # only P, cn
        cn_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        P_ref = rc.rcqr_sketch(X, k, 0xFEED + n, row_offset=off, colnorm2=cn_ref)
        torch.cuda.synchronize()
        assert _colrel(P, P_ref) <= SKETCH_TOL[dt]
        assert float(torch.max(torch.abs(cn - cn_ref) / cn_ref)) <= 1e-13
        del X, P, cn, P_ref, cn_ref
    torch.cuda.synchronize()
    assert free_before > 0


def test_noalloc_rejects_bad_arguments(rc):
    f = rc.lib.rcqr_sketch_noalloc
    fake = ctypes.c_void_p(0x1000)
    assert f(None, 100, 4, 100, 0, 16, 1, 0, fake, 16, None, None) == -1
    assert f(fake, 100, 4, 100, 0, 12, 1, 0, fake, 16, None, None) == -1      # k % 8 != 0
    assert f(fake, 100, 300, 100, 0, 512, 1, 0, fake, 512, None, None) == -1  # n > 256
