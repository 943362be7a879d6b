"""Randomized Cholesky QR (Balabanov, arXiv 2210.09953) on one GB300.

The computation lives in ``librcqr.so`` (CUDA kernels for sm_103a behind the
C ABI of ``include/rcqr.h``); ``_binding`` is its thin ctypes binding and is
loaded on first use of any ``rcqr_*`` name, so that ``inputs`` (seeded test
matrices) can be imported without a built library.
"""
import importlib

__all__ = ["rcqr_workspace_size", "rcqr_theta_table", "rcqr_theta_scale", "rcqr_sketch",
           "rcqr_small_qr", "rcqr_qrcp", "rcqr_trsm", "rcqr_gram", "rcqr_chol_update",
           "rcqr_factor", "rcqr_reduced"]


def __getattr__(name):
    if name.startswith("rcqr_") or name in ("RcqrError", "F64", "F32", "BF16", "DIRECT", "DIRECT2",
                                            "RR", "RR2", "lib", "colmajor", "status_string"):
        return getattr(importlib.import_module("._binding", __name__), name)
    raise AttributeError(name)
