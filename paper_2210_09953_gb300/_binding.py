"""ctypes binding of librcqr.so (argument marshalling only).

Every function here has the name of the C entry point it calls and takes
torch tensors for the device arrays; it passes their data pointers, the
caller's current CUDA stream and a workspace tensor, and raises RcqrError on
a non-OK status.  No arithmetic of the method happens here: every step runs
in the CUDA kernels of the library.  Importing this module loads the library
and fails loudly if it is missing or was not built.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librcqr.so")

F64, F32, BF16 = 0, 1, 2
DIRECT, DIRECT2, RR, RR2, SRR, SRR2 = 0, 1, 2, 3, 4, 5
THETA_GAUSSIAN, THETA_RADEMACHER, THETA_SRHT = 0, 1, 2
STATUS_NAMES = {0: "RCQR_OK", -1: "RCQR_EINVAL", -2: "RCQR_ENOTSPD", -3: "RCQR_ERANK0",
                -4: "RCQR_ECUDA", -5: "RCQR_ETIMEOUT", -6: "RCQR_EWORKSPACE", -7: "RCQR_EUNSUPPORTED"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2210_09953_gb300.build`")
lib = ctypes.CDLL(LIB_PATH)

_i64, _u64, _i32, _dbl, _vp, _sz = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t)

_SIGS = {
    "rcqr_status_string": (ctypes.c_char_p, [_i32]),
    "rcqr_workspace_size": (_sz, [_i64, _i64, _i64, _i32, _i32]),
    "rcqr_reduced_workspace_size": (_sz, [_i64, _i64, _i64, _i64, _i32]),
    "rcqr_set_wait_polls": (ctypes.c_uint32, [ctypes.c_uint32]),
    "rcqr_probe_scratch_bytes": (_sz, []),
    "rcqr_probe": (_i64, [_i32, _i32, _vp, _sz, _vp]),
    "rcqr_theta_table": (_i32, [_vp]),
    "rcqr_theta_scale": (_dbl, [_i64]),
    "rcqr_sketch": (_i32, [_vp, _i64, _i64, _i64, _i32, _i64, _u64, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "rcqr_sketch_theta": (_i32, [_vp, _i64, _i64, _i64, _i32, _i64, _u64, _i32, _i64, _vp, _i64, _vp, _vp, _sz,
                                 _vp]),
    "rcqr_small_qr": (_i32, [_vp, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp]),
    "rcqr_qrcp": (_i32, [_vp, _i64, _i64, _i64, _vp, _dbl, _vp, _i64, _vp, _vp, _vp, _sz, _vp, _vp]),
    "rcqr_srrqr": (_i32, [_vp, _i64, _i64, _i64, _vp, _dbl, _dbl, _vp, _i64, _vp, _vp, _vp, _sz, _vp, _vp]),
    "rcqr_trsm": (_i32, [_vp, _i64, _i64, _i64, _i32, _vp, _i64, _vp, _vp, _vp, _i64, _vp, _sz, _vp]),
    "rcqr_gram": (_i32, [_vp, _i64, _i64, _i64, _i32, _vp, _vp, _i64, _vp, _sz, _vp]),
    "rcqr_trsm_gram": (_i32, [_vp, _i64, _i64, _i64, _i32, _vp, _i64, _vp, _vp, _vp, _i64, _vp, _i64, _vp, _sz,
                              _vp]),
    "rcqr_chol_update": (_i32, [_vp, _i64, _i64, _vp, _vp, _i64, _vp, _i64, _vp, _vp]),
    "rcqr_factor": (_i32, [_vp, _i64, _i64, _i64, _i32, _i64, _u64, _i32, _dbl, _vp, _i64, _vp, _i64,
                           _vp, _vp, _vp, _sz, _vp, _vp]),
    "rcqr_factor_theta": (_i32, [_vp, _i64, _i64, _i64, _i32, _i64, _u64, _i32, _i32, _dbl, _vp, _i64, _vp,
                                 _i64, _vp, _vp, _vp, _sz, _vp, _vp]),
    "rcqr_factor_implicit": (_i32, [_vp, _i64, _i64, _i64, _i32, _i64, _u64, _vp, _i64, _vp, _i64, _vp, _i64, _vp,
                                    _sz, _vp, _vp]),
    "rcqr_implicit_workspace_size": (_sz, [_i64, _i64, _i64]),
    "rcqr_implicit_q_times": (_i32, [_vp, _i64, _i64, _i64, _i32, _vp, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _sz,
                                     _vp]),
    "rcqr_implicit_qt_times": (_i32, [_vp, _i64, _i64, _i64, _i32, _vp, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _sz,
                                      _vp]),
    "rcqr_colblock_workspace_size": (_sz, [_i64, _i64, _i64, _i64, _i32]),
    "rcqr_colblock_step": (_i32, [_vp, _i64, _i64, _i64, _i32, _i64, _u64, _i64, _i32, _vp, _i64, _vp, _i64, _vp,
                                  _i64, _vp, _sz, _vp, _vp]),
    "rcqr_factor_colwise": (_i32, [_vp, _i64, _i64, _i64, _i32, _i64, _u64, _i64, _i32, _vp, _i64, _vp, _i64, _vp,
                                   _i64, _vp, _sz, _vp, _vp]),
    "rcqr_reduced": (_i32, [_vp, _i64, _i64, _i64, _i32, _i64, _u64, _vp, _i64, _i64, _vp, _i64, _vp,
                            _i64, _vp, _i64, _vp, _sz, _vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class RcqrError(RuntimeError):
    def __init__(self, func, status):
        super().__init__(f"{func} returned {STATUS_NAMES.get(status, status)}")
        self.status = status


def _check(func, status):
    if status != 0:
        raise RcqrError(func, status)


def prec_of(dtype):
    return {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[dtype]


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _ld(t):
    """Leading dimension of a column-major (m, n) tensor (stride (1, ld))."""
    if t.dim() != 2 or (t.stride(0) != 1 and t.shape[0] > 1):
        raise ValueError("expected a column-major (m, n) tensor with stride (1, ld)")
    return t.stride(1) if t.shape[1] > 1 else max(t.shape[0], 1)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _workspace(nbytes, device):
    n = max(int(nbytes), 1)
    return torch.empty(n + 256, dtype=torch.uint8, device=device)


def _aligned_ptr(ws):
    p = ws.data_ptr()
    return ctypes.c_void_p((p + 255) & ~255), ws.numel() - ((-p) % 256) - 1


def status_string(s):
    return lib.rcqr_status_string(s).decode()


def rcqr_workspace_size(m, n, k, variant=DIRECT, prec=F64):
    return int(lib.rcqr_workspace_size(m, n, k, variant, prec))


def rcqr_reduced_workspace_size(m, n, k, l=0, prec=F64):
    return int(lib.rcqr_reduced_workspace_size(m, n, k, l, prec))


def rcqr_set_wait_polls(polls):
    """Bound of the sketch pipeline's device waits for later calls (0: the default); returns the previous one."""
    return int(lib.rcqr_set_wait_polls(polls))


PROBE_PHILOX, PROBE_FFMA, PROBE_DFMA, PROBE_IMAD = 0, 1, 2, 3


def rcqr_probe(kind, iters, scratch):
    """Launch one throughput probe on the current stream; returns its operation count."""
    ops = int(lib.rcqr_probe(kind, iters, _ptr(scratch), scratch.numel() * scratch.element_size(), _stream()))
    if ops < 0:
        raise RcqrError("rcqr_probe", -1)
    return ops


def rcqr_theta_table():
    out = (ctypes.c_int32 * 256)()
    _check("rcqr_theta_table", lib.rcqr_theta_table(ctypes.cast(out, ctypes.c_void_p)))
    return [int(v) for v in out]


def rcqr_theta_scale(k):
    return float(lib.rcqr_theta_scale(k))


def colmajor(m, n, dtype, device, ld=None):
    ld = m if ld is None else ld
    return torch.empty((n, ld), dtype=dtype, device=device).t()[:m, :]


def rcqr_sketch(X, k, seed, row_offset=0, P=None, colnorm2=None, workspace=None, theta=THETA_GAUSSIAN):
    m, n = X.shape
    prec = prec_of(X.dtype)
    if P is None:
        P = colmajor(k, n, torch.float64, X.device)
    ws = workspace if workspace is not None else _workspace(rcqr_workspace_size(m, n, k, DIRECT, prec), X.device)
    wp, wb = _aligned_ptr(ws)
    if theta == THETA_GAUSSIAN:
        _check("rcqr_sketch", lib.rcqr_sketch(_ptr(X), m, n, _ld(X), prec, k, seed, row_offset, _ptr(P), _ld(P),
                                              _ptr(colnorm2), wp, wb, _stream()))
    else:
        _check("rcqr_sketch_theta", lib.rcqr_sketch_theta(_ptr(X), m, n, _ld(X), prec, k, seed, theta, row_offset,
                                                          _ptr(P), _ld(P), _ptr(colnorm2), wp, wb, _stream()))
    return P


def rcqr_small_qr(P, want_S=True):
    k, n = P.shape
    R = colmajor(n, n, torch.float64, P.device)
    S = colmajor(k, n, torch.float64, P.device) if want_S else None
    ws = _workspace(rcqr_workspace_size(max(k, 8), n, max(8, (k + 7) // 8 * 8), DIRECT, F64), P.device)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_small_qr", lib.rcqr_small_qr(_ptr(P), k, n, _ld(P), _ptr(S), _ld(S) if S is not None else 0,
                                              _ptr(R), _ld(R), wp, wb, _stream()))
    return (S, R) if want_S else R


def rcqr_qrcp(P, tau, colnorm2=None):
    k, n = P.shape
    R = colmajor(n, n, torch.float64, P.device)
    perm = torch.empty(n, dtype=torch.int32, device=P.device)
    rank = torch.empty(1, dtype=torch.int64, device=P.device)
    status = torch.zeros(2, dtype=torch.int32, device=P.device)
    ws = _workspace(rcqr_workspace_size(max(k, 8), n, max(8, (k + 7) // 8 * 8), DIRECT, F64), P.device)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_qrcp", lib.rcqr_qrcp(_ptr(P), k, n, _ld(P), _ptr(colnorm2), float(tau), _ptr(R), _ld(R),
                                      _ptr(perm), _ptr(rank), wp, wb, _ptr(status), _stream()))
    return R, perm, rank, status


def rcqr_srrqr(P, tau, f=1.5, colnorm2=None):
    """Column pivoting followed by Gu-Eisenstat swaps with parameter f: (R, perm, rank, status)."""
    k, n = P.shape
    R = colmajor(n, n, torch.float64, P.device)
    perm = torch.empty(n, dtype=torch.int32, device=P.device)
    rank = torch.empty(1, dtype=torch.int64, device=P.device)
    status = torch.zeros(2, dtype=torch.int32, device=P.device)
    ws = _workspace(rcqr_workspace_size(max(k, 8), n, max(8, (k + 7) // 8 * 8), DIRECT, F64), P.device)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_srrqr", lib.rcqr_srrqr(_ptr(P), k, n, _ld(P), _ptr(colnorm2), float(tau), float(f), _ptr(R),
                                        _ld(R), _ptr(perm), _ptr(rank), wp, wb, _ptr(status), _stream()))
    return R, perm, rank, status


def rcqr_trsm(X, R, perm=None, rank=None, Q=None, workspace=None):
    m, n = X.shape
    prec = prec_of(X.dtype)
    if Q is None:
        Q = colmajor(m, n, torch.float64 if prec == F64 else torch.float32, X.device)
    ws = workspace if workspace is not None else _workspace(
        rcqr_workspace_size(m, n, max(8, (n + 7) // 8 * 8), DIRECT, prec), X.device)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_trsm", lib.rcqr_trsm(_ptr(X), m, n, _ld(X), prec, _ptr(R), _ld(R), _ptr(perm), _ptr(rank),
                                      _ptr(Q), _ld(Q), wp, wb, _stream()))
    return Q


def rcqr_trsm_gram(X, R, perm=None, rank=None, Q=None, workspace=None):
    """(Q, A): Q = X R^{-1} and A = Q^T Q in one pass (mixed path, n <= 64)."""
    m, n = X.shape
    prec = prec_of(X.dtype)
    if Q is None:
        Q = colmajor(m, n, torch.float32, X.device)
    A = colmajor(n, n, torch.float64, X.device)
    ws = workspace if workspace is not None else _workspace(
        rcqr_workspace_size(m, n, max(8, (n + 7) // 8 * 8), DIRECT2, prec), X.device)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_trsm_gram", lib.rcqr_trsm_gram(_ptr(X), m, n, _ld(X), prec, _ptr(R), _ld(R), _ptr(perm),
                                                _ptr(rank), _ptr(Q), _ld(Q), _ptr(A), _ld(A), wp, wb, _stream()))
    return Q, A


def rcqr_gram(Q, rank=None):
    m, n = Q.shape
    prec = prec_of(Q.dtype)
    A = colmajor(n, n, torch.float64, Q.device)
    ws = _workspace(rcqr_workspace_size(m, n, max(8, (n + 7) // 8 * 8), DIRECT, prec), Q.device)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_gram", lib.rcqr_gram(_ptr(Q), m, n, _ld(Q), prec, _ptr(rank), _ptr(A), _ld(A), wp, wb,
                                      _stream()))
    return A


def rcqr_chol_update(A, R, rank=None):
    n = A.shape[0]
    Rp = colmajor(n, n, torch.float64, A.device)
    status = torch.zeros(2, dtype=torch.int32, device=A.device)
    _check("rcqr_chol_update", lib.rcqr_chol_update(_ptr(A), n, _ld(A), _ptr(rank), _ptr(Rp), _ld(Rp),
                                                    _ptr(R), _ld(R), _ptr(status), _stream()))
    return Rp, status


def rcqr_factor(X, k, seed, variant=DIRECT2, tau=0.0, Q=None, workspace=None, R=None, rank=None, status=None,
                theta=THETA_GAUSSIAN):
    """Returns (Q, R, perm, rank, status); perm is None for the direct variants.  Q, R, rank and
    status may be given (preallocated buffers); the others are allocated on the current stream."""
    m, n = X.shape
    prec = prec_of(X.dtype)
    dev = X.device
    if Q is None:
        Q = colmajor(m, n, torch.float64 if prec == F64 else torch.float32, dev)
    if R is None:
        R = colmajor(n, n, torch.float64, dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev) if variant in (RR, RR2, SRR, SRR2) else None
    if rank is None:
        rank = torch.empty(1, dtype=torch.int64, device=dev)
    if status is None:
        status = torch.zeros(2, dtype=torch.int32, device=dev)
    ws = workspace if workspace is not None else _workspace(rcqr_workspace_size(m, n, k, variant, prec), dev)
    wp, wb = _aligned_ptr(ws)
    if theta == THETA_GAUSSIAN:
        _check("rcqr_factor", lib.rcqr_factor(_ptr(X), m, n, _ld(X), prec, k, seed, variant, float(tau), _ptr(Q),
                                              _ld(Q), _ptr(R), _ld(R), _ptr(perm), _ptr(rank), wp, wb, _ptr(status),
                                              _stream()))
    else:
        _check("rcqr_factor_theta", lib.rcqr_factor_theta(_ptr(X), m, n, _ld(X), prec, k, seed, theta, variant,
                                                          float(tau), _ptr(Q), _ld(Q), _ptr(R), _ld(R), _ptr(perm),
                                                          _ptr(rank), wp, wb, _ptr(status), _stream()))
    return Q, R, perm, rank, status


def rcqr_factor_implicit(X, k, seed, Q1=None, workspace=None):
    """RCholeskyQR2 without its last substitution: returns (Q1, R, Rp, status), Q = Q1 Rp^{-1}."""
    m, n = X.shape
    prec = prec_of(X.dtype)
    dev = X.device
    if Q1 is None:
        Q1 = colmajor(m, n, torch.float64 if prec == F64 else torch.float32, dev)
    R = colmajor(n, n, torch.float64, dev)
    Rp = colmajor(n, n, torch.float64, dev)
    status = torch.zeros(2, dtype=torch.int32, device=dev)
    ws = workspace if workspace is not None else _workspace(rcqr_workspace_size(m, n, k, DIRECT2, prec), dev)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_factor_implicit", lib.rcqr_factor_implicit(_ptr(X), m, n, _ld(X), prec, k, seed, _ptr(Q1), _ld(Q1),
                                                            _ptr(R), _ld(R), _ptr(Rp), _ld(Rp), wp, wb, _ptr(status),
                                                            _stream()))
    return Q1, R, Rp, status


def rcqr_implicit_q_times(Q1, Rp, Y):
    """Z = Q Y = Q1 (Rp^{-1} Y) (m x c, Q1's type); Y n x c float64."""
    m, n = Q1.shape
    c = Y.shape[1]
    prec = F64 if Q1.dtype == torch.float64 else F32
    Z = colmajor(m, c, Q1.dtype, Q1.device)
    ws = _workspace(lib.rcqr_implicit_workspace_size(m, n, c), Q1.device)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_implicit_q_times", lib.rcqr_implicit_q_times(_ptr(Q1), m, n, _ld(Q1), prec, _ptr(Rp), _ld(Rp),
                                                              _ptr(Y), _ld(Y), c, _ptr(Z), _ld(Z), wp, wb, _stream()))
    return Z


def rcqr_implicit_qt_times(Q1, Rp, B):
    """Z = Q^T B = Rp^{-T} (Q1^T B) (n x c, float64); B m x c of Q1's type."""
    m, n = Q1.shape
    c = B.shape[1]
    prec = F64 if Q1.dtype == torch.float64 else F32
    Z = colmajor(n, c, torch.float64, Q1.device)
    ws = _workspace(lib.rcqr_implicit_workspace_size(m, n, c), Q1.device)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_implicit_qt_times", lib.rcqr_implicit_qt_times(_ptr(Q1), m, n, _ld(Q1), prec, _ptr(Rp), _ld(Rp),
                                                                _ptr(B), _ld(B), c, _ptr(Z), _ld(Z), wp, wb, _stream()))
    return Z


def rcqr_factor_colwise(X, k, seed, b, rgs=False):
    """Alg. 4 over the column blocks of X (width b): returns (Q, S, R, status)."""
    m, n = X.shape
    prec = prec_of(X.dtype)
    dev = X.device
    Q = colmajor(m, n, torch.float64 if prec == F64 else torch.float32, dev)
    S = colmajor(k, n, torch.float64, dev)
    R = torch.zeros((n, n), dtype=torch.float64, device=dev).t()
    status = torch.zeros(2, dtype=torch.int32, device=dev)
    need = max(int(lib.rcqr_colblock_workspace_size(m, min(b, n - i0), k, i0, prec)) for i0 in range(0, n, b))
    ws = _workspace(need, dev)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_factor_colwise", lib.rcqr_factor_colwise(_ptr(X), m, n, _ld(X), prec, k, seed, b, int(rgs), _ptr(Q),
                                                          _ld(Q), _ptr(S), _ld(S), _ptr(R), _ld(R), wp, wb,
                                                          _ptr(status), _stream()))
    return Q, S, R, status


def rcqr_colblock_step(Xi, k, seed, i0, Q, S, R, rgs=False):
    """One block of Alg. 4 into the caller's (Q, S, R); returns status."""
    m, b = Xi.shape
    prec = prec_of(Xi.dtype)
    status = torch.zeros(2, dtype=torch.int32, device=Xi.device)
    ws = _workspace(lib.rcqr_colblock_workspace_size(m, b, k, i0, prec), Xi.device)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_colblock_step", lib.rcqr_colblock_step(_ptr(Xi), m, b, _ld(Xi), prec, k, seed, i0, int(rgs), _ptr(Q),
                                                        _ld(Q), _ptr(S), _ld(S), _ptr(R), _ld(R), wp, wb,
                                                        _ptr(status), _stream()))
    return status


def rcqr_reduced(X, k, seed, L=None, want_S=True):
    """Returns (Z, S, R, status); L (l x m, float64, column-major) or None for L = Theta."""
    m, n = X.shape
    prec = prec_of(X.dtype)
    dev = X.device
    l = k if L is None else L.shape[0]
    Z = colmajor(l, n, torch.float64, dev)
    S = colmajor(k, n, torch.float64, dev) if want_S else None
    R = colmajor(n, n, torch.float64, dev)
    status = torch.zeros(2, dtype=torch.int32, device=dev)
    ws = _workspace(rcqr_reduced_workspace_size(m, n, k, l if L is not None else 0, prec), dev)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_reduced", lib.rcqr_reduced(_ptr(X), m, n, _ld(X), prec, k, seed, _ptr(L), l,
                                            _ld(L) if L is not None else 0, _ptr(Z), _ld(Z), _ptr(S),
                                            _ld(S) if S is not None else 0, _ptr(R), _ld(R), wp, wb,
                                            _ptr(status), _stream()))
    return Z, S, R, status


class rcqr_problem(ctypes.Structure):
    _fields_ = [("X", _vp), ("m", _i64), ("n", _i64), ("ldx", _i64), ("k", _i64), ("seed", _u64),
                ("Q", _vp), ("ldq", _i64), ("R", _vp), ("ldr", _i64), ("perm", _vp), ("rank", _vp),
                ("dev_status", _vp)]


lib.rcqr_batched_workspace_size.restype = _sz
lib.rcqr_batched_workspace_size.argtypes = [_vp, _i32, _i32, _i32]
lib.rcqr_factor_batched.restype = _i32
lib.rcqr_factor_batched.argtypes = [_vp, _i32, _i32, _i32, _dbl, _vp, _sz, _vp]
lib.rcqr_tune_batched.restype = _i32
lib.rcqr_tune_batched.argtypes = [_vp, _i32, _i32, _i32, _dbl, _vp, _sz, _vp, _vp]


class Batch:
    """Device buffers and the host problem array of one batched call (kept alive together)."""

    def __init__(self, Xs, ks, seed, variant, tau=0.0):
        self.Xs = Xs
        self.variant, self.tau = variant, float(tau)
        self.prec = prec_of(Xs[0].dtype)
        dev = Xs[0].device
        qdt = torch.float64 if self.prec == F64 else torch.float32
        rr = variant in (RR, RR2, SRR, SRR2)
        self.Qs, self.Rs, self.perms, self.ranks = [], [], [], []
        self.status = torch.zeros((len(Xs), 2), dtype=torch.int32, device=dev)
        arr = (rcqr_problem * len(Xs))()
        for i, (X, k) in enumerate(zip(Xs, ks)):
            m, n = X.shape
            Q = colmajor(m, n, qdt, dev)
            R = colmajor(n, n, torch.float64, dev)
            perm = torch.empty(n, dtype=torch.int32, device=dev) if rr else None
            rank = torch.empty(1, dtype=torch.int64, device=dev)
            self.Qs.append(Q), self.Rs.append(R), self.perms.append(perm), self.ranks.append(rank)
            arr[i] = rcqr_problem(X.data_ptr(), m, n, _ld(X), k, seed, Q.data_ptr(), _ld(Q), R.data_ptr(), _ld(R),
                                  perm.data_ptr() if perm is not None else None, rank.data_ptr(),
                                  self.status[i].data_ptr())
        self.arr = arr
        nbytes = lib.rcqr_batched_workspace_size(ctypes.cast(arr, _vp), len(Xs), variant, self.prec)
        if nbytes == 0:
            raise RcqrError("rcqr_batched_workspace_size", -1)
        self.ws = _workspace(nbytes, dev)

    def run(self):
        wp, wb = _aligned_ptr(self.ws)
        _check("rcqr_factor_batched", lib.rcqr_factor_batched(ctypes.cast(self.arr, _vp), len(self.Xs), self.variant,
                                                              self.prec, self.tau, wp, wb, _stream()))

    def tune(self):
        wp, wb = _aligned_ptr(self.ws)
        best = ctypes.c_int(0)
        _check("rcqr_tune_batched", lib.rcqr_tune_batched(ctypes.cast(self.arr, _vp), len(self.Xs), self.variant,
                                                          self.prec, self.tau, wp, wb, _stream(), ctypes.byref(best)))
        return best.value


def rcqr_factor_batched(Xs, ks, seed, variant=RR, tau=0.0):
    """Factor every X in Xs (problem i uses Theta stream i); returns the Batch with Qs, Rs, perms, ranks, status."""
    b = Batch(Xs, ks, seed, variant, tau)
    b.run()
    return b


lib.rcqr_qr_adjoint_workspace_size.restype = _sz
lib.rcqr_qr_adjoint_workspace_size.argtypes = [_i64, _i64]
lib.rcqr_qr_adjoint.restype = _i32
lib.rcqr_qr_adjoint.argtypes = [_vp, _i64, _i64, _i64, _i32, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp,
                                _sz, _vp]


def rcqr_qr_adjoint(Q, R, Qbar, Rbar):
    """Xbar of the thin QR map for the factors (Q, R) and incoming gradients (Qbar, Rbar)."""
    m, n = Q.shape
    prec = F64 if Q.dtype == torch.float64 else F32
    Xbar = colmajor(m, n, Q.dtype, Q.device)
    ws = _workspace(lib.rcqr_qr_adjoint_workspace_size(m, n), Q.device)
    wp, wb = _aligned_ptr(ws)
    _check("rcqr_qr_adjoint", lib.rcqr_qr_adjoint(_ptr(Q), m, n, _ld(Q), prec, _ptr(R), _ld(R), _ptr(Qbar), _ld(Qbar),
                                                  _ptr(Rbar), _ld(Rbar), _ptr(Xbar), _ld(Xbar), wp, wb, _stream()))
    return Xbar
