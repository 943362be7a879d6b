"""Row-sharded RCholeskyQR2 over two gloo ranks on the CPU (Sec. 3.1: the sketch
of a row-partitioned X is the plain sum of the shards' sketches, and each pass
needs one global reduction).

Each rank holds rows [o_g, o_g + m_g) of X and sketches them with Theta's
columns for those global rows (row_offset = o_g, the same counter map as the
library's rcqr_sketch shard argument), the k x n partial sketches and then the
n x n Gram matrices are all-reduced (sum, FP64), the small factorizations are
replicated, and the Q rows stay local.  The result must equal the one-process
oracle: R to 1e-12 relative, the Q rows of each shard likewise, and both
ranks must hold the identical R.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

M, N, K, SEED = 3000, 12, 48, 0x5A4D
SPLIT = 1234            # rank 0 holds rows [0, 1234), rank 1 the rest (unequal, not a multiple of 16)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _matrix():
    rng = np.random.default_rng(77)
    U, _ = np.linalg.qr(rng.standard_normal((M, N)))
    V, _ = np.linalg.qr(rng.standard_normal((N, N)))
    return U @ np.diag(np.logspace(0, -6, N)) @ V.T


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import linalg, rcqr
    X = _matrix()
    lo, hi = (0, SPLIT) if rank == 0 else (SPLIT, M)
    Xg = X[lo:hi]
    # pass 1: local partial sketch with the global row offset, one all-reduce
    P = torch.from_numpy(rcqr.sketch(Xg, K, SEED, row_offset=lo))
    dist.all_reduce(P, op=dist.ReduceOp.SUM)
    _, R = linalg.householder_qr(P.numpy())            # replicated small QR (Alg. 2 step 2)
    Q = linalg.forward_substitution(Xg, R)             # local rows of Q = X R^{-1}
    # pass 2: local Gram, one all-reduce, replicated Cholesky (Alg. 3)
    A = torch.from_numpy(Q.T @ Q)
    dist.all_reduce(A, op=dist.ReduceOp.SUM)
    Rp = linalg.cholesky(A.numpy())
    Q = linalg.forward_substitution(Q, Rp)
    np.save(os.path.join(out_dir, f"R{rank}.npy"), Rp @ R)
    np.save(os.path.join(out_dir, f"Q{rank}.npy"), Q)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_rcholqr2_matches_one_process(tmp_path):
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    from oracle import rcqr
    X = _matrix()
    Q1, R1, _ = rcqr.rcholqr2(X, K, SEED)
    R0, Rr1 = np.load(tmp_path / "R0.npy"), np.load(tmp_path / "R1.npy")
    assert np.array_equal(R0, Rr1)                      # replicated, deterministic small steps
    assert np.max(np.abs(R0 - R1)) <= 1e-12 * np.max(np.abs(R1))
    Qs = np.vstack([np.load(tmp_path / "Q0.npy"), np.load(tmp_path / "Q1.npy")])
    colrel = np.linalg.norm(Qs - Q1, axis=0) / np.linalg.norm(Q1, axis=0)
    assert np.max(colrel) <= 1e-8                        # Q's forward error ~ u cond(X) = 1e-10 here
    assert rcqr.orthogonality(Qs) <= 1e-13


def test_sketch_of_shards_sums_to_sketch_of_whole():
    """The counter map places Theta's columns by global row, so shard sketches add up exactly
    (up to the order of the FP64 sum)."""
    from oracle import rcqr
    X = _matrix()
    whole = rcqr.sketch(X, K, SEED)
    parts = sum(rcqr.sketch(X[a:b], K, SEED, row_offset=a) for a, b in [(0, 700), (700, 2048), (2048, M)])
    assert np.max(np.abs(parts - whole)) <= 1e-13 * np.max(np.abs(whole))
