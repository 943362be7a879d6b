"""Benchmark: GB/s of X factored by RCholeskyQR2 on one GB300 (and N replicas under torchrun).

Workload (the paper's first test family, Sec. 6.1 / 6.3, at the size of the
headline configuration): X = U diag(sigma) V^T, 4,194,304 x 64, sigma
log-spaced from 1 to 1e-8 (cond 1e8), Gaussian sketch with k = 256,
column-major with ld = m, RCholeskyQR2 (Alg. 3).  The headline ``value`` is
the mixed path (X stored FP32: exact sketch, FP64 small factorizations, FP32
output Q); the FP64 path (X and Q in FP64) is measured on the same matrix and
reported beside it.  Inputs are larger than L2 (1.07 GB / 2.15 GB), so no
flush is needed between steps.

--impl reference times the CPU FP64 oracle on a bounded row sample of the
same workload (the slow baseline; the oracle is test infrastructure that only
this arm, the cpu_baseline field and the tests execute).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, K, COND = 4194304, 64, 256, 1e8
METRIC = "GB/s of X factored (RCholeskyQR2, mixed path: FP32 X) at stated ||Q^TQ-I||"


def workload_name(m, n=None, k=None):
    n = N if n is None else n      # the module's N and K, as main() sets them from the arguments
    k = K if k is None else k
    return f"rcholqr2 {m}x{n} k={k} cond 1e8 (U diag(sigma) V^T), X f32 column-major"


SEED_X, SEED_THETA = 1002, 0x5EED0002
ORACLE_ROWS = 1 << 22          # the CPU oracle's sample: the whole matrix (about 10-20 s on 16 cores)
# DRAM bytes (read + write) per call on the 4M x 64 FP32 workload, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum of every kernel of the call, captured on a
# 1M-row launch and scaled by 4: per-row traffic is the same).  None where the kernels
# changed after the last capture.
TRAFFIC = {"sketch": 4 * (268463168 + 1105536 + 286893696 + 24914688 + 19934720),
           "trsm_gram": 4 * (27721 + 268700608 + 225607168 + 6237888),
           "trsm": 4 * (27721 + 268585643 + 204263595)}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--m", type=int, default=M)
    p.add_argument("--n", type=int, default=N, help="columns (the default is the headline workload)")
    p.add_argument("--k", type=int, default=K, help="sketch rows")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-path measurement")
    p.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline oracle timing")
    p.add_argument("--no-variants", action="store_true", help="skip the timings of the other variants and sizes")
    p.add_argument("--no-e2e", action="store_true", help="skip the streamed end-to-end measurement")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_time(m_rows, n=None, k=None, dtype="f32"):
    """Time the CPU oracle's RCholeskyQR2 on the first m_rows rows of the workload family."""
    n = N if n is None else n
    k = K if k is None else k
    import numpy as np
    import torch
    from paper_2210_09953_gb300 import inputs
    from oracle import rcqr as orc
    X = inputs.svd_matrix(m_rows, n, COND, SEED_X, dtype=dtype, device="cpu")
    Xh = X.to(torch.float64).numpy()
    t0 = time.perf_counter()
    Q, R, _ = orc.rcholqr2(Xh, k, SEED_THETA)
    dt = time.perf_counter() - t0
    bytes_x = m_rows * n * (4 if dtype == "f32" else 8)
    return bytes_x / dt / 1e9, dt, float(orc.orthogonality(Q))


def cpu_baseline_record(m_rows):
    gbs, dt, orth = oracle_time(m_rows)
    return {"value": round(gbs, 4), "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"RCholeskyQR2 of the first {m_rows} rows (x{N}, FP32-stored, cond 1e8, k={K}) in "
                      f"{dt:.1f} s, numpy FP64 with its default BLAS threads"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    rows = min(args.m, ORACLE_ROWS // 4)   # a bounded sample of the workload's rows
    vals = []
    for _ in range(args.warmup):
        oracle_time(rows)
    for _ in range(args.steps):
        gbs, dt, _ = oracle_time(rows)
        vals.append(gbs)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4),
            "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.m), "sample_rows": rows},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"first {rows} rows per step"},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"rcqr_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7 and parts[0].isdigit():
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [int(r[0]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": int(rows[0][1]), "reasons": sorted(reasons),
                "samples": len(rows)}


def spectral_dev(G):
    """||G - I||_2 of a small Gram matrix, on the host."""
    import torch
    Gh = G.detach().cpu()
    return float(torch.linalg.matrix_norm(Gh - torch.eye(Gh.shape[0], dtype=Gh.dtype), ord=2))


def conditioned(m, n, cond, seed, dtype, dev):
    """X = G diag(sigma) V^T with G Gaussian (near-orthonormal columns for m >> n), sigma
    log-spaced over cond, V orthonormal: condition number ~cond, built with one GEMM."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    G = torch.randn((m, n), dtype=torch.float32, device=dev, generator=g)
    V, _ = torch.linalg.qr(torch.randn((n, n), dtype=torch.float64, generator=torch.Generator().manual_seed(seed)))
    sigma = torch.logspace(0, -torch.log10(torch.tensor(float(cond))).item(), n, dtype=torch.float64)
    B = (sigma[:, None] * V.T).to(torch.float32).to(dev)
    X = torch.empty((n, m), dtype=torch.float32, device=dev).t()
    X.copy_(G @ B)
    del G
    return X if dtype == "f32" else X.to(torch.bfloat16).t().contiguous().t()


def measure_variants(rc, inputs, timed, dev, X32, ws32, Q32):
    """Time the other rows of the path: RCholeskyQR, the reduced variant, RRRCholeskyQR2,
    16M x 128 FP32/BF16, 512 batched RR problems, the adjoint at 1M x 256."""
    import torch
    from paper_2210_09953_gb300 import autograd
    out = {}
    m = X32.shape[0]

    def gbs(nbytes, ms):
        return round(nbytes / (ms * 1e-3) / 1e9, 2)

    ms = timed(lambda: rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.DIRECT, Q=Q32, workspace=ws32), 5, 2)
    out["rcholqr_mixed_4Mx64"] = {"ms": round(ms, 3), "GB/s": gbs(m * N * 4, ms)}
    ms = timed(lambda: rc.rcqr_reduced(X32, K, SEED_THETA), 5, 2)
    out["reduced_mixed_4Mx64"] = {"ms": round(ms, 3), "GB/s": gbs(m * N * 4, ms)}
    # the Rademacher embedding (one Philox bit per entry): the sketch call alone and RCholeskyQR2
    P = rc.colmajor(K, N, torch.float64, dev)
    ms = timed(lambda: rc.rcqr_sketch(X32, K, SEED_THETA, P=P, workspace=ws32, theta=rc.THETA_RADEMACHER), 5, 2)
    out["sketch_rademacher_4Mx64"] = {"ms": round(ms, 4), "GB/s": gbs(m * N * 4, ms)}
    ms = timed(lambda: rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.DIRECT2, Q=Q32, workspace=ws32,
                                      theta=rc.THETA_RADEMACHER), 5, 2)
    Qr, Rr, _, _, st_r = rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.DIRECT2, Q=Q32, workspace=ws32,
                                        theta=rc.THETA_RADEMACHER)
    Gr = Qr.double().t() @ Qr.double()
    out["rcholqr2_mixed_4Mx64_rademacher"] = {"ms": round(ms, 3), "GB/s": gbs(m * N * 4, ms),
                                              "orth_QtQ_minus_I": spectral_dev(Gr), "status": int(st_r[0])}
    # the SRHT (random signs, sampled Hadamard rows), applied as the same +-1 product
    ms = timed(lambda: rc.rcqr_sketch(X32, K, SEED_THETA, P=P, workspace=ws32, theta=rc.THETA_SRHT), 5, 2)
    out["sketch_srht_4Mx64"] = {"ms": round(ms, 4), "GB/s": gbs(m * N * 4, ms)}
    ms = timed(lambda: rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.DIRECT2, Q=Q32, workspace=ws32,
                                      theta=rc.THETA_SRHT), 5, 2)
    Qr, Rr, _, _, st_r = rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.DIRECT2, Q=Q32, workspace=ws32,
                                        theta=rc.THETA_SRHT)
    Gr = Qr.double().t() @ Qr.double()
    out["rcholqr2_mixed_4Mx64_srht"] = {"ms": round(ms, 3), "GB/s": gbs(m * N * 4, ms),
                                        "orth_QtQ_minus_I": spectral_dev(Gr), "status": int(st_r[0])}
    del P, Gr
    ws_rr = torch.empty(rc.rcqr_workspace_size(m, N, K, rc.RR2, rc.F32) + 256, dtype=torch.uint8, device=dev)
    ms = timed(lambda: rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.RR2, tau=1e-5, Q=Q32, workspace=ws_rr), 5, 2)
    _, _, _, rank, _ = rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.RR2, tau=1e-5, Q=Q32, workspace=ws_rr)
    out["rrrcholqr2_mixed_4Mx64_tau1e-5"] = {"ms": round(ms, 3), "GB/s": gbs(m * N * 4, ms), "rank": int(rank[0])}
    # the same with the strong RRQR (Gu-Eisenstat swaps, f = 1.5)
    ms = timed(lambda: rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.SRR2, tau=1e-5, Q=Q32, workspace=ws_rr), 5, 2)
    _, _, _, rank, _ = rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.SRR2, tau=1e-5, Q=Q32, workspace=ws_rr)
    out["srrrcholqr2_mixed_4Mx64_tau1e-5"] = {"ms": round(ms, 3), "GB/s": gbs(m * N * 4, ms), "rank": int(rank[0])}
    del ws_rr

    # configuration 3: 16,777,216 x 128, k = 512, RCholeskyQR2 (condition 1e8 by construction)
    for prec in ("f32", "bf16"):
        X = conditioned(1 << 24, 128, 1e8, 1003, prec, dev)
        Q = rc.colmajor(1 << 24, 128, torch.float32, dev)
        ws = torch.empty(rc.rcqr_workspace_size(1 << 24, 128, 512, rc.DIRECT2, rc.prec_of(X.dtype)) + 256,
                         dtype=torch.uint8, device=dev)
        ms = timed(lambda: rc.rcqr_factor(X, 512, 0x5EED0003, variant=rc.DIRECT2, Q=Q, workspace=ws), 3, 1)
        G = Q.double().T @ Q.double()
        orth = float(torch.linalg.matrix_norm(G.cpu() - torch.eye(128, dtype=torch.float64), ord=2))
        out[f"rcholqr2_{prec}_16Mx128"] = {"ms": round(ms, 3), "GB/s": gbs(X.numel() * X.element_size(), ms),
                                           "orth_QtQ_minus_I": orth}
        del X, Q, ws, G
        torch.cuda.empty_cache()

    # configuration 4: 512 rank-deficient FP32 problems, one batched call replayed from a CUDA graph
    shapes = inputs.batched_shapes(512, 1004)
    Xs = [inputs.rank_deficient(mm, nn, nn // 2, 4000 + i, noise=1e-12, dtype="f32", device=dev)
          for i, (mm, nn) in enumerate(shapes)]
    b = rc.Batch(Xs, [4 * nn for _, nn in shapes], 0x5EED0004, rc.RR, 1e-5)
    streams = b.tune()                  # the stream-count tuner, then capture with its choice
    b.run()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run()
    ms = timed(graph.replay, 5, 2)
    total = sum(mm * nn * 4 for mm, nn in shapes)
    ok = bool((b.status[:, 0] == 0).all())
    out["batched_rr_512"] = {"ms": round(ms, 3), "GB/s": gbs(total, ms), "problems": 512,
                             "x_bytes": total, "cuda_graph": True, "tuned_streams": streams, "status_ok": ok}
    del Xs, b, graph
    torch.cuda.empty_cache()

    # configuration 5: the adjoint, 1,048,576 x 256 FP32, k = 1024
    X = conditioned(1 << 20, 256, 1e6, 1005, "f32", dev)
    ms_f = timed(lambda: rc.rcqr_factor(X, 1024, 0xAD30, variant=rc.DIRECT2), 3, 1)
    Xg = X.clone().requires_grad_(True)
    W1 = torch.randn_like(X)
    Qf, Rf = autograd.rcholqr2(Xg, 1024, 0xAD30)
    loss = torch.sum(W1 * Qf) + torch.sum(Rf)

    def backward():
        Xg.grad = None
        torch.autograd.grad(loss, Xg, retain_graph=True)
    ms_b = timed(backward, 3, 1)
    out["adjoint_rcholqr2_f32_1Mx256"] = {"forward_ms": round(ms_f, 3), "backward_ms": round(ms_b, 3),
                                          "GB/s_forward": gbs(X.numel() * 4, ms_f)}
    del X, Xg, W1, Qf, Rf, loss
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2210_09953_gb300 import _binding as rc
    from paper_2210_09953_gb300 import inputs

    m = args.m
    # replicas: every rank factors its own matrix (weak scaling, no collective on the data path)
    X64 = inputs.svd_matrix(m, N, COND, SEED_X + rank, dtype="f64", device=dev)
    X32 = X64.to(torch.float32).t().contiguous().t()
    stream = torch.cuda.current_stream()

    def make_buffers(X):
        prec = rc.prec_of(X.dtype)
        qdt = torch.float64 if prec == rc.F64 else torch.float32
        Q = rc.colmajor(m, N, qdt, dev)
        ws = torch.empty(rc.rcqr_workspace_size(m, N, K, rc.DIRECT2, prec) + 256, dtype=torch.uint8, device=dev)
        return Q, ws

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(steps):
            fn()
        end.record(stream)
        torch.cuda.synchronize()
        ms = start.elapsed_time(end) / steps
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t[0])
        return ms

    Q32, ws32 = make_buffers(X32)

    def step32():
        rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.DIRECT2, Q=Q32, workspace=ws32)

    with Clocks(local) as clk:
        ms32 = timed(step32, args.steps, args.warmup)
    clocks = clk.summary()
    Q, R, _, _, status = rc.rcqr_factor(X32, K, SEED_THETA, variant=rc.DIRECT2, Q=Q32, workspace=ws32)
    torch.cuda.synchronize()
    ok32 = int(status[0]) == 0
    G = (Q.double().t() @ Q.double())
    orth32 = spectral_dev(G)
    res32 = float(torch.norm(Q.double() @ R - X32.double()) / torch.norm(X32.double()))
    bytes32 = m * N * 4
    value = world * bytes32 / (ms32 * 1e-3) / 1e9

    # dominant kernel: the sketch (Alg. 2 step 1), timed alone on the same stream
    P = rc.colmajor(K, N, torch.float64, dev)
    ms_sketch = timed(lambda: rc.rcqr_sketch(X32, K, SEED_THETA, P=P, workspace=ws32), max(3, args.steps), 2)
    R1 = rc.rcqr_small_qr(P, want_S=False)
    ms_trsm = timed(lambda: rc.rcqr_trsm(X32, R1, Q=Q32), max(3, args.steps), 2)
    # the dominant kernel of the step: the first substitution fused with the Gram (one launch
    # plus its R preparation and the Gram reduction)
    ms_tg = timed(lambda: rc.rcqr_trsm_gram(X32, R1, Q=Q32, workspace=ws32), max(3, args.steps), 2) if N <= 64 else None

    fp64 = None
    if not args.no_fp64:
        Q64, ws64 = make_buffers(X64)

        def step64():
            rc.rcqr_factor(X64, K, SEED_THETA, variant=rc.DIRECT2, Q=Q64, workspace=ws64)
        ms64 = timed(step64, max(1, min(args.steps, 3)), 1)
        Qd, Rd, _, _, st64 = rc.rcqr_factor(X64, K, SEED_THETA, variant=rc.DIRECT2, Q=Q64, workspace=ws64)
        torch.cuda.synchronize()
        Gd = Qd.t() @ Qd
        fp64 = {"value": round(world * m * N * 8 / (ms64 * 1e-3) / 1e9, 3), "unit": "GB/s",
                "ms_per_step": round(ms64, 3),
                "orth": spectral_dev(Gd),
                "status": int(st64[0])}
        del Q64, ws64

    e2e = None
    if not args.no_e2e:
        # End to end through the public call, streaming: every step copies its X from pinned host
        # memory, factors it and copies Q and R back.  Three device buffer sets (X, Q, R, rank,
        # status and workspace each, allocated once, so no buffer changes hands between streams)
        # on three streams let step s+1's upload, step s's factorization and step s-1's download
        # run at the same time; every timed step's copies are inside the timed region.  Host
        # buffers are flat pinned arrays viewed column-major, so each transfer is one copy.
        Xh_flat = torch.empty(N * m, dtype=torch.float32, pin_memory=True)
        Xh_flat.view(N, m).t().copy_(X32)
        Qh_flat = torch.empty(N * m, dtype=torch.float32, pin_memory=True)
        Rh = torch.empty((N, N), dtype=torch.float64, pin_memory=True).t()
        NSETS = 3
        bufs = []
        for _ in range(NSETS):
            Xd = rc.colmajor(m, N, torch.float32, dev)
            Qd = rc.colmajor(m, N, torch.float32, dev)
            Rd = rc.colmajor(N, N, torch.float64, dev)
            rkd = torch.empty(1, dtype=torch.int64, device=dev)
            std = torch.zeros(2, dtype=torch.int32, device=dev)
            wsd = torch.empty(rc.rcqr_workspace_size(m, N, K, rc.DIRECT2, rc.F32) + 256, dtype=torch.uint8,
                              device=dev)
            bufs.append((Xd, Xd.t().reshape(-1), Qd, Qd.t().reshape(-1), Rd, rkd, std, wsd))
        s_in, s_run, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)

        def e2e_steps(count, marks=None):
            done_out = [None] * NSETS       # event: the buffer set's previous Q download finished
            for s in range(count):
                Xd, Xf, Qd, Qf, Rd, rkd, std, wsd = bufs[s % NSETS]
                ev = {}
                with torch.cuda.stream(s_in):
                    if done_out[s % NSETS] is not None:
                        s_in.wait_event(done_out[s % NSETS])
                    if marks is not None:
                        ev["up0"] = torch.cuda.Event(enable_timing=True)
                        ev["up0"].record(s_in)
                    Xf.copy_(Xh_flat, non_blocking=True)
                    up = torch.cuda.Event(enable_timing=marks is not None)
                    up.record(s_in)
                with torch.cuda.stream(s_run):
                    s_run.wait_event(up)
                    rc.rcqr_factor(Xd, K, SEED_THETA, variant=rc.DIRECT2, Q=Qd, workspace=wsd, R=Rd, rank=rkd,
                                   status=std)
                    ran = torch.cuda.Event(enable_timing=marks is not None)
                    ran.record(s_run)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ran)
                    Qh_flat.copy_(Qf, non_blocking=True)
                    Rh.copy_(Rd, non_blocking=True)
                    dn = torch.cuda.Event(enable_timing=marks is not None)
                    dn.record(s_out)
                    done_out[s % NSETS] = dn
                if marks is not None:
                    ev.update(up=up, ran=ran, dn=dn)
                    marks.append(ev)
            for st_ in (s_in, s_run, s_out):
                stream.wait_stream(st_)

        e2e_steps(NSETS)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_e2e = max(16, args.steps)
        e0.record(stream)
        for st_ in (s_in, s_run, s_out):
            st_.wait_stream(stream)
        e2e_steps(n_e2e)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = e0.elapsed_time(e1) / n_e2e
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms_e2e], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e2e = float(t[0])
        # where the streamed steps' time goes (an untimed run with an event at every phase boundary):
        # per step the upload, factorization and download intervals, and the mean period
        marks = []
        e2e_steps(6, marks)
        torch.cuda.synchronize()
        t0 = marks[0]["up0"]
        tl = [{"up": (t0.elapsed_time(mk["up0"]), t0.elapsed_time(mk["up"])),
               "run": (t0.elapsed_time(mk["up"]), t0.elapsed_time(mk["ran"])),
               "down": (t0.elapsed_time(mk["ran"]), t0.elapsed_time(mk["dn"]))} for mk in marks]
        period = (tl[-1]["down"][1] - tl[1]["down"][1]) / (len(tl) - 2)
        Xf0, Qf0 = bufs[0][1], bufs[0][3]
        ms_h2d = timed(lambda: Xf0.copy_(Xh_flat, non_blocking=True), 3, 1)
        ms_d2h = timed(lambda: Qh_flat.copy_(Qf0, non_blocking=True), 3, 1)

        def both():
            with torch.cuda.stream(s_in):
                Xf0.copy_(Xh_flat, non_blocking=True)
            with torch.cuda.stream(s_out):
                Qh_flat.copy_(bufs[1][3], non_blocking=True)
            for st_ in (s_in, s_out):
                stream.wait_stream(st_)

        def both_timed():
            for st_ in (s_in, s_out):
                st_.wait_stream(stream)
            both()
        ms_both = timed(both_timed, 3, 1)
        e2e_timeline = {"period_ms": round(period, 3),
                        "upload_ms": round(statistics.median(b - a for a, b in (t["up"] for t in tl)), 3),
                        "factor_ms": round(statistics.median(b - a for a, b in (t["run"] for t in tl)), 3),
                        "download_ms": round(statistics.median(b - a for a, b in (t["down"] for t in tl)), 3),
                        "h2d_and_d2h_together_ms": round(ms_both, 3),
                        "steps": [{k: [round(v[0], 3), round(v[1], 3)] for k, v in t.items()} for t in tl]}
        e2e = {"value": round(world * m * N * 4 / (ms_e2e * 1e-3) / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": m * N * 4, "d2h_bytes_per_step": m * N * 4 + N * N * 8,
               "ms_per_step": round(ms_e2e, 3), "h2d_ms": round(ms_h2d, 3), "d2h_ms": round(ms_d2h, 3),
               "buffer_sets": NSETS, "timeline": e2e_timeline}
        del bufs, Xh_flat, Qh_flat
        torch.cuda.empty_cache()

    # measured arithmetic roofs (throughput probes, each launch timed alone)
    scratch = torch.empty(int(rc.lib.rcqr_probe_scratch_bytes()), dtype=torch.uint8, device=dev)
    probes = {}
    for name, kind, iters in (("philox_calls", rc.PROBE_PHILOX, 2000), ("ffma", rc.PROBE_FFMA, 20000),
                              ("dfma", rc.PROBE_DFMA, 2000), ("imad", rc.PROBE_IMAD, 20000)):
        ops = [0]

        def run_probe(kind=kind, iters=iters):
            ops[0] = rc.rcqr_probe(kind, iters, scratch)
        ms = timed(run_probe, 3, 1)
        probes[name] = ops[0] / (ms * 1e-3)
    del scratch

    variants = None
    headline = (m, N, K) == (M, 64, 256)
    if not args.no_variants and headline:
        variants = measure_variants(rc, inputs, timed, dev, X32, ws32, Q32)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # rooflines of the three bulk calls of the step, each against the measured HBM bandwidth:
    # algorithmic bytes = X read once (sketch), X read + Q written (substitution fused with the
    # Gram, and the in-place pass-2 substitution timed here as X -> Q); `roofline` is the call
    # with the largest share of the step
    def roof(name, kernel, nbytes, ms):
        ach = nbytes / (ms * 1e-3) / 1e9
        tr = TRAFFIC.get(name) if (m, N, K) == (M, 64, 256) else None
        return {"kernel": kernel, "bound": "hbm", "achieved": round(ach, 2), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "traffic": tr, "peak_source": peak_src,
                "algorithmic_bytes": nbytes, "ms": round(ms, 4)}
    roofs = {
        "sketch": roof("sketch", "rcqr_sketch: block_exp_kernel + sketch_tc_kernel + reduction (FP32 X)",
                       m * N * 4, ms_sketch),
        "trsm": roof("trsm", "rcqr_trsm: trsm32 SIMT substitution + prep (FP32 X -> Q)", m * N * 8, ms_trsm),
    }
    if ms_tg is not None:
        roofs["trsm_gram"] = roof("trsm_gram", ("rcqr_trsm_gram: trsm_tc_kernel (blocked substitution on tcgen05 "
                                                "fused with A = Q^T Q)" if 32 < N <= 64 else
                                                "rcqr_trsm_gram: trsm32_gram_kernel") +
                                  " + prep + Gram reduction (FP32 X)", m * N * 8, ms_tg)
    dominant = max(roofs, key=lambda k_: roofs[k_]["ms"])
    # the sketch against its generation roof: k Theta entries per X row, 16 entries per
    # Philox call for the Gaussian levels (measured Philox calls/s x 16 entries/call)
    gen_peak = probes["philox_calls"] * 16 / 1e9
    gen_ach = K * m / (ms_sketch * 1e-3) / 1e9
    roof_gen = {"kernel": roofs["sketch"]["kernel"], "bound": "alu", "achieved": round(gen_ach, 2),
                "peak": round(gen_peak, 2), "unit": "G Theta entries/s", "frac": round(gen_ach / gen_peak, 4),
                "peak_source": "measured: rcqr_probe Philox4x32-10 calls/s x 16 bytes (entries) per call"}
    # per factorization (mixed path, Alg. 3): status reset, sketch (block exponents, tensor-core
    # sketch, reduction), Householder R + sign fix, rank, substitution prep + substitution fused
    # with the Gram + Gram reduction, Cholesky update, substitution prep + substitution
    launches_per_step = 13

    if rank == 0:
        cpu = None
        if not args.no_cpu:
            # bounded: the oracle's cost grows with m n^2, so wider workloads take fewer rows
            cpu = cpu_baseline_record(min(m, ORACLE_ROWS * 64 // max(N, 64)))
        line = {
            "metric": METRIC,
            "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms32, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 storage / f64 sketch and small ops",
            "data": "synthetic",
            "config": {"workload": workload_name(m),
                       "seed_theta": SEED_THETA, "l2": "inputs larger than L2 (no flush)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "accuracy": {"orth_QtQ_minus_I": orth32, "residual_rel_F": res32, "status_ok": ok32},
            "fp64_path": fp64,
            "variants": variants,
            "kernels_ms": {"sketch": round(ms_sketch, 4), "trsm": round(ms_trsm, 4),
                           "trsm_gram": round(ms_tg, 4) if ms_tg is not None else None},
            "roofline": roofs[dominant],
            "rooflines": roofs,
            "roofline_sketch_generation": roof_gen,
            "measured_rates": {"philox_calls_per_s": round(probes["philox_calls"], 1),
                               "fp32_fma_per_s": round(probes["ffma"], 1), "fp64_fma_per_s": round(probes["dfma"], 1),
                               "int32_mad_per_s": round(probes["imad"], 1)},
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    global N, K
    args = parse()
    N, K = args.n, args.k
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
