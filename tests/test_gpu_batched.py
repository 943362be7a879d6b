"""Batched rank-revealing factorizations (many uneven problems in one call, CUDA-graph capturable).

Each problem i of the batch must equal the oracle's Alg. 7 (with the column
normalisation of Sec. 4 and, for RR2, one CholeskyQR pass) run with Theta's
stream index i: same rank, same pivots, X[:, perm] = Q R within the stated
precision, and Q orthonormal after the second pass.
"""
import numpy as np
import pytest
import torch

from oracle import rcqr as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2210_09953_gb300 import _binding
    return _binding


def host64(t):
    return t.detach().to("cpu", torch.float64).numpy()


def make_batch(count, seed):
    from paper_2210_09953_gb300 import inputs
    shapes = inputs.batched_shapes(count, seed, m_lo=3000, m_hi=40000)
    Xs = [inputs.rank_deficient(m, n, n // 2, 500 + i, noise=1e-12, dtype="f32", device="cuda")
          for i, (m, n) in enumerate(shapes)]
    return Xs, [4 * n for _, n in shapes]


@pytest.mark.parametrize("variant", [2, 3])
def test_batched_rr_matches_oracle_per_problem(rc, variant):
    Xs, ks = make_batch(10, 77)
    tau, seed = 1e-5, 0xBA7C4
    b = rc.rcqr_factor_batched(Xs, ks, seed, variant=variant, tau=tau)
    torch.cuda.synchronize()
    assert np.all(b.status.cpu().numpy()[:, 0] == 0)
    for i, X in enumerate(Xs):
        Xh = host64(X)
        n = Xh.shape[1]
        if variant == 2:
            Qo, So, Ro, permo, ro = orc.rrrcholqr(Xh, ks[i], seed, tau, stream=i)
        else:
            Qo, Ro, permo, ro = orc.rrrcholqr2(Xh, ks[i], seed, tau, stream=i)
        r = int(b.ranks[i][0])
        assert r == ro == n // 2
        assert b.perms[i].cpu().numpy().tolist() == permo.tolist()
        Q, R = host64(b.Qs[i]), host64(b.Rs[i])
        D = np.linalg.norm(Xh, axis=0)
        E = (Xh[:, permo] - Q[:, :r] @ R[:r]) / D[permo][None, :]
        assert np.linalg.norm(E) <= 2 * tau + 1e-4
        if variant == 3:
            assert orc.orthogonality(Q[:, :r]) <= 100 * r * 2.0 ** -24


def test_batched_graph_capture_replays_the_same_results(rc):
    Xs, ks = make_batch(8, 5)
    b = rc.Batch(Xs, ks, 99, rc.RR2, 1e-5)
    b.run()                                          # first call: streams, constants, attributes
    torch.cuda.synchronize()
    ref = [host64(R) for R in b.Rs]
    for R in b.Rs:
        R.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.run()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    for R, Rr in zip(b.Rs, ref):
        assert np.array_equal(host64(R), Rr)


def test_batched_tuner_picks_a_stream_count(rc, tmp_path, monkeypatch):
    monkeypatch.setenv("RCQR_TUNE_CACHE", str(tmp_path / "tune.json"))
    Xs, ks = make_batch(6, 11)
    b = rc.Batch(Xs, ks, 3, rc.RR, 1e-5)
    best = b.tune()
    assert best in (1, 2, 4, 6, 8, 16)
    assert (tmp_path / "tune.json").read_text().startswith("{")
    b.run()
    torch.cuda.synchronize()
    assert np.all(b.status.cpu().numpy()[:, 0] == 0)
