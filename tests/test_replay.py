"""Replay of repeated one-call requests (gk_set_replay): a graph construction or fit repeated with equal arguments
runs as one captured CUDA graph and gives the results of a direct call bit for bit; other arguments are captured
anew; a call inside a caller's own capture runs directly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture()
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01813_gb300 import gkm
    gkm.load()
    yield gkm
    gkm.set_replay(False)


def _data(n=12000, d=48, seed=3):
    g = np.random.default_rng(seed)
    c = g.uniform(-10, 10, (60, d))
    return torch.from_numpy((c[g.integers(0, 60, n)] + g.standard_normal((n, d))).astype(np.float32)).cuda()


def _buffers(G, X, kappa, k, iters, tau=3, xi=50):
    n, d = X.shape
    ws = G.workspace(max(G.workspace_size_build(n, d, kappa, xi, tau, 128),
                         G.workspace_size(G.GK_OP_FIT, n, d, k, kappa)))
    return dict(gi=torch.empty((n, kappa), dtype=torch.int32, device="cuda"),
                gd=torch.empty((n, kappa), device="cuda"), l0=torch.empty(n, dtype=torch.int32, device="cuda"),
                lab=torch.empty(n, dtype=torch.int32, device="cuda"), C=torch.empty((k, d), device="cuda"),
                cnt=torch.empty(k, dtype=torch.int32, device="cuda"), ws=ws)


def _run(G, X, b, kappa, k, iters, seed, want_log=False, tau=3):
    s = G.build_knn_graph(X, kappa, 50, tau, 128, seed, labels_out=b["l0"], g_idx=b["gi"], g_dist=b["gd"],
                          want_log=want_log, precision=1, ws=b["ws"])
    f = G.kmeans_fit(X, k, b["gi"], iters, seed=seed + 1, labels_out=b["lab"], C_out=b["C"], counts_out=b["cnt"],
                     want_log=want_log, precision=1, ws=b["ws"])
    torch.cuda.synchronize()
    return [t.clone() for t in (b["gi"], b["gd"], b["l0"], b["lab"], b["C"], b["cnt"])], s[3], f[3]


def test_replay_equals_direct_calls(G):
    X = _data()
    kappa, k, iters = 16, 150, 4
    b = _buffers(G, X, kappa, k, iters)
    G.set_replay(False)
    ref, slog, flog = _run(G, X, b, kappa, k, iters, 5, want_log=True)
    G.set_replay(True)
    with torch.cuda.stream(torch.cuda.Stream()):  # a stream of its own (the legacy default one runs directly)
        for _ in range(3):  # capture, then two replays
            got, s2, f2 = _run(G, X, b, kappa, k, iters, 5, want_log=True)
            assert all(torch.equal(a, c) for a, c in zip(ref, got))
            assert s2 == slog and f2 == flog
        # another seed: captured anew, equal to its direct call
        other, _, _ = _run(G, X, b, kappa, k, iters, 6)
    G.set_replay(False)
    direct, _, _ = _run(G, X, b, kappa, k, iters, 6)
    assert all(torch.equal(a, c) for a, c in zip(other, direct))
    assert not torch.equal(other[0], ref[0])


def test_call_inside_a_callers_capture_runs_directly(G):
    X = _data(n=6000, d=32, seed=4)
    kappa, k, iters = 12, 60, 2
    b = _buffers(G, X, kappa, k, iters, tau=2)
    G.set_replay(False)
    ref, _, _ = _run(G, X, b, kappa, k, iters, 7, tau=2)
    G.set_replay(True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _run(G, X, b, kappa, k, iters, 7, tau=2)  # warm-up outside the capture
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            G.build_knn_graph(X, kappa, 50, 2, 128, 7, labels_out=b["l0"], g_idx=b["gi"], g_dist=b["gd"],
                              want_log=False, precision=1, ws=b["ws"])
            G.kmeans_fit(X, k, b["gi"], iters, seed=8, labels_out=b["lab"], C_out=b["C"], counts_out=b["cnt"],
                         want_log=False, precision=1, ws=b["ws"])
    b["gi"].zero_()
    graph.replay()
    torch.cuda.synchronize()
    got = [t.clone() for t in (b["gi"], b["gd"], b["l0"], b["lab"], b["C"], b["cnt"])]
    assert all(torch.equal(a, c) for a, c in zip(ref, got))
