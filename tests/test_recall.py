"""Top-1 recall estimator (Sec. 5): each query's exact nearest neighbour against the oracle's brute force
(FP64; near ties, where FP32 and FP64 may order two neighbours differently, are checked to be ties), its
distance against the FP64 value, and the hit count against the graph's first entries."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1705_01813_gb300 import datagen  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01813_gb300 import gkm
    gkm.load()
    return gkm


def _blobs(n, d, seed, centers=20):
    g = np.random.default_rng(seed)
    c = g.uniform(-10, 10, size=(centers, d))
    return (c[g.integers(0, centers, n)] + g.standard_normal((n, d))).astype(np.float32)


def _check(G, X, queries, gi, exact=False):
    Xd = torch.from_numpy(X).cuda()
    q = torch.from_numpy(queries.astype(np.int32)).cuda()
    hits, nn, nd = G.graph_recall(Xd, gi, q)
    torch.cuda.synchronize()
    nn, nd = nn.cpu().numpy(), nd.cpu().numpy()
    bi, bd = O.brute_knn(X, 1)
    X64 = X.astype(np.float64)
    for t, i in enumerate(queries):
        j, jo = nn[t], bi[i, 0]
        dj = ((X64[i] - X64[j]) ** 2).sum()
        assert j != i and 0 <= j < X.shape[0]
        if exact:
            assert j == jo and nd[t] == bd[i, 0]
        elif j != jo:  # a near tie decided in FP32
            assert abs(dj - bd[i, 0]) <= 1e-5 * bd[i, 0], (t, i, j, jo)
        assert abs(nd[t] - dj) <= (X.shape[1] + 2) * 2.0 ** -24 * dj + 1e-30
    want = int((gi.cpu().numpy()[queries, 0] == nn).sum())
    assert int(hits.item()) == want
    return want / len(queries)


@pytest.mark.parametrize("n,d,m", [(3001, 33, 77), (4096, 64, 64), (2003, 128, 300), (130, 5, 1)])
def test_recall_matches_brute_force(G, n, d, m):
    X = _blobs(n, d, n + d)
    gi, _, _, _ = G.build_knn_graph(torch.from_numpy(X).cuda(), 10, xi=50, tau=3, seed=1)
    g = np.random.default_rng(m)
    queries = np.concatenate([[0, n - 1], g.integers(0, n, m)])[:max(m, 1)]
    r = _check(G, X, queries, gi)
    assert 0.0 <= r <= 1.0


def test_recall_integer_data_exact(G):
    X = datagen.sift_like(5000, 128, 200, seed=3)
    gi, _, _, _ = G.build_knn_graph(torch.from_numpy(X).cuda(), 20, xi=50, tau=4, seed=2)
    queries = np.random.default_rng(5).integers(0, 5000, 257)
    _check(G, X, queries, gi, exact=True)


def test_recall_of_exact_graph_is_one(G):
    # k0 = 1 (n < 2 xi): one round compares all pairs, the graph is the exact KNN graph
    X = _blobs(90, 16, 9)
    gi, _, _, _ = G.build_knn_graph(torch.from_numpy(X).cuda(), 8, xi=50, tau=1, seed=3, max_cluster=128)
    queries = np.arange(90)
    assert _check(G, X, queries, gi) == 1.0


def test_recall_bf16_equals_fp32(G):
    X = _blobs(2500, 96, 11)
    xb = torch.from_numpy(X).cuda().to(torch.bfloat16)
    gi, _, _, _ = G.build_knn_graph(xb.float(), 10, xi=50, tau=2, seed=4)
    q = torch.from_numpy(np.random.default_rng(7).integers(0, 2500, 100).astype(np.int32)).cuda()
    a = G.graph_recall(xb, gi, q)
    b = G.graph_recall(xb.float(), gi, q)
    assert all(torch.equal(x, y) for x, y in zip(a, b))


def test_recall_query_out_of_range_is_reported(G):
    X = _blobs(500, 8, 13)
    Xd = torch.from_numpy(X).cuda()
    gi, _, _, _ = G.build_knn_graph(Xd, 6, xi=50, tau=1, seed=5)
    q = torch.tensor([3, 500, 7], dtype=torch.int32, device="cuda")
    ws = G.workspace(G.workspace_size(G.GK_OP_RECALL, 500, 8, 3, 6))
    hits, nn, nd = G.graph_recall(Xd, gi, q, ws=ws)
    assert G.read_status(ws) == G.GK_ERR_INVALID
    assert nn[1].item() == -1 and hits.item() <= 2
