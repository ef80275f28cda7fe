"""Boost form of GK-means (Eq. 2 state, Alg. 2's move step with Eq. 3 gains): the CUDA path against the oracle,
element by element.

Both sides fix the arithmetic the same way (FP64, composite vectors summed in ascending sample id, squared norms by
halving folds over the zero-padded vector, the gain term by term with each operation rounded once), so every
decision agrees and the final state is the same bits: labels, sizes, composite vectors D and their squared norms S.
Sizes span several 32-lane rows and ragged tails (d = 17, 100, 300, 960), the widest graph rows (kappa = 128),
visit sequences with repeats, BF16 samples, and a 10^6 x 128, k = 10^4, kappa = 50 problem (the SIFT-shaped
workload) checked on a prefix of its epoch and by properties that hold at any size."""
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


def _graph(X, kappa, seed):
    """A random neighbour list per sample (no self, no repeats): the move step reads only the ids."""
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    G = np.empty((n, kappa), np.int32)
    for i in range(n):
        row = rng.choice(n - 1, kappa, replace=False)
        G[i] = row + (row >= i)
    return G


def _state_equal(gpu, ora, what):
    Lg, Dg, cg, Sg = (t.cpu().numpy() for t in gpu)
    Lo, Do, co, So = ora
    assert np.array_equal(Lg, Lo), f"{what}: labels differ at {np.flatnonzero(Lg != Lo)[:10]}"
    assert np.array_equal(cg, co), f"{what}: counts"
    assert np.array_equal(Dg, Do), f"{what}: D max |diff| {np.abs(Dg - Do).max()}"
    assert np.array_equal(Sg, So), f"{what}: S"


def _run_both(G, X, gi, L0, k, orders, bf16=False):
    orc = O.default()
    Xo = datagen.bf16_bits_to_f32(datagen.to_bf16_bits(X)) if bf16 else X
    Xt = torch.from_numpy(Xo).cuda()
    if bf16:
        Xt = Xt.to(torch.bfloat16)
    Lt = torch.from_numpy(L0.astype(np.int32)).cuda()
    D, cnt, S = G.boost_init(Xt, Lt, k)
    Do, co, So = orc.boost_init(Xo, L0, k)
    _state_equal((Lt, D, cnt, S), (L0, Do, co, So), "init")
    Lo = L0.astype(np.int32)
    git = torch.from_numpy(gi).cuda()
    for e, order in enumerate(orders):
        mv = G.boost_epoch(Xt, git, torch.from_numpy(order.astype(np.int32)).cuda(), Lt, k, D, cnt, S)
        Lo, Do, co, So, mo, _ = orc.boost_epoch(Xo, gi, order, Lo, k, Do, co, So)
        assert int(mv.item()) == mo, f"epoch {e}: moves {int(mv.item())} vs {mo}"
        _state_equal((Lt, D, cnt, S), (Lo, Do, co, So), f"epoch {e}")
    return Lo, mo


CASES = [
    # n, d, k, kappa, data, bf16
    (3000, 128, 30, 10, "sift", False),
    (2000, 17, 20, 5, "gauss", False),
    (2500, 100, 40, 50, "gauss", False),
    (1600, 300, 16, 12, "gauss", True),
    (1200, 960, 12, 8, "gauss", False),
    (900, 32, 40, 128, "gauss", False),
    (1000, 1, 8, 3, "gauss", False),
]


@pytest.mark.parametrize("n,d,k,kappa,data,bf16", CASES)
def test_boost_epochs_equal_oracle(G, n, d, k, kappa, data, bf16):
    X = (datagen.sift_like(n, d, 200, seed=n + d) if data == "sift"
         else datagen.gauss_mixture(n, d, 2 * k, seed=n + d))
    gi = _graph(X, kappa, seed=d)
    L0 = O.default().init_labels(n, k, 11)
    rng = np.random.default_rng(kappa)
    orders = [rng.permutation(n), rng.integers(0, n, 2 * n), rng.permutation(n)]
    _, moves = _run_both(G, X, gi, L0, k, orders, bf16)


def test_boost_on_knn_graph_from_tree(G):
    """The paper's configuration at a small size: the two-means tree's partition (Alg. 1) and an exact KNN graph,
    then epochs of the move step; the objective I (Eq. 2) rises and the distortion falls."""
    orc = O.default()
    X = datagen.sift_like(4000, 64, 100, seed=3)
    k = 40
    gi, _ = orc.brute_knn(X, 16)
    L0 = orc.two_means_tree(X, k, iters=2, seed=1)
    rng = np.random.default_rng(2)
    Do, co, So = orc.boost_init(X, L0, k)
    I0 = float((So / co).sum())
    Lo, _ = _run_both(G, X, gi, L0, k, [rng.permutation(4000) for _ in range(3)])
    D1, c1, S1 = orc.boost_init(X, Lo, k)
    assert float((S1 / c1).sum()) > I0


def test_boost_edge_cases(G):
    orc = O.default()
    X = datagen.gauss_mixture(500, 24, 10, seed=4)
    gi = _graph(X, 6, seed=1)
    # no visits: nothing changes, n_moved = 0
    L0 = orc.init_labels(500, 10, 2)
    Xt, git = torch.from_numpy(X).cuda(), torch.from_numpy(gi).cuda()
    Lt = torch.from_numpy(L0).cuda()
    D, cnt, S = G.boost_init(Xt, Lt, 10)
    D0, S0 = D.clone(), S.clone()
    mv = G.boost_epoch(Xt, git, torch.empty(0, dtype=torch.int32, device="cuda"), Lt, 10, D, cnt, S)
    assert int(mv.item()) == 0 and torch.equal(D, D0) and torch.equal(S, S0)
    # k = 1: no candidates; singletons (k = n / 2 with pairs and lone samples) follow the oracle
    _run_both(G, X, gi, np.zeros(500, np.int32), 1, [np.arange(500)])
    L1 = np.repeat(np.arange(250), 2).astype(np.int32)
    idx = np.arange(0, 248, 5)
    L1[2 * idx + 1] = idx + 1  # clusters 0, 5, 10, ... keep one member, the next ones three
    _run_both(G, X, gi, L1, 250, [np.random.default_rng(5).permutation(500)])
    # bad arguments are refused on the host
    with pytest.raises(G.GkError):
        G.boost_epoch(Xt, torch.from_numpy(_graph(X, 6, 1)[:, :0].copy()).cuda(), Lt[:1].clone(), Lt, 10, D, cnt, S)
    Xw = torch.zeros(4, 1025, device="cuda")
    with pytest.raises(G.GkError):
        G.boost_init(Xw, torch.zeros(4, dtype=torch.int32, device="cuda"), 2)


def test_boost_bad_visit_id_is_reported(G):
    """A visit id out of range sets GK_ERR_INVALID and that visit makes no move; the other visits still follow the
    oracle."""
    orc = O.default()
    X = datagen.gauss_mixture(800, 16, 8, seed=6)
    gi = _graph(X, 5, seed=2)
    L0 = orc.init_labels(800, 8, 3)
    order = np.random.default_rng(1).permutation(800).astype(np.int32)
    bad = order.copy()
    bad[100] = 800
    Xt = torch.from_numpy(X).cuda()
    Lt = torch.from_numpy(L0).cuda()
    ws = G.workspace(G.workspace_size(G.GK_OP_BOOST, 800, 16, 8, 5))
    D, cnt, S = G.boost_init(Xt, Lt, 8, ws=ws)
    G.boost_epoch(Xt, torch.from_numpy(gi).cuda(), torch.from_numpy(bad).cuda(), Lt, 8, D, cnt, S, ws=ws)
    assert G.read_status(ws) == G.GK_ERR_INVALID
    Do, co, So = orc.boost_init(X, L0, 8)
    Lo, Do, co, So, _, _ = orc.boost_epoch(X, gi, np.delete(order, 100), L0, 8, Do, co, So)
    _state_equal((Lt, D, cnt, S), (Lo, Do, co, So), "bad visit skipped")


def test_boost_sift_full_size_prefix_and_properties(G):
    """The SIFT-shaped workload (10^6 x 128, k = 10^4, kappa = 50; the tree's partition, the graph built by the
    library): the first 20,000 visits equal the oracle's bit for bit; after the whole epoch the state is the Eq. 2
    state of the final labels (counts exactly, D and S to FP64 rounding), and the objective has risen."""
    n, d, k, kappa = 1_000_000, 128, 10_000, 50
    X = datagen.sift_like(n, d)
    Xt = torch.from_numpy(X).cuda()
    gi_t = G.build_knn_graph(Xt, kappa, xi=50, tau=4, seed=1, want_log=False)[0]
    L0 = G.two_means_tree(Xt, k, iters=2, seed=1)
    order = torch.randperm(n, generator=torch.Generator().manual_seed(3)).to(torch.int32)
    gi = gi_t.cpu().numpy()
    orc = O.default()
    L0n = L0.cpu().numpy()
    Lt = L0.clone()
    D, cnt, S = G.boost_init(Xt, Lt, k)
    Do, co, So = orc.boost_init(X, L0n, k)
    _state_equal((Lt, D, cnt, S), (L0n, Do, co, So), "init")
    I0 = float((So / np.maximum(co, 1))[co > 0].sum())
    m0 = 20_000
    pre = order[:m0].numpy()
    G.boost_epoch(Xt, gi_t, order[:m0].cuda(), Lt, k, D, cnt, S)
    Lo, Do, co, So, _, _ = orc.boost_epoch(X, gi, pre, L0n, k, Do, co, So)
    _state_equal((Lt, D, cnt, S), (Lo, Do, co, So), "prefix")
    mv = G.boost_epoch(Xt, gi_t, order[m0:].cuda(), Lt, k, D, cnt, S)
    assert int(mv.item()) > 0
    D2, c2, S2 = G.boost_init(Xt, Lt.clone(), k)
    assert torch.equal(c2, cnt)
    assert torch.allclose(D, D2, rtol=1e-12, atol=1e-6) and torch.allclose(S, S2, rtol=1e-12)
    ne = cnt > 0
    assert float((S[ne] / cnt[ne]).sum()) > I0
