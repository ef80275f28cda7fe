"""Two-means tree (Alg. 1): the CUDA path's labels against the oracle's, element by element.

Both sides take every decision in FP32 with the same definition of the squared distance (one accumulator over
ascending coordinates, one fused multiply-add per step) and round each centre from an FP64 mean, so the labels
agree exactly.  (A cluster of more than 512 members has its FP64 sums added in chunks on the GPU; a centre could
then differ in its last FP32 bit only if its FP64 mean lay within 1e-16 of a rounding boundary.)"""
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


def _sizes(n, k):
    # sizes, left to right, that n and k alone fix (whole depths first, then the larger, then leftmost clusters)
    sizes = [n]
    while 2 * len(sizes) <= k:
        sizes = [h for m in sizes for h in ((m + 1) // 2, m // 2)]
    picked = set(sorted(range(len(sizes)), key=lambda j: (-sizes[j], j))[:k - len(sizes)])
    out = []
    for j, m in enumerate(sizes):
        out += [(m + 1) // 2, m // 2] if j in picked else [m]
    return out


def _run(G, X, k, iters, seed):
    L = G.two_means_tree(torch.from_numpy(X).cuda(), k, iters=iters, seed=seed)
    torch.cuda.synchronize()
    return L.cpu().numpy()


@pytest.mark.parametrize("n,d,k,iters,kind", [
    (20000, 32, 200, 2, "gauss"),    # several chunk blocks per cluster at depths 0-5; a partial last depth
    (12000, 48, 128, 3, "int"),      # k a power of two; integer data (exact sums)
    (5003, 7, 1000, 1, "gauss"),     # narrow rows, small clusters
    (3000, 130, 37, 0, "gauss"),     # seeds only; a ragged stage of coordinates
    (777, 5, 777, 2, "int"),         # k = n: every cluster one sample
    (4099, 16, 3, 4, "gauss"),       # one split below the root
    (2, 3, 2, 2, "gauss"),
])
def test_tree_equals_oracle(G, n, d, k, iters, kind):
    g = np.random.default_rng(n + k)
    if kind == "int":
        X = g.integers(0, 256, (n, d)).astype(np.float32)
    else:
        X = datagen.gauss_mixture(n, d, max(2, min(64, n // 20)), seed=n)
    got = _run(G, X, k, iters, seed=k + iters)
    want = O.two_means_tree(X, k, iters=iters, seed=k + iters)
    assert np.array_equal(got, want), np.flatnonzero(got != want)[:10]
    assert np.bincount(got, minlength=k).tolist() == _sizes(n, k)


def test_tree_single_cluster_and_determinism(G):
    X = datagen.gauss_mixture(5000, 24, 10, seed=3)
    assert (_run(G, X, 1, 2, 0) == 0).all()
    a, b = _run(G, X, 50, 2, 9), _run(G, X, 50, 2, 9)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, _run(G, X, 50, 2, 10))


def test_tree_bf16_equals_fp32_on_widened_samples(G):
    X = datagen.gauss_mixture(9000, 64, 30, seed=4)
    Xb = torch.from_numpy(X).cuda().to(torch.bfloat16)
    got = G.two_means_tree(Xb, 100, iters=2, seed=2)
    ref = G.two_means_tree(Xb.float(), 100, iters=2, seed=2)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    want = O.two_means_tree(Xb.float().cpu().numpy(), 100, iters=2, seed=2)
    assert np.array_equal(got.cpu().numpy(), want)


def test_tree_row_stride(G):
    X = datagen.gauss_mixture(3000, 20, 12, seed=5)
    wide = torch.zeros((3000, 27), device="cuda")
    wide[:, :20] = torch.from_numpy(X).cuda()
    got = G.two_means_tree(wide[:, :20], 40, iters=2, seed=1)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), O.two_means_tree(X, 40, iters=2, seed=1))


def test_tree_full_size(G):
    # SIFT-shaped size (10^6 x 128, k = 10^4, chunk blocks of 512 members over the large clusters): the sizes that
    # n and k fix, a repeat bit for bit, and the two depths below the root against the oracle run at k = 4 (each
    # of the 10^4 clusters lies inside one of its 4)
    n, d, k = 1_000_000, 128, 10_000
    X = torch.randn((n, d), device="cuda", generator=torch.Generator(device="cuda").manual_seed(7))
    L1 = G.two_means_tree(X, k, iters=2, seed=3)
    L2 = G.two_means_tree(X, k, iters=2, seed=3)
    torch.cuda.synchronize()
    assert torch.equal(L1, L2)
    sizes = _sizes(n, k)
    assert torch.bincount(L1.long(), minlength=k).cpu().tolist() == sizes
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    bounds = np.cumsum(_sizes(n, 4))[:-1]
    outer = np.searchsorted(bounds, starts, side="right")  # the depth-2 cluster holding each of the k clusters
    want = O.two_means_tree(X.cpu().numpy(), 4, iters=2, seed=3)
    assert np.array_equal(outer[L1.cpu().numpy()], want)
