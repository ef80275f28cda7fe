"""BF16 sample storage: every entry point that reads the samples, given BF16 samples, returns what
the FP32 call returns on the same samples widened to FP32, bit for bit (the kernels widen each
element exactly as they read it and keep the FP32 arithmetic).  The FP32 path is checked against
the oracle elsewhere; one update is checked against the oracle here directly, on the widened
samples.  Widths cover the 16-byte vector paths (d a multiple of 8), the scalar paths (odd d), the
tensor-core refinement (64 <= d <= 128; BF16 samples staged uncentred, FP32 samples centred) and wide
rows; one case has a padded row stride."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from tests import parity as P  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01813_gb300 import gkm
    gkm.load()
    return gkm


def _pair(n, d, seed, centers=20, box=10.0, ld=None):
    """(BF16 samples on the device, the same samples widened to FP32), optionally inside a wider row."""
    g = np.random.default_rng(seed)
    c = g.uniform(-box, box, size=(centers, d))
    X = (c[g.integers(0, centers, n)] + g.standard_normal((n, d))).astype(np.float32)
    xb = torch.from_numpy(X).cuda().to(torch.bfloat16)
    if ld is not None and ld > d:
        wide = torch.zeros((n, ld), dtype=torch.bfloat16, device="cuda")
        wide[:, :d] = xb
        xb = wide[:, :d]
    return xb, xb.float()


def _same(a, b):
    for x, y in zip(a, b):
        if isinstance(x, torch.Tensor):
            assert torch.equal(x, y)
        else:
            assert x == y


@pytest.mark.parametrize("n,d,kappa", [(3000, 32, 20), (1037, 33, 50), (2000, 128, 16), (501, 5, 8),
                                       (1500, 512, 40), (999, 264, 24)])  # 256-element chunks, ragged last one
def test_init_graph(G, n, d, kappa):
    xb, xf = _pair(n, d, d)
    _same(G.init_graph(xb, kappa, 11), G.init_graph(xf, kappa, 11))


@pytest.mark.parametrize("precision", [0, 1, 2, 4])
@pytest.mark.parametrize("n,d,k,kappa,ld", [(20000, 32, 200, 20, None), (5003, 33, 97, 16, None),
                                            (4001, 128, 300, 12, None), (3001, 960, 40, 10, None),
                                            (6007, 64, 120, 20, 72)])
def test_assign_step(G, n, d, k, kappa, ld, precision):
    xb, xf = _pair(n, d, n, ld=ld)
    gi, _ = G.init_graph(xf, kappa, 3)
    L = G.init_labels(n, k, 5)
    C = torch.randn((k, d), device="cuda") * 4
    a = G.assign_step(xb, gi, C, L, precision=precision)
    b = G.assign_step(xf, gi, C, L, precision=precision)
    _same(a, b)


@pytest.mark.parametrize("precision", [3])
def test_assign_tensor_core_screening_rejects_bf16_samples(G, precision):
    xb, _ = _pair(1000, 32, 1)
    gi, _ = G.init_graph(xb, 8, 3)
    L = G.init_labels(1000, 10, 5)
    C = torch.randn((10, 32), device="cuda")
    with pytest.raises(G.GkError) as e:
        G.assign_step(xb, gi, C, L, precision=precision)
    assert e.value.code == G.GK_ERR_INVALID and "BF16 samples" in str(e.value)
    with pytest.raises(G.GkError):
        G.build_knn_graph(xb, 8, xi=50, tau=1, precision=precision)


@pytest.mark.parametrize("n,d,k,ld", [(20000, 32, 200, None), (5003, 36, 97, None), (4099, 33, 600, None),
                                      (3001, 960, 40, None), (7001, 24, 50, 40), (12000, 256, 120, None)])
def test_update_step(G, n, d, k, ld):
    xb, xf = _pair(n, d, n + 1, ld=ld)
    L = G.init_labels(n, k, 7)
    a = G.update_step(xb, L, k, torch.zeros((k, d), device="cuda"))
    b = G.update_step(xf, L, k, torch.zeros((k, d), device="cuda"))
    _same(a, b)


def test_update_step_matches_oracle_on_widened_samples(G):
    n, d, k = 12007, 40, 150
    xb, xf = _pair(n, d, 17)
    L = G.init_labels(n, k, 19)
    C, cnt, _, _, _ = G.update_step(xb, L, k, torch.zeros((k, d), device="cuda"))
    Co, cnto, _, _ = O.update(xf.cpu().numpy(), L.cpu().numpy(), k, np.zeros((k, d)))
    assert np.array_equal(cnt.cpu().numpy(), cnto.astype(np.int32))
    P.check_centroids(C.cpu().numpy(), Co, cnto)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n,d,k,kappa,cap", [(20000, 32, 400, 20, 128), (5003, 68, 60, 33, 128),
                                             (6007, 80, 20, 10, 128), (1501, 65, 9, 12, 128),
                                             (4001, 128, 90, 12, 128), (3001, 960, 50, 50, 128),
                                             (2000, 8, 3, 16, 500), (2003, 200, 40, 20, 128),
                                             (4001, 512, 80, 40, 128), (3000, 256, 2, 24, 300)])
def test_graph_refine(G, n, d, k, kappa, cap, precision):
    xb, xf = _pair(n, d, n + d)
    L = G.init_labels(n, k, 23)
    gb = G.init_graph(xf, kappa, 29)
    gf = tuple(t.clone() for t in gb)
    G.graph_refine(xb, L, k, *gb, max_cluster=cap, precision=precision)
    G.graph_refine(xf, L, k, *gf, max_cluster=cap, precision=precision)
    _same(gb, gf)


def test_group_entry_points(G):
    n, d, k, kappa = 9001, 96, 120, 16
    xb, xf = _pair(n, d, 31)
    L = G.init_labels(n, k, 37)
    off, mem, cnt = G.group_by_label(L, k)
    Cb = G.update_from_groups(xb, off, mem, k, torch.zeros((k, d), device="cuda"))
    Cf = G.update_from_groups(xf, off, mem, k, torch.zeros((k, d), device="cuda"))
    assert torch.equal(Cb, Cf)
    gb = G.init_graph(xf, kappa, 41)
    gf = tuple(t.clone() for t in gb)
    G.graph_refine_groups(xb, off, mem, k, *gb, precision=1)
    G.graph_refine_groups(xf, off, mem, k, *gf, precision=1)
    _same(gb, gf)


@pytest.mark.parametrize("precision", [0, 1, 2, 4])
@pytest.mark.parametrize("n,d,k", [(20000, 32, 200), (8009, 100, 80)])
def test_fit_and_build(G, n, d, k, precision):
    xb, xf = _pair(n, d, n - d)
    a = G.build_knn_graph(xb, 16, xi=50, tau=3, seed=43, precision=precision)
    b = G.build_knn_graph(xf, 16, xi=50, tau=3, seed=43, precision=precision)
    _same(a, b)
    L0 = G.init_labels(n, k, 47)
    _same(G.kmeans_fit(xb, k, a[0], 5, init_labels=L0, precision=precision),
          G.kmeans_fit(xf, k, a[0], 5, init_labels=L0, precision=precision))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("d", [512, 128, 96])
def test_graph_refine_unit_vectors(G, d, precision):
    """Deep-feature-shaped rows (weakly concentrated von Mises-Fisher unit vectors, stored BF16): all pair
    distances lie close together, the case that tests the Gram's error bound hardest (d <= 128)."""
    from paper_1705_01813_gb300 import datagen
    n, k, kappa = 6000, 120, 40
    xb = datagen.deep_like_device(n, d, 1200, 50.0, seed=53, device="cuda")
    xf = xb.float()
    L = G.init_labels(n, k, 59)
    gb = G.init_graph(xf, kappa, 61)
    gf = tuple(t.clone() for t in gb)
    for _ in range(2):
        G.graph_refine(xb, L, k, *gb, precision=precision)
        G.graph_refine(xf, L, k, *gf, precision=precision)
    _same(gb, gf)


@pytest.mark.parametrize("precision", [0, 2, 4])
def test_assign_unit_vectors_many_candidates(G, precision):
    """Deep-feature-shaped rows at the ratio n / k = 10 of the 10^7 x 512 workload: every sample has
    about kappa + 1 distinct candidate clusters at nearly equal distances, the hardest case for the
    BF16 and int8 screenings' bounds."""
    from paper_1705_01813_gb300 import datagen
    n, d, k, kappa = 20000, 512, 2000, 40
    xb = datagen.deep_like_device(n, d, 4000, 50.0, seed=67, device="cuda")
    xf = xb.float()
    gi, _ = G.init_graph(xf, kappa, 71)
    L = G.init_labels(n, k, 73)
    C, _, _, _, _ = G.update_step(xf, L, k, torch.zeros((k, d), device="cuda"))
    a = G.assign_step(xb, gi, C, L, precision=precision)
    b = G.assign_step(xf, gi, C, L, precision=0)
    _same(a, b)
