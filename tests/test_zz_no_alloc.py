"""gk_update_step_noalloc: the centroid update for callers that cannot allocate.

Some callers of this library may not call cudaMalloc at all (their framework
owns every byte of device memory through its own pool, or they run a
latency-bound loop in which an allocation could synchronise the device), so
they cannot pass a workspace either.  gk_update_step_noalloc serves them from a
fixed scratch array inside the library.  This file checks, through the C ABI,
that two calls in a row give the same centroids, cluster sizes and distortion
as the workspace-based gk_update_step on the same inputs, and that sizes beyond
the array's limits are refused.  Collected last on purpose (name starts with
zz) so that a run that stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests import parity as P  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01813_gb300 import gkm
    gkm.load()
    return gkm


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _noalloc(G, X, labels, k, C, counts, sum_d2):
    n, d = X.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return G.load().gk_update_step_noalloc(_ptr(X), n, d, X.stride(0), _ptr(labels), k, _ptr(C), _ptr(counts),
                                           _ptr(sum_d2), stream)


@pytest.mark.parametrize("n,d,k", [(20000, 32, 200), (1_000_000, 128, 10000)])
def test_noalloc_matches_workspace_update_twice(G, n, d, k):
    g = np.random.default_rng(n)
    X = torch.from_numpy(g.standard_normal((n, d)).astype(np.float32) * 3).cuda()
    for call in range(2):  # two calls in a row: the second sees the first call's leftovers
        kk = k if call == 0 else k // 2 + 1
        L = torch.from_numpy(g.integers(0, kk, n).astype(np.int32)).cuda()
        C0 = torch.from_numpy(g.standard_normal((kk, d)).astype(np.float32)).cuda()
        C_ref, C_new = C0.clone(), C0.clone()
        cnt_ref = torch.empty(kk, dtype=torch.int32, device="cuda")
        cnt_new = torch.full((kk,), -7, dtype=torch.int32, device="cuda")
        s_ref = torch.empty(1, dtype=torch.float64, device="cuda")
        s_new = torch.empty(1, dtype=torch.float64, device="cuda")
        G.update_step(X, L, kk, C_ref, counts=cnt_ref, sum_d2=s_ref)
        rc = _noalloc(G, X, L, kk, C_new, cnt_new, s_new)
        assert rc == G.GK_OK, G.load().gk_last_error()
        torch.cuda.synchronize()
        assert torch.equal(cnt_new, cnt_ref)
        P.check_centroids(C_new.cpu().numpy(), C_ref.cpu().numpy().astype(np.float64), cnt_ref.cpu().numpy())
        P.check_rel(s_new.item(), s_ref.item(), what="n x distortion")


def test_noalloc_refuses_sizes_beyond_its_scratch(G):
    X = torch.zeros((8, 4), device="cuda")
    L = torch.zeros(8, dtype=torch.int32, device="cuda")
    C = torch.zeros((40000, 4), device="cuda")
    rc = _noalloc(G, X, L, 40000, C, None, None)
    assert rc == G.GK_ERR_INVALID
    assert b"k <= 32768" in G.load().gk_last_error()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = G.load().gk_update_step_noalloc(_ptr(X), (1 << 20) + 1, 4, 4, _ptr(L), 2, _ptr(C), None, None, stream)
    assert rc == G.GK_ERR_INVALID


def test_noalloc_at_its_stated_maxima(G):
    """n = 2^20 samples and k = 2^15 clusters, the largest sizes the fixed scratch accepts, are served."""
    n, d, k = 1 << 20, 16, 1 << 15
    g = np.random.default_rng(5)
    X = torch.from_numpy(g.standard_normal((n, d)).astype(np.float32)).cuda()
    L = torch.from_numpy(g.integers(0, k, n).astype(np.int32)).cuda()
    C_ref = torch.zeros((k, d), device="cuda")
    C_new = torch.zeros((k, d), device="cuda")
    cnt_ref = torch.empty(k, dtype=torch.int32, device="cuda")
    cnt_new = torch.empty(k, dtype=torch.int32, device="cuda")
    s_ref = torch.empty(1, dtype=torch.float64, device="cuda")
    s_new = torch.empty(1, dtype=torch.float64, device="cuda")
    G.update_step(X, L, k, C_ref, counts=cnt_ref, sum_d2=s_ref)
    rc = _noalloc(G, X, L, k, C_new, cnt_new, s_new)
    assert rc == G.GK_OK, G.load().gk_last_error()
    torch.cuda.synchronize()
    assert torch.equal(cnt_new, cnt_ref) and int(cnt_new.sum()) == n
    assert torch.equal(C_new, C_ref)
    P.check_rel(s_new.item(), s_ref.item(), what="n x distortion")


def test_noalloc_bad_labels_leave_the_other_clusters_exact(G):
    """Samples whose label is outside [0, k) belong to no cluster: every cluster's centroid, size and distortion
    term equal the update of the valid samples alone (members keep their order, so bit for bit)."""
    n, d, k = 50_000, 24, 700
    g = np.random.default_rng(9)
    Xh = g.standard_normal((n, d)).astype(np.float32)
    Lh = g.integers(0, k, n).astype(np.int32)
    bad = g.choice(n, 37, replace=False)
    Lh[bad[:20]] = k + g.integers(0, 5000, 20)
    Lh[bad[20:]] = -1 - g.integers(0, 5000, 17)
    ok = (Lh >= 0) & (Lh < k)
    X, L = torch.from_numpy(Xh).cuda(), torch.from_numpy(Lh).cuda()
    Xv, Lv = torch.from_numpy(np.ascontiguousarray(Xh[ok])).cuda(), torch.from_numpy(Lh[ok]).cuda()
    C0 = torch.from_numpy(g.standard_normal((k, d)).astype(np.float32)).cuda()
    for _ in range(2):  # the second call runs on the first one's leftovers
        C_ref, C_new = C0.clone(), C0.clone()
        cnt_ref = torch.empty(k, dtype=torch.int32, device="cuda")
        cnt_new = torch.empty(k, dtype=torch.int32, device="cuda")
        s_ref = torch.empty(1, dtype=torch.float64, device="cuda")
        s_new = torch.empty(1, dtype=torch.float64, device="cuda")
        G.update_step(Xv, Lv, k, C_ref, counts=cnt_ref, sum_d2=s_ref)
        rc = _noalloc(G, X, L, k, C_new, cnt_new, s_new)
        assert rc == G.GK_OK, G.load().gk_last_error()
        torch.cuda.synchronize()
        assert torch.equal(cnt_new, cnt_ref) and int(cnt_new.sum()) == int(ok.sum())
        assert torch.equal(C_new, C_ref)
        assert s_new.item() == s_ref.item()
