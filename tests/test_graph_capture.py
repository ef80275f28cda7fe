"""The library's step calls can be captured into a CUDA graph: a replay gives the same graph, labels and
centroids, bit for bit, as launching the same calls one by one."""
import pytest

from paper_1705_01813_gb300 import datagen


def _steps(g, torch, X, bufs, w, precision):
    gi, gd, la, lb, off, mem, cnt, C0, s, ws = bufs
    n = X.shape[0]
    g.init_graph(X, w["kappa"], 5, gi, gd, ws=ws)
    g.init_labels(n, w["k0"], 5, out=la)
    C0.zero_()
    g.group_by_label(la, w["k0"], off, mem, cnt, ws=ws)
    g.update_from_groups(X, off, mem, w["k0"], C0, cnt, s[0:1], ws=ws)
    cur, nxt = la, lb
    for _ in range(3):
        g.assign_step(X, gi, C0, cur, nxt, None, s[1:2], None, precision, mem, ws=ws)
        g.group_by_label(nxt, w["k0"], off, mem, cnt, ws=ws)
        g.update_from_groups(X, off, mem, w["k0"], C0, cnt, s[0:1], ws=ws)
        g.graph_refine_groups(X, off, mem, w["k0"], gi, gd, 128, precision, ws=ws)
        cur, nxt = nxt, cur
    return cur


@pytest.mark.gpu
@pytest.mark.parametrize("d,precision", [(32, 0), (64, 1), (128, 1)])
def test_captured_steps_equal_launched_steps(d, precision):
    import torch

    from paper_1705_01813_gb300 import gkm
    n, kappa, k0 = 12007, 16, 240
    X = torch.from_numpy(datagen.gauss_mixture(n, d, 60, seed=d)).cuda()
    dev = X.device
    i32, f32 = torch.int32, torch.float32

    def alloc():
        ws = gkm.Workspace(max(gkm.workspace_size(gkm.GK_OP_FIT, n, d, k0, kappa),
                               gkm.workspace_size(gkm.GK_OP_REFINE, n, d, k0, kappa)), dev)
        return (torch.empty((n, kappa), dtype=i32, device=dev), torch.empty((n, kappa), dtype=f32, device=dev),
                torch.empty(n, dtype=i32, device=dev), torch.empty(n, dtype=i32, device=dev),
                torch.empty(k0 + 1, dtype=i32, device=dev), torch.empty(n, dtype=i32, device=dev),
                torch.empty(k0, dtype=i32, device=dev), torch.empty((k0, d), dtype=f32, device=dev),
                torch.empty(2, dtype=torch.float64, device=dev), ws)

    w = {"kappa": kappa, "k0": k0}
    a = alloc()
    la = _steps(gkm, torch, X, a, w, precision)
    torch.cuda.synchronize()
    b = alloc()
    _steps(gkm, torch, X, b, w, precision)  # warm-up outside the capture
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        lb = _steps(gkm, torch, X, b, w, precision)
    for q in (0, 1, 5):  # scribble over the outputs, then replay
        b[q].fill_(-7)
    graph.replay()
    torch.cuda.synchronize()
    assert gkm.read_status(a[-1]) == gkm.GK_OK and gkm.read_status(b[-1]) == gkm.GK_OK
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])  # graph
    assert torch.equal(la, lb) and torch.equal(a[7], b[7])      # labels, centroids
