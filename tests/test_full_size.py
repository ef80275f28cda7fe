"""Parity at the benchmark sizes, in the launch configuration bench.py times (the step entry points on one
workspace, the precision level its tuner picks for the workload), on sampled outputs that the oracle computes
one by one: rows of the random initial graph, centroids of sampled clusters after an update, labels of sampled
samples after an assignment, and rows of sampled samples after a refinement, in the graph construction's first
round at k0 and in the fit's first iteration at k.

The samples are drawn as the bench draws them.  Host copies hold only the rows a check reads (a lazily
allocated n x d array), so the 10^7 x 512 workload needs no 20 GB host copy; the sampled assignment is checked
on an equivalent small problem (the sampled samples, their candidate clusters renumbered in increasing order,
so that ties still go to the smaller label).  Comparison rules: tests/parity.py (integer-valued SIFT-shaped data:
graph rows bit for bit)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1705_01813_gb300 import datagen  # noqa: E402
from tests import parity as P  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [("sift_n1000000_d128_k10000", 1), ("gist_n1000000_d960_k10000", 1), ("deep_n10000000_d512_k1000000", 2)]
M = 48  # sampled samples (and clusters) per check


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01813_gb300 import gkm
    gkm.load()
    return gkm


def _device_samples(w):
    if w.storage == "bf16":
        return datagen.deep_like_device(w.n, w.d, w.extra["n_dirs"], 50.0, w.seed, device="cuda")
    if w.name.startswith("gist"):
        return datagen.gist_like_device(w.n, w.d, w.extra.get("n_latent", 1000), w.seed, device="cuda")
    return torch.from_numpy(w.data()).cuda()


class Rows:
    """Host FP32 copy of the samples holding only the rows fetched so far (the rest reads as zeros)."""

    def __init__(self, X):
        self.X = X
        self.h = np.zeros(tuple(X.shape), np.float32)  # pages are touched only where rows are written
        self.have = np.zeros(X.shape[0], bool)

    def need(self, ids):
        ids = np.unique(np.asarray(ids, np.int64).ravel())
        ids = ids[~self.have[ids]]
        if ids.size:
            t = torch.from_numpy(ids).cuda()
            self.h[ids] = self.X[t].float().cpu().numpy()
            self.have[ids] = True
        return self.h


def _oracle_assign_sampled(xrows, own, nbl, U, C_U):
    """The oracle's assignment of the sampled samples on an equivalent small problem: sample q has the own label
    own[q] and neighbour labels nbl[q]; the candidate clusters U (ascending) are renumbered 0, 1, ... in that
    order and C_U holds their centroids.  Returns (labels, best distances)."""
    m, kappa = nbl.shape
    remap = {int(u): t for t, u in enumerate(U)}
    Xs = np.zeros((m + m * kappa, xrows.shape[1]), np.float32)
    Xs[:m] = xrows
    Gs = np.zeros((m + m * kappa, kappa), np.int32)
    Gs[:m] = m + np.arange(m * kappa, dtype=np.int32).reshape(m, kappa)
    Ls = np.zeros(m + m * kappa, np.int32)
    Ls[:m] = [remap[int(v)] for v in own]
    Ls[m:] = [remap[int(v)] for v in nbl.ravel()]
    lo, best, _ = O.assign(Xs, Gs, np.asarray(C_U, np.float64), Ls, rows=np.arange(m))
    return U[lo], best


def _check_update(R, C_gpu, off, mem, clusters):
    Cg = C_gpu[torch.from_numpy(clusters).cuda().long()].cpu().numpy()
    Co = np.zeros(Cg.shape, np.float64)
    for t, r in enumerate(clusters):
        ids = mem[off[r]:off[r + 1]]
        if ids.size:
            Co[t] = O.update(R.need(ids)[ids], np.zeros(ids.size, np.int32), 1)[0][0]
    P.check_centroids(Cg, Co, off[clusters + 1] - off[clusters])


def _check_assign(R, gi, lab_in, C_gpu, lab_out, rows):
    rt = torch.from_numpy(rows).cuda().long()
    own = lab_in[rt].cpu().numpy()
    nbl = lab_in[gi[rt].long()].cpu().numpy()
    U = np.unique(np.concatenate([own, nbl.ravel()]))
    C_U = C_gpu[torch.from_numpy(U).cuda().long()].cpu().numpy()
    xrows = R.need(rows)[rows]
    lo, best = _oracle_assign_sampled(xrows, own, nbl, U, C_U)
    lg = lab_out[rt].cpu().numpy()
    pos = {int(u): t for t, u in enumerate(U)}
    for q in np.nonzero(lg != lo)[0]:  # a near tie: the GPU's label is within the tolerance of the oracle's best
        dg = ((xrows[q].astype(np.float64) - C_U[pos[int(lg[q])]].astype(np.float64)) ** 2).sum()
        assert dg <= best[q] * (1 + P.REL) + 1e-30, (rows[q], lg[q], lo[q])


@pytest.mark.parametrize("name,precision", CASES, ids=[c[0] for c in CASES])
def test_full_size_sampled_parity(G, name, precision):
    w = datagen.WORKLOADS[name]
    X = _device_samples(w)
    torch.cuda.empty_cache()
    n, d, kappa, k0, k = w.n, w.d, w.kappa, w.k0, w.k
    exact = name.startswith("sift")
    g = np.random.default_rng(170501813)
    rows = np.unique(np.concatenate([[0, n - 1], g.integers(0, n, M)]))
    R = Rows(X)
    kmax = max(k0, k)
    ws = G.workspace(max(G.workspace_size(G.GK_OP_FIT, n, d, kmax, kappa),
                         G.workspace_size(G.GK_OP_REFINE, n, d, kmax, kappa)))
    # the random initial graph
    gi, gd = G.init_graph(X, kappa, w.seed, ws=ws)
    gi_h = gi[torch.from_numpy(rows).cuda().long()].cpu().numpy()
    R.need(np.concatenate([rows, gi_h.ravel()]))
    oi, od = O.init_graph_rows(R.h, kappa, w.seed, rows)
    P.check_graph(R.h, gi_h, gd[torch.from_numpy(rows).cuda().long()].cpu().numpy(), oi, od, rows=rows,
                  exact=exact)
    # the construction's first round at k0: update, assignment, update, refinement
    la = G.init_labels(n, k0, w.seed)
    off, mem, cnt = G.group_by_label(la, k0, ws=ws)
    C0 = torch.zeros((k0, d), device="cuda")
    G.update_from_groups(X, off, mem, k0, C0, cnt, ws=ws)
    off_h, mem_h = off.cpu().numpy(), mem.cpu().numpy()
    clusters = np.unique(g.integers(0, k0, M))
    _check_update(R, C0, off_h, mem_h, clusters)
    lb = torch.empty_like(la)
    G.assign_step(X, gi, C0, la, lb, None, None, None, precision, mem, ws=ws)
    _check_assign(R, gi, la, C0, lb, rows)
    off, mem, cnt = G.group_by_label(lb, k0, ws=ws)
    G.update_from_groups(X, off, mem, k0, C0, cnt, ws=ws)
    rt = torch.from_numpy(rows).cuda().long()
    before_i, before_d = gi[rt].cpu().numpy(), gd[rt].cpu().numpy()
    G.graph_refine_groups(X, off, mem, k0, gi, gd, w.max_cluster, precision, ws=ws)
    after_i, after_d = gi[rt].cpu().numpy(), gd[rt].cpu().numpy()
    lb_h, off_h, mem_h = lb.cpu().numpy(), off.cpu().numpy(), mem.cpu().numpy()
    run_ids = [mem_h[off_h[r]:off_h[r + 1]] for r in lb_h[rows]]
    R.need(np.concatenate([rows, before_i.ravel(), after_i.ravel()] + run_ids))
    ri, rd = O.graph_refine_rows(R.h, lb_h, k0, rows, before_i, before_d.astype(np.float64), w.max_cluster)
    P.row_invariants(R.h, after_i, after_d, rows=rows)
    P.check_graph(R.h, after_i, after_d, ri, rd, rows=rows, exact=exact)
    # the fit's first iteration at k on this graph: update and assignment
    lf = G.init_labels(n, k, w.seed + 1)
    off, mem, cnt = G.group_by_label(lf, k, ws=ws)
    C = torch.zeros((k, d), device="cuda")
    G.update_from_groups(X, off, mem, k, C, cnt, ws=ws)
    off_h, mem_h = off.cpu().numpy(), mem.cpu().numpy()
    _check_update(R, C, off_h, mem_h, np.unique(g.integers(0, k, M)))
    lg = torch.empty_like(lf)
    G.assign_step(X, gi, C, lf, lg, None, None, None, precision, mem, ws=ws)
    _check_assign(R, gi, lf, C, lg, rows)
    assert G.read_status(ws) == G.GK_OK
