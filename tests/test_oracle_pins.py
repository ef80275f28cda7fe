"""Pins of the FP64 oracle to things other than itself (CPU only).

Each check compares the oracle with a value fixed by the paper or by
mathematics: hand-worked examples (tests/golden/worked_1d.json), the published
SplitMix64 outputs (tests/golden/splitmix64.json), special cases that reduce to
textbook routines (a complete graph makes the graph-guided assignment
exhaustive Lloyd; k0 = 1 makes Alg. 3 an exact KNN search), closed forms (the
Eq. 2 identity n E = sum ||x||^2 - I; the assignment's near-tie margin as the
gap of the two smallest entries of the full distance table), and invariants (non-increasing
distortion, sorted duplicate-free graph rows, result-neutral visited set).
The two-means tree (Alg. 1) is pinned by the cluster sizes that n and k alone
fix, by one-dimensional data (every cluster a run of consecutive values), by
its root split against textbook 2-means followed by a median split, and by
separated blobs.  The boost form (Eq. 3 gains, Alg. 2's move step) is pinned by
hand-worked moves, ties and singletons (tests/golden/worked_boost.json), by
each visit checked against the k-means objective recomputed from scratch, by
its fixed FP64 summation order on vectors where the order decides the
rounding, and by the Eq. 2 identity over a whole epoch.

The second half plants plausible mistakes in a copy of the oracle's C source
and shows that at least one pin fails for each.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TAG_LABELS = 0x4C41424C00000000
TAG_GRAPH = 0x4752415000000000
TAG_TREE = 0x5452454500000000


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _col(x):
    return np.asarray(x, np.float32).reshape(-1, 1)


def _blobs(n, d, centers, seed, spread=0.6):
    g = np.random.default_rng(seed)
    c = g.uniform(-5, 5, size=(centers, d))
    z = g.integers(0, centers, n)
    return (c[z] + spread * g.standard_normal((n, d))).astype(np.float32)


def _np_means(X, L, k, C_old):
    X64 = X.astype(np.float64)
    S = np.zeros((k, X.shape[1]))
    np.add.at(S, L, X64)
    cnt = np.bincount(L, minlength=k)
    C = C_old.copy()
    nz = cnt > 0
    C[nz] = S[nz] / cnt[nz, None]
    return C, cnt


def _np_d2(X, C):
    X64 = X.astype(np.float64)
    return ((X64[:, None, :] - np.asarray(C, np.float64)[None, :, :]) ** 2).sum(-1)


# ---------------------------------------------------------------- checks ----

def check_splitmix(orc):
    g = _golden("splitmix64.json")
    assert orc.splitmix64_stream(1234567, 5) == [int(v) for v in g["seed_1234567_first5"]]
    assert orc.splitmix64_stream(0, 1)[0] == int(g["seed_0_first"])
    # the counter form used for the seeded start is output c+1 of the published generator
    for key in (0, 1234567, 0xDEADBEEF ^ TAG_LABELS):
        seq = orc.splitmix64_stream(key, 40)
        assert [orc.draw(key, c) for c in range(40)] == seq


def check_init_labels(orc):
    n, k, seed = 5000, 37, 99
    L = orc.init_labels(n, k, seed)
    seq = orc.splitmix64_stream(seed ^ TAG_LABELS, n)
    assert np.array_equal(L, np.array([v % k for v in seq], np.int32))
    cnt = np.bincount(L, minlength=k)
    chi2 = ((cnt - n / k) ** 2 / (n / k)).sum()
    assert chi2 < 3 * k  # roughly uniform


def check_init_graph(orc):
    X = _blobs(300, 5, 4, 3)
    n, kappa, seed = X.shape[0], 7, 11
    gi, gd = orc.init_graph(X, kappa, seed)
    full = _np_d2(X, X)
    key = seed ^ TAG_GRAPH
    for i in range(n):
        row = gi[i]
        assert i not in row and len(set(row.tolist())) == kappa
        assert np.array_equal(gd[i], full[i, row])
        keys = list(zip(gd[i].tolist(), row.tolist()))
        assert keys == sorted(keys)
        # the set follows the rejection rule over the published generator's outputs
        want, a = [], 0
        while len(want) < kappa:
            j = orc.draw(key, (i << 32) | a) % n
            a += 1
            if j != i and j not in want:
                want.append(j)
        assert sorted(want) == sorted(row.tolist())


def check_worked_assign(orc):
    g = _golden("worked_1d.json")
    a = g["assign"]
    X = _col(a["x"])
    C, cnt, E, _ = orc.update(X, a["labels"], a["k"])
    assert np.allclose(C, a["centroids_before"], rtol=0, atol=1e-15)
    assert E == pytest.approx(a["distortion_before"], rel=1e-15)
    Lo, best, uniq = orc.assign(X, a["graph"], C, a["labels"])
    assert Lo.tolist() == a["labels_after_assign"]
    assert np.allclose(best, a["best_d2"], rtol=0, atol=1e-15)
    assert uniq.tolist() == a["uniq"]
    assert best.mean() == pytest.approx(a["distortion_after_assign"], rel=1e-15)
    C2, _, E2, _ = orc.update(X, Lo, a["k"], C)
    assert np.allclose(C2, a["centroids_after_update"], rtol=0, atol=1e-15)
    assert E2 == pytest.approx(a["distortion_after_update"], rel=1e-15)
    for case in ("own_label", "tie"):
        c = g[case]
        Lo, _, _ = orc.assign(_col(c["x"]), c["graph"], c["centroids"], c["labels"])
        assert Lo.tolist() == c["labels_after_assign"], case


def check_worked_margin(orc):
    g = _golden("worked_1d.json")["margin"]
    m = orc.assign_margin(_col(g["x"]), np.asarray(g["graph"]), np.asarray(g["centroids"]), np.asarray(g["labels"]))
    assert np.array_equal(m, np.asarray([float(v) for v in g["margin"]]))


def check_margin_complete_graph(orc):
    """With every cluster a candidate, the margin is the relative gap of the two smallest entries of each row of
    the full distance table (numpy sort): the textbook second-nearest-centroid gap."""
    g = np.random.default_rng(21)
    n, d, k = 300, 5, 7
    X = g.standard_normal((n, d)).astype(np.float32)
    L = g.permutation(np.arange(n) % k).astype(np.int32)
    members = [np.nonzero(L == r)[0][0] for r in range(k)]
    G = np.tile(np.asarray(members, np.int32), (n, 1))
    C = g.standard_normal((k, d))
    D = np.sort(_np_d2(X, C), axis=1)
    want = (D[:, 1] - D[:, 0]) / D[:, 0]
    got = orc.assign_margin(X, G, C, L)
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    # and a sample's assigned cluster is its nearest one whenever its margin is positive
    Lo, _, _ = orc.assign(X, G, C, L)
    pos = got > 0
    assert np.array_equal(Lo[pos], np.argmin(_np_d2(X, C), 1)[pos])


def check_assign_complete_graph(orc):
    X = _blobs(60, 3, 5, 5)
    n, k = X.shape[0], 7
    g = np.random.default_rng(1)
    L = g.permutation(np.arange(n) % k).astype(np.int32)
    C, _, _, _ = orc.update(X, L, k)
    G = np.array([[j for j in range(n) if j != i] for i in range(n)], np.int32)
    Lg, bg, uq = orc.assign(X, G, C, L)
    Le, be = orc.assign_exhaustive(X, C)
    D = _np_d2(X, C)
    assert np.array_equal(Lg, Le)
    assert np.array_equal(Le, D.argmin(1).astype(np.int32))  # argmin: first (smaller) label on ties
    assert np.allclose(be, D.min(1), rtol=1e-14, atol=0)
    assert np.array_equal(bg, be)
    assert (uq == k).all()


def check_assign_restricted(orc):
    """With a sparse graph only the own and the neighbours' clusters are candidates."""
    X = _blobs(200, 4, 6, 7)
    n, k, kappa = X.shape[0], 12, 3
    g = np.random.default_rng(2)
    L = g.integers(0, k, n).astype(np.int32)
    C, _, E0, _ = orc.update(X, L, k)
    G = np.stack([g.choice(np.delete(np.arange(n), i), kappa, replace=False) for i in range(n)]).astype(np.int32)
    Lo, best, uq = orc.assign(X, G, C, L)
    D = _np_d2(X, C)
    for i in range(n):
        Q = sorted(set([L[i]] + [L[j] for j in G[i]]))
        assert uq[i] == len(Q)
        sub = D[i, Q]
        assert Lo[i] == Q[int(np.argmin(sub))]
        assert best[i] == pytest.approx(sub.min(), rel=1e-14)
    # own label among the candidates: the assignment never raises the distortion
    assert best.mean() <= E0 * (1 + 1e-15)


def check_update(orc):
    X = _blobs(500, 6, 5, 9)
    n, k = X.shape[0], 9
    g = np.random.default_rng(3)
    L = g.integers(0, k - 2, n).astype(np.int32)  # clusters k-2, k-1 empty
    C_old = g.standard_normal((k, X.shape[1]))
    C, cnt, E, I = orc.update(X, L, k, C_old)
    Cn, cn = _np_means(X, L, k, C_old)
    assert np.array_equal(cnt, cn)
    assert np.allclose(C, Cn, rtol=1e-13, atol=1e-13)
    assert np.array_equal(C[k - 2:], C_old[k - 2:])  # empty clusters keep their centroid
    direct = ((X.astype(np.float64) - C[L]) ** 2).sum(1).mean()
    assert E == pytest.approx(direct, rel=1e-12)
    # Eq. 2: with exact means n E = sum ||x||^2 - sum_r D_r'D_r / n_r
    sx = (X.astype(np.float64) ** 2).sum()
    assert n * E == pytest.approx(sx - I, rel=1e-9)


def _np_lloyd(X, L, k, iters):
    C = np.zeros((k, X.shape[1]))
    C, _ = _np_means(X, L, k, C)
    for _ in range(iters):
        L = _np_d2(X, C).argmin(1)
        C, _ = _np_means(X, L, k, C)
    return L.astype(np.int32), C


def check_fit(orc):
    X = _blobs(80, 2, 4, 13)
    n, k, T = X.shape[0], 6, 5
    L0 = orc.init_labels(n, k, 4)
    G = np.array([[j for j in range(n) if j != i] for i in range(n)], np.int32)
    L, C, cnt, E = orc.fit(X, k, G, T, L0)
    Ln, Cn = _np_lloyd(X, L0, k, T)
    assert np.array_equal(L, Ln)
    assert np.allclose(C[cnt > 0], Cn[cnt > 0], rtol=1e-12, atol=1e-12)
    assert (np.diff(E) <= 1e-12 * E[:-1]).all()
    # a sparse graph: still non-increasing at every half step
    Xb = _blobs(1500, 8, 30, 14)
    Gb, _ = orc.brute_knn(Xb, 6)
    L0b = orc.init_labels(Xb.shape[0], 40, 5)
    _, _, _, Eb = orc.fit(Xb, 40, Gb, 6, L0b)
    assert (np.diff(Eb) <= 1e-12 * Eb[:-1]).all()


def check_worked_refine(orc):
    r = _golden("worked_1d.json")["refine"]
    X = _col(r["x"])
    for cap, key in ((128, "cap128"), (2, "cap2")):
        gi, gd = orc.graph_refine(X, r["labels"], r["k"], r["graph_idx"], r["graph_dist"], cap)
        assert gi.tolist() == r[key + "_idx"], cap
        assert gd.tolist() == [[float(v) for v in row] for row in r[key + "_dist"]], cap


def _np_knn(X, kappa):
    D = _np_d2(X, X)
    n = X.shape[0]
    idx = np.empty((n, kappa), np.int32)
    for i in range(n):
        js = np.array([j for j in range(n) if j != i])
        order = np.lexsort((js, D[i, js]))[:kappa]
        idx[i] = js[order]
    return idx, np.take_along_axis(D, idx.astype(np.int64), 1)


def check_exact_knn_special_case(orc):
    X = _blobs(90, 4, 3, 21)
    X[10] = X[3]  # an exact tie in distance
    kappa = 8
    bi, bd = orc.brute_knn(X, kappa)
    ni, nd = _np_knn(X, kappa)
    assert np.array_equal(bi, ni) and np.allclose(bd, nd, rtol=1e-14, atol=0)
    # n < 2 xi gives k0 = 1: one cluster, one round of exhaustive pairs = exact KNN
    gi, gd, L, _ = orc.build_graph(X, kappa, xi=50, tau=1, max_cluster=128, seed=3)
    assert (L == 0).all()
    assert np.array_equal(gi, bi) and np.array_equal(gd, bd)


def _row_invariants(X, gi, gd):
    n, kappa = gi.shape
    full = _np_d2(X, X)
    for i in range(n):
        row = gi[i].tolist()
        assert i not in row and len(set(row)) == kappa
        keys = list(zip(gd[i].tolist(), row))
        assert keys == sorted(keys)
        assert np.allclose(gd[i], full[i, gi[i]], rtol=1e-14, atol=0)


def check_graph_invariants_and_monotone(orc):
    X = _blobs(700, 8, 12, 31)
    kappa, xi = 10, 50
    prev = None
    bi, _ = orc.brute_knn(X, 1)
    rec = []
    for tau in range(0, 5):
        gi, gd, _, E = orc.build_graph(X, kappa, xi=xi, tau=tau, max_cluster=128, seed=8)
        _row_invariants(X, gi, gd)
        if prev is not None:
            # the kappa-th and top-1 keys only ever improve from round to round
            assert (gd[:, -1] <= prev[1][:, -1]).all()
            assert (gd[:, 0] <= prev[1][:, 0]).all()
        rec.append(float((gi[:, 0] == bi[:, 0]).mean()))
        prev = (gi, gd)
    assert all(b >= a for a, b in zip(rec, rec[1:]))
    assert rec[-1] > rec[0]


def check_visited_neutral(orc):
    X = _blobs(400, 6, 8, 41)
    a = orc.build_graph(X, 9, xi=40, tau=4, max_cluster=32, seed=5, use_visited=False)
    b = orc.build_graph(X, 9, xi=40, tau=4, max_cluster=32, seed=5, use_visited=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def check_refine_rows_and_chunks(orc):
    X = _blobs(900, 5, 10, 51)
    n, k, kappa, cap = X.shape[0], 6, 6, 40  # clusters of ~150 cut into runs of <= 40
    g = np.random.default_rng(6)
    L = g.integers(0, k, n).astype(np.int32)
    gi0, gd0 = orc.init_graph(X, kappa, 77)
    gi, gd = orc.graph_refine(X, L, k, gi0, gd0, cap)
    rows = g.choice(n, 50, replace=False)
    ri, rd = orc.graph_refine_rows(X, L, k, rows, gi0[rows], gd0[rows], cap)
    assert np.array_equal(ri, gi[rows]) and np.array_equal(rd, gd[rows])
    # every new neighbour comes from the row's own run of its cluster
    off, mem = orc.group_csr(L, k)
    run_of = np.empty(n, np.int64)
    for r in range(k):
        m = off[r + 1] - off[r]
        nc = -(-m // cap)
        base, rem = m // nc, m % nc
        for c in range(nc):
            s0 = c * base + min(c, rem)
            sz = base + (1 if c < rem else 0)
            assert sz <= cap and sz >= base
            run_of[mem[off[r] + s0: off[r] + s0 + sz]] = r * 100000 + c
    for i in range(n):
        for j in set(gi[i].tolist()) - set(gi0[i].tolist()):
            assert run_of[j] == run_of[i]


def check_init_graph_rows(orc):
    # the row-restricted form (for spot checks at full size) gives the full construction's rows
    X = _blobs(500, 6, 5, 13)
    gi, gd = orc.init_graph(X, 9, 21)
    rows = [0, 499, 7, 250, 7]
    ri, rd = orc.init_graph_rows(X, 9, 21, rows)
    assert np.array_equal(ri, gi[rows]) and np.array_equal(rd, gd[rows])


def check_group_csr(orc):
    g = np.random.default_rng(8)
    L = g.integers(0, 50, 3000).astype(np.int32)
    off, mem = orc.group_csr(L, 53)
    assert np.array_equal(mem, np.argsort(L, kind="stable").astype(np.int32))
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(L, minlength=53))]))


# Alg. 1 (two-means tree).  Cluster sizes depend on n and k only: every split halves a cluster (u the larger
# half), whole levels of the tree are split before the next one starts, and a partial last level splits its
# largest clusters first, leftmost first among equal sizes.
def _tree_sizes(n, k):
    sizes = [n]
    while 2 * len(sizes) <= k:
        sizes = [h for m in sizes for h in ((m + 1) // 2, m // 2)]
    picked = set(sorted(range(len(sizes)), key=lambda j: (-sizes[j], j))[:k - len(sizes)])
    out = []
    for j, m in enumerate(sizes):
        out += [(m + 1) // 2, m // 2] if j in picked else [m]
    return out


def check_tree_sizes(orc):
    g = np.random.default_rng(11)
    sweep = [(int(n), int(g.integers(1, n + 1))) for n in g.integers(2, 300, 60)]
    for n, k in [(1000, 7), (10, 6), (10, 7), (37, 37), (64, 1), (100, 3), (1001, 12), (5, 4), (7, 5), (6, 5)] + sweep:
        X = g.standard_normal((n, 3)).astype(np.float32)
        L = orc.two_means_tree(X, k, iters=2, seed=n + k)
        assert L.min() == 0 and L.max() == k - 1
        assert np.bincount(L, minlength=k).tolist() == _tree_sizes(n, k), (n, k)


def check_tree_1d(orc):
    # d = 1: d(x, c_u) - d(x, c_v) is linear in x, so every bisection splits the sorted values at their middle and
    # every cluster is a run of consecutive values (distinct integers: no rounding ties)
    g = np.random.default_rng(12)
    x = g.permutation(997).astype(np.float32)
    for k, iters in [(2, 0), (5, 1), (16, 3), (50, 2)]:
        L = orc.two_means_tree(_col(x), k, iters=iters, seed=k)
        runs = L[np.argsort(x)]
        assert (np.diff(runs) != 0).sum() == k - 1, (k, iters)


def _tree_seeds(orc, ids, depth, seed):
    h = [(orc.draw(seed ^ TAG_TREE, (depth << 32) | int(i)), int(i)) for i in ids]
    (_, a), (_, b) = sorted(h)[:2]
    return a, b


def check_tree_root_split(orc):
    # k = 2 is one bisection: Lloyd's 2-means (textbook numpy, FP64) from the seed pair, then the ceil(n/2) members
    # with the smallest d(x, c_u) - d(x, c_v) (ties by id) form cluster 0
    g = np.random.default_rng(13)
    for n, d, iters, seed in [(301, 5, 0, 1), (301, 5, 1, 2), (400, 2, 3, 3), (257, 7, 4, 4)]:
        X = (g.standard_normal((n, d)) + 3 * (g.random((n, 1)) < 0.3)).astype(np.float32)
        a, b = _tree_seeds(orc, range(n), 0, seed)
        C = X[[a, b]].astype(np.float64)
        for _ in range(iters):
            D = _np_d2(X, C)
            C, _ = _np_means(X, (D[:, 1] < D[:, 0]).astype(np.int64), 2, C)
        D = _np_d2(X, C)
        order = np.lexsort((np.arange(n), D[:, 0] - D[:, 1]))
        want = np.ones(n, np.int32)
        want[order[:(n + 1) // 2]] = 0
        assert np.array_equal(orc.two_means_tree(X, 2, iters=iters, seed=seed), want), (n, iters)
        # k = 3 splits the larger (left) half of that same root split further
        L3 = orc.two_means_tree(X, 3, iters=iters, seed=seed)
        assert np.array_equal(L3 == 2, want == 1)


def _np_tree(orc, X, k, iters, seed):
    """Alg. 1 restated with every decision in FP64 (numpy): pop the largest cluster (shallowest, then leftmost),
    seeds by the tree's draw, `iters` Lloyd 2-means passes with FP64 means (an empty half keeps its centre), then
    the ceil(m/2) members of smallest (d(x, c_u) - d(x, c_v), id) form u.  Returns the labels (leaves numbered left
    to right) and the smallest relative margin of any of its decisions (Lloyd side choices and the split
    boundaries): above the FP32 oracle's rounding, the two must take every decision alike."""
    X64 = X.astype(np.float64)
    leaves = [(np.arange(X.shape[0]), 0)]
    margin = np.inf
    while len(leaves) < k:
        j = max(range(len(leaves)), key=lambda q: (len(leaves[q][0]), -leaves[q][1], -q))
        ids, depth = leaves[j]
        a, b = _tree_seeds(orc, ids, depth, seed)
        C = X64[[a, b]]
        Y = X64[ids]
        for _ in range(iters):
            D = _np_d2(Y, C)
            margin = min(margin, float(np.min(np.abs(D[:, 0] - D[:, 1]) / (D[:, 0] + D[:, 1] + 1e-300))))
            C, _ = _np_means(Y, (D[:, 1] < D[:, 0]).astype(np.int64), 2, C)
        D = _np_d2(Y, C)
        key = D[:, 0] - D[:, 1]
        order = np.lexsort((ids, key))
        h = (len(ids) + 1) // 2
        if 0 < h < len(ids):
            ks = key[order]
            margin = min(margin, float((ks[h] - ks[h - 1]) / (np.abs(D).max() + 1e-300)))
        u, v = np.sort(ids[order[:h]]), np.sort(ids[order[h:]])
        leaves[j:j + 1] = [(u, depth + 1), (v, depth + 1)]
    L = np.empty(X.shape[0], np.int32)
    for c, (ids, _) in enumerate(leaves):
        L[ids] = c
    return L, margin


def _partition_sse(X, L, k):
    C, _ = _np_means(X, L, k, np.zeros((k, X.shape[1])))
    return float(((X.astype(np.float64) - C[L]) ** 2).sum())


def check_tree_fp64_decisions(orc):
    # the FP32-decision oracle (reading T3) against the same algorithm deciding in FP64: where no FP64 decision
    # lies within 1e-4 (relative) of its threshold the labels are equal; otherwise the partition's quality is
    # close to it (uniform samples, many clusters: margins down to about 1e-6) in its labels and distortion
    g = np.random.default_rng(15)
    exact = 0
    cases = [(200, 3, 5, 0, 1), (200, 3, 5, 2, 2), (333, 6, 9, 1, 3), (150, 2, 16, 3, 4), (400, 8, 7, 2, 5),
             (120, 4, 30, 1, 6), (600, 5, 12, 2, 7), (2000, 2, 40, 2, 8), (3000, 1, 50, 1, 9), (1500, 3, 60, 3, 10)]
    for q, (n, d, k, iters, seed) in enumerate(cases):
        if q < 7:
            X = (g.uniform(-5, 5, (6, d))[g.integers(0, 6, n)] + g.standard_normal((n, d))).astype(np.float32)
        else:
            X = g.uniform(-1, 1, (n, d)).astype(np.float32)
        want, margin = _np_tree(orc, X, k, iters, seed)
        got = orc.two_means_tree(X, k, iters=iters, seed=seed)
        assert np.bincount(got, minlength=k).tolist() == np.bincount(want, minlength=k).tolist()
        if margin > 1e-4:
            assert np.array_equal(got, want), (n, d, k, iters, margin)
            exact += 1
        else:
            assert (got == want).mean() >= 0.95, (n, d, k, iters, margin)
            e64, e32 = _partition_sse(X, want, k), _partition_sse(X, got, k)
            assert abs(e32 - e64) <= 1e-3 * e64, (e32, e64)
    assert exact >= 3  # most cases decide with a margin: the equality above is exercised


def check_tree_blobs(orc):
    # 8 tight, well separated blobs of 64 samples: the equal-size splits fall between blobs, one blob per cluster
    g = np.random.default_rng(14)
    c = g.uniform(-10, 10, (8, 4))
    z = np.repeat(np.arange(8), 64)
    X = (c[z] + 0.01 * g.standard_normal((512, 4))).astype(np.float32)
    L = orc.two_means_tree(X, 8, iters=5, seed=5)
    for b in range(8):
        assert len(set(L[z == b].tolist())) == 1
    assert len(set(L.tolist())) == 8



# ------------------------------------------------------------- boost form ----

def check_boost_fold(orc):
    """The boost form's FP64 squared norm: hand-worked halving folds that a running sum or adjacent pairs get
    wrong, and exact integer sums at lengths that are not powers of two."""
    f = _golden("worked_boost.json")["fold"]
    for v, want in zip(f["vectors"], f["values"]):
        assert orc.fold_sq(np.asarray(v, np.float64)) == want
    rng = np.random.default_rng(3)
    for d in (1, 2, 3, 17, 100, 129):
        v = rng.integers(-1000, 1000, d)
        assert orc.fold_sq(v.astype(np.float64)) == float(sum(int(a) * int(a) for a in v))


def _boost_run(orc, case):
    X = _col(case["x"])
    D, cnt, S = orc.boost_init(X, case["labels"], case["k"])
    return (D, cnt, S) + orc.boost_epoch(X, case["graph"], case["order"], case["labels"], case["k"], D, cnt, S)


def check_boost_worked(orc):
    g = _golden("worked_boost.json")
    D0, c0, S0, L, D, cnt, S, moves, gains = _boost_run(orc, g["move"])
    m = g["move"]
    assert D0.tolist() == m["D_before"] and c0.tolist() == m["counts_before"] and S0.tolist() == m["S_before"]
    assert L.tolist() == m["labels_after"] and D.tolist() == m["D_after"]
    assert cnt.tolist() == m["counts_after"] and S.tolist() == m["S_after"]
    assert gains.tolist() == m["gains"] and moves == m["moves"]
    t = g["tie"]
    _, _, _, L, D, cnt, S, moves, _ = _boost_run(orc, t)
    assert L.tolist() == t["labels_after"] and D.tolist() == t["D_after"]
    assert cnt.tolist() == t["counts_after"] and S.tolist() == t["S_after"] and moves == t["moves"]
    s1 = g["singleton"]
    _, _, _, L, _, _, _, moves, _ = _boost_run(orc, s1)
    assert L.tolist() == s1["labels_after"] and moves == s1["moves"]


def _sse(X, L, k):
    """k-means objective by brute force: sum of squared distances to the member means (Eq. 1)."""
    X = X.astype(np.float64)
    cnt = np.bincount(L, minlength=k).astype(np.float64)
    C = np.zeros((k, X.shape[1]))
    np.add.at(C, L, X)
    C[cnt > 0] /= cnt[cnt > 0, None]
    return float(((X - C[L]) ** 2).sum())


def check_boost_brute_force(orc):
    """Each visit of the move step, checked against the k-means objective computed from scratch: a move lowers
    the sum of squared errors by exactly its gain (Eq. 2: n E = sum ||x||^2 - I) and goes to the candidate cluster
    of lowest objective; a sample that stays has no candidate that would lower it (or is alone)."""
    rng = np.random.default_rng(7)
    for n, d, k, kappa in ((40, 3, 5, 4), (60, 2, 8, 6), (30, 5, 3, 29)):
        X = rng.integers(-20, 21, (n, d)).astype(np.float32)
        L = rng.integers(0, k, n).astype(np.int32)
        L[:k] = np.arange(k)
        G = np.stack([rng.choice(np.delete(np.arange(n), i), kappa, replace=False) for i in range(n)])
        D, cnt, S = orc.boost_init(X, L, k)
        order = rng.integers(0, n, 3 * n)
        moved = 0
        for i in order:
            before = _sse(X, L, k)
            u = L[i]
            Q = sorted(set(L[G[i]].tolist()) - {u})
            L2, D, cnt, S, mv, gains = orc.boost_epoch(X, G, [i], L, k, D, cnt, S)
            alt = {v: _sse(X, np.where(np.arange(n) == i, v, L), k) for v in Q}
            if mv:
                v = int(L2[i])
                assert v in Q and np.bincount(L, minlength=k)[u] >= 2
                assert gains[0] > 0
                assert before - alt[v] == pytest.approx(gains[0], rel=1e-9, abs=1e-9)
                assert alt[v] <= min(alt.values()) + 1e-9 * max(1.0, before)
                moved += 1
            else:
                assert np.array_equal(L2, L)
                if np.bincount(L, minlength=k)[u] >= 2 and Q:
                    assert min(alt.values()) >= before - 1e-9 * max(1.0, before)
            L = L2
            D0, c0, S0 = orc.boost_init(X, L, k)  # integer data: every sum is exact in any order
            assert np.array_equal(D, D0) and np.array_equal(cnt, c0) and np.array_equal(S, S0)
        assert moved > 0


def check_boost_epoch_invariants(orc):
    """A whole epoch over a permutation on clustered data: the objective I (Eq. 2) rises by the sum of the
    gains, the state matches the Eq. 2 state of the final labels, and the distortion falls."""
    from paper_1705_01813_gb300 import datagen
    X = datagen.sift_like(2000, 16, 40, seed=5)
    k = 40
    gi, _ = orc.brute_knn(X, 10)
    L = orc.init_labels(2000, k, 9)
    D, cnt, S = orc.boost_init(X, L, k)
    I0 = float((S / cnt).sum())
    order = np.random.default_rng(1).permutation(2000)
    L2, D2, cnt2, S2, mv, gains = orc.boost_epoch(X, gi, order, L, k, D, cnt, S)
    I1 = float((S2 / cnt2).sum())
    assert mv > 100 and (gains >= 0).all() and (gains > 0).sum() == mv
    assert I1 - I0 == pytest.approx(gains.sum(), rel=1e-9)
    D3, cnt3, S3 = orc.boost_init(X, L2, k)
    assert np.array_equal(cnt2, cnt3)
    assert np.allclose(D2, D3, rtol=1e-12, atol=1e-9) and np.allclose(S2, S3, rtol=1e-12)
    assert _sse(X, L2, k) < _sse(X, L, k)
    sq = float((X.astype(np.float64) ** 2).sum())
    assert (sq - I1) == pytest.approx(_sse(X, L2, k), rel=1e-9)


CHECKS = [check_splitmix, check_init_labels, check_init_graph, check_worked_assign, check_worked_margin,
          check_margin_complete_graph, check_assign_complete_graph,
          check_assign_restricted, check_update, check_fit, check_worked_refine, check_exact_knn_special_case,
          check_graph_invariants_and_monotone, check_visited_neutral, check_refine_rows_and_chunks,
          check_init_graph_rows, check_group_csr, check_tree_sizes, check_tree_1d, check_tree_root_split,
          check_tree_fp64_decisions, check_tree_blobs, check_boost_fold, check_boost_worked,
          check_boost_brute_force, check_boost_epoch_invariants]


@pytest.mark.parametrize("check", CHECKS, ids=[c.__name__ for c in CHECKS])
def test_oracle_pin(check):
    check(O.default())


def test_paper_trends():
    """Qualitative claims on synthetic data: recall rises with tau (Sec. 4.3, Fig. 3 text) and a
    sample visits fewer clusters than it has neighbours (Sec. 4.2)."""
    from paper_1705_01813_gb300 import datagen
    X = datagen.gauss_mixture(3000, 16, 40, seed=1)
    orc = O.default()
    bi, _ = orc.brute_knn(X, 1)
    r1 = (orc.build_graph(X, 10, xi=50, tau=1, seed=2)[0][:, 0] == bi[:, 0]).mean()
    gi, gd, L, E = orc.build_graph(X, 10, xi=50, tau=6, seed=2)
    r6 = (gi[:, 0] == bi[:, 0]).mean()
    assert r6 > r1 and r6 > 0.5
    k = 30
    L0 = orc.init_labels(X.shape[0], k, 3)
    Lf, C, cnt, Ef = orc.fit(X, k, gi, 5, L0)
    _, _, uq = orc.assign(X, gi, C, Lf)
    assert uq.mean() < 10
    # close to exhaustive Lloyd from the same start (Sec. 5.3: quality drops very little)
    Ln, Cn = _np_lloyd(X, L0, k, 5)
    En = ((X.astype(np.float64) - Cn[Ln]) ** 2).sum(1).mean()
    assert Ef[-1] <= En * 1.05
    # the two-means tree as the initial partition (Alg. 2 starts from it, Sec. 4.2): the fit on the graph ends
    # lower than from random labels
    Lt = orc.two_means_tree(X, k, iters=2, seed=3)
    _, _, _, Et = orc.fit(X, k, gi, 5, Lt)
    assert Et[-1] < Ef[-1]


def _boost_windows(orc, X, G, order, L0, k, rng, rule=True):
    """The speculative schedule of the GPU epoch, restated on the oracle: every visit of a window is decided
    against the state at the window's start; the window commits, in order, up to the first visit that depends on
    an earlier visit of the window that would move (its sample or a neighbour is that visit's sample, or its own
    cluster or a candidate is one that visit leaves or joins; with rule=False whole windows commit). Returns the
    number of committed visits whose speculative decision differs from the sequential walk's."""
    D, cnt, S = orc.boost_init(X, L0, k)
    L, s, wrong = L0.copy(), 0, 0
    while s < len(order):
        win = order[s:s + int(rng.integers(1, 33))]
        moving, spec, first = [], [], len(win)
        for p_, i in enumerate(win):
            u = int(L[i])
            items_s, items_c = {int(i)} | set(G[i].tolist()), {u} | (set(L[G[i]].tolist()) - {u})
            if rule and any(mi in items_s or mu in items_c or mv in items_c for mi, mu, mv in moving):
                first = p_
                break
            v = int(orc.boost_epoch(X, G, [i], L, k, D, cnt, S)[0][i])  # against the window's start state
            spec.append(v)
            if v != u:
                moving.append((int(i), u, v))
        for p_ in range(first):  # the sequential walk over the committed visits, one visit at a time
            L, D, cnt, S = orc.boost_epoch(X, G, win[p_:p_ + 1], L, k, D, cnt, S)[:4]
            wrong += int(L[win[p_]]) != spec[p_]
        s += first
    return wrong


def test_boost_window_commit_rule_matches_sequential_decisions():
    """Every visit the GPU epoch's window schedule commits was decided on exactly the state the sequential walk
    gives it, whatever the window sizes; without the dependence rule, some speculative decisions are wrong."""
    orc = O.default()
    rng = np.random.default_rng(4)
    wrong_without = 0
    for n, d, k, kappa in ((300, 3, 12, 6), (200, 2, 40, 5)):
        X = rng.integers(-30, 31, (n, d)).astype(np.float32)
        L0 = rng.integers(0, k, n).astype(np.int32)
        L0[:k] = np.arange(k)
        G = np.stack([rng.choice(np.delete(np.arange(n), i), kappa, replace=False) for i in range(n)]).astype(np.int32)
        order = rng.integers(0, n, 3 * n).astype(np.int32)
        assert _boost_windows(orc, X, G, order, L0, k, np.random.default_rng(1)) == 0
        wrong_without += _boost_windows(orc, X, G, order, L0, k, np.random.default_rng(1), rule=False)
    assert wrong_without > 0

# ------------------------------------------------------- planted mistakes ----

MUTANTS = [
    ("own_label_dropped", "Q[u++] = L_in[i];", "(void)0;", check_worked_assign),
    ("tie_to_larger", "(da == db && ia < ib)", "(da == db && ia > ib)", check_worked_assign),
    ("distance_sign", "double diff = (double)a[t] - c[t];", "double diff = (double)a[t] + c[t];",
     check_worked_assign),
    ("empty_cluster_zeroed", "        if (counts[r] == 0)\n            continue;\n        double dd = 0.0;",
     "        if (counts[r] == 0) {\n            for (int64_t t = 0; t < d; t++) C[(int64_t)r * d + t] = 0.0;\n"
     "            continue;\n        }\n        double dd = 0.0;", check_update),
    ("I_without_division", "I += dd / (double)counts[r];", "I += dd;", check_update),
    ("merge_without_dedupe", "        if (row[q] == j)\n            return;", "        if (0)\n            return;",
     check_worked_refine),
    ("run_start_wrong", "*start = c * base + (c < rem ? c : rem);", "*start = c * base;",
     check_refine_rows_and_chunks),
    ("knn_self_allowed", "            if (j == i)\n                continue;\n            double dist = or_d2_ff(X + i * ld",
     "            double dist = or_d2_ff(X + i * ld", check_exact_knn_special_case),
    ("init_graph_self_allowed", "            if (j == i)\n                continue;\n            int dup = 0;",
     "            int dup = 0;", check_init_graph),
    ("graph_seed_reused", "uint64_t key = seed ^ OR_TAG_GRAPH;", "uint64_t key = seed ^ OR_TAG_LABELS;",
     check_init_graph),
    ("tree_half_floor", "int64_t h = (m + 1) / 2;\n    for (int64_t p = 0; p < m; p++)",
     "int64_t h = m / 2;\n    for (int64_t p = 0; p < m; p++)", check_tree_root_split),
    ("tree_key_sign", "keys[p].key = or_d2_f32(x, cu, d) - or_d2_f32(x, cv, d);",
     "keys[p].key = or_d2_f32(x, cv, d) - or_d2_f32(x, cu, d);", check_tree_root_split),
    ("margin_runner_up_not_shifted", "                d2 = d1;\n                d1 = dd;", "                d1 = dd;",
     check_worked_margin),
    ("tree_no_iterations", "it < iters; it++", "it < 0; it++", check_tree_root_split),
    ("tree_depth_tiebreak_dropped", "(depth[r] < depth[s] ||", "(0 ||", check_tree_sizes),
    ("tree_labels_by_creation", "labels[perm[p]] = rank;", "labels[perm[p]] = s;", check_tree_sizes),
    ("tree_seed_depth_ignored", "((uint64_t)(uint32_t)depth << 32)", "((uint64_t)0 << 32)",
     check_tree_fp64_decisions),
    ("boost_u_denominator", "Du_minus_x_sq / (double)(nu - 1)", "Du_minus_x_sq / (double)nu", check_boost_worked),
    ("boost_tie_to_larger", "(g == best && v < bv)", "(g == best && v > bv)", check_boost_worked),
    ("boost_u_sign", "            Dm[t] = Dm[t] - x[t];", "            Dm[t] = Dm[t] + x[t];", check_boost_worked),
    ("boost_own_label_candidate", "int seen = v == u;", "int seen = 0;", check_boost_brute_force),
    ("boost_first_neighbour_only", "for (int32_t j = 0; j < kappa; j++) {\n            int32_t v = L[G[i * kappa + j]];",
     "for (int32_t j = 0; j < 1; j++) {\n            int32_t v = L[G[i * kappa + j]];", check_boost_brute_force),
    ("boost_fold_adjacent", "w[j] = w[j] + w[j + h];", "w[j] = w[2 * j] + w[2 * j + 1];", check_boost_fold),
    ("boost_init_skips_first", "for (int64_t i = 0; i < n; i++) { /* ascending id",
     "for (int64_t i = 1; i < n; i++) { /* ascending id", check_boost_worked),
    ("tree_v_keeps_left_range", "off[t] = off[s] + h; /* v */", "off[t] = off[s]; off[s] += m - h; /* v */",
     check_tree_1d),
]


@pytest.mark.parametrize("name,find,repl,check", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, find, repl, check):
    src = open(os.path.join(os.path.dirname(O.__file__), "gkm_oracle.c")).read()
    assert src.count(find) >= 1, name
    mut = tmp_path / f"{name}.c"
    mut.write_text(src.replace(find, repl))
    lib = O.compile_source(str(mut), str(tmp_path / f"lib{name}.so"))
    with pytest.raises(AssertionError):
        check(O.Oracle(lib))


def test_oracle_results_do_not_depend_on_threads():
    """The oracle's parallel loops write each result from one thread and keep every sum's order, so one thread and
    several give the same bits (graph, labels, centroids, distortion logs)."""
    from paper_1705_01813_gb300 import datagen
    X = datagen.sift_like(4000, 64, 40, seed=2)
    orc = O.default()
    before = orc.set_threads(0)
    out = {}
    try:
        for th in (1, 4):
            orc.set_threads(th)
            gi, gd, L, E = orc.build_graph(X, 20, xi=50, tau=4, seed=3)
            Lf, C, cnt, Ef = orc.fit(X, 40, gi, 5, orc.init_labels(4000, 40, 4))
            out[th] = (gi, gd, L, E, Lf, C, cnt, Ef)
    finally:
        orc.set_threads(before)
    assert all(np.array_equal(a, b) for a, b in zip(out[1], out[4]))
