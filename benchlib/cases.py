"""Workloads behind the kernel-counter summaries in profiles/: each case makes the library calls that its
summary's ncu command captured, on seeded synthetic samples generated here.

    python -m benchlib.cases deep_assign_bf16
    python -m benchlib.cases gist_refine
    python -m benchlib.cases deep_refine_rounds [--tau T]
    python -m benchlib.cases sift_assign_levels [--levels 1,3] [--reps R]
    python -m benchlib.cases assign_large_table [--precision P]
    python -m benchlib.cases tree --n 1000000 --d 128 --k 10000 --iters 2 --calls 2
    python -m benchlib.cases boost [--visits V] [--calls C]

deep_assign_bf16  10^6 x 512 BF16 deep-feature-shaped samples (200,000 vMF directions, kappa_vMF = 50, seed 11);
                  graph construction with kappa = 40, tau = 1 at precision 2, then two fit iterations at
                  k = 100,000 (a centroid table far larger than L2, like the 10^7 x 512 workload's).
deep_refine_rounds  the deep_assign_bf16 samples; graph construction with kappa = 40, xi = 50 and --tau rounds
                  (default 4) at precision 0 (the FP32 tile refinement at this width).
gist_refine       3 x 10^5 x 960 GIST-shaped samples (1,000 latent centres, seed 5); graph construction with
                  kappa = 50, xi = 50, tau = 3 at precision 1 (the FP32 tile refinement at this width).
sift_assign_levels  the SIFT-shaped assignment after graph construction and fit, timed per precision level.
assign_large_table  one assignment over a 10^6-row centroid table (10^6 x 512 BF16 unit vectors, k = 10^6,
                  a random kappa = 40 graph, random labels); --precision selects the screening level.
boost             the boost form's epoch (Eq. 3 gains, Alg. 2 move step) on the SIFT-shaped sizes, from the
                  library's graph and fit partition, over prefixes of seeded visit permutations.
tree              the two-means tree (Alg. 1) on N(0, 1) samples drawn by a CUDA torch generator seeded with
                  --data-seed (BF16 with --bf16); --calls tree calls on one workspace, the first a warm-up;
                  prints one JSON line with the mean time of the other calls and the device status word.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def deep_assign_bf16(argv):
    import torch

    from paper_1705_01813_gb300 import datagen, gkm
    X = datagen.deep_like_device(1_000_000, 512, 200_000, 50.0, seed=11, device="cuda")
    torch.cuda.empty_cache()
    gi, _, _, _ = gkm.build_knn_graph(X, 40, xi=50, tau=1, seed=1, precision=2)
    _, _, _, log = gkm.kmeans_fit(X, 100_000, gi, 2, seed=2, precision=2)
    torch.cuda.synchronize()
    print("deep_assign_bf16 final distortion", log[-1])


def gist_refine(argv):
    import torch

    from paper_1705_01813_gb300 import datagen, gkm
    X = torch.from_numpy(datagen.gist_like(300_000, 960, 1000, seed=5)).cuda()
    _, _, _, log = gkm.build_knn_graph(X, 50, xi=50, tau=3, seed=1, precision=1)
    torch.cuda.synchronize()
    print("gist_refine final distortion", log[-1])


def deep_refine_rounds(argv):
    """Graph construction on the deep-feature-shaped samples of deep_assign_bf16 (10^6 x 512 BF16, 200,000 vMF
    directions, seed 11) with kappa = 40, xi = 50 and --tau rounds (default 4) at precision 0: every round's
    refinement runs the FP32 tile kernels on runs of about 50 members, as the 10^7 x 512 workload's do."""
    import torch

    from paper_1705_01813_gb300 import datagen, gkm
    ap = argparse.ArgumentParser(prog="benchlib.cases deep_refine_rounds")
    ap.add_argument("--tau", type=int, default=4)
    a = ap.parse_args(argv)
    X = datagen.deep_like_device(1_000_000, 512, 200_000, 50.0, seed=11, device="cuda")
    torch.cuda.empty_cache()
    _, _, _, log = gkm.build_knn_graph(X, 40, xi=50, tau=a.tau, seed=1, precision=0)
    torch.cuda.synchronize()
    print("deep_refine_rounds final distortion", log[-1])


def sift_assign_levels(argv):
    """The SIFT-shaped workload's assignment (10^6 x 128 FP32, 10^4 latent centres, k = 10^4, kappa = 50) after
    graph construction (tau = 10) and a 10-iteration fit, timed with CUDA events at each --levels precision
    (default 1 and 3) with the samples grouped by the fit's labels; prints one JSON line of ms per call."""
    import torch

    from paper_1705_01813_gb300 import datagen, gkm
    ap = argparse.ArgumentParser(prog="benchlib.cases sift_assign_levels")
    ap.add_argument("--levels", default="1,3")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--stats", action="store_true",
                    help="also print the candidate-union sizes of 128-sample tiles in label order")
    a = ap.parse_args(argv)
    w = datagen.WORKLOADS["sift_n1000000_d128_k10000"]
    X = torch.from_numpy(w.data()).cuda()
    gi, _, _, _ = gkm.build_knn_graph(X, w.kappa, xi=w.xi, tau=w.tau, seed=w.seed, precision=1, want_log=False)
    lab, C, _, _ = gkm.kmeans_fit(X, w.k, gi, w.iters, seed=w.seed + 1, precision=1)
    _, mem, _ = gkm.group_by_label(lab, w.k)
    if a.stats:
        cand = torch.cat([lab[mem.long()][:, None], lab[gi[mem.long()].long()]], 1)  # label order, n x (kappa + 1)
        srt = cand.sort(1).values
        u = 1 + (srt[:, 1:] != srt[:, :-1]).sum(1)
        nt = (w.n + 127) // 128
        pad = torch.full((nt * 128 - w.n, w.kappa + 1), -1, dtype=cand.dtype, device=cand.device)
        tiles = torch.cat([cand, pad]).view(nt, -1).sort(1).values
        U = 1 + (tiles[:, 1:] != tiles[:, :-1]).sum(1) - (tiles[:, 0] < 0).long()
        q = torch.quantile(U.float(), torch.tensor([0.1, 0.5, 0.9], device=U.device)).tolist()
        print(json.dumps({"distinct_candidates_per_sample": float(u.float().mean()),
                          "tile_union_mean": float(U.float().mean()), "tile_union_p10_p50_p90": q,
                          "tiles_over_1024": float((U > 1024).float().mean())}))
    ws = gkm.workspace(gkm.workspace_size(gkm.GK_OP_ASSIGN, w.n, w.d, w.k, w.kappa), X.device)
    out = torch.empty_like(lab)
    res = {}
    ref = None
    for p in [int(v) for v in a.levels.split(",")]:
        gkm.assign_step(X, gi, C, lab, out, None, None, None, p, mem, ws=ws)
        torch.cuda.synchronize()
        ref = out.clone() if ref is None else ref
        assert torch.equal(out, ref), "levels disagree"
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            gkm.assign_step(X, gi, C, lab, out, None, None, None, p, mem, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        res[p] = e0.elapsed_time(e1) / a.reps
    print(json.dumps({"ms_per_call": res, "status": gkm.read_status(ws)}))


def assign_large_table(argv):
    """One assignment at the deep-feature fit's ratios with a centroid table far larger than L2: 10^6 x 512 BF16
    unit vectors (normalised N(0, 1), seed 5), k = 10^6 centroids on sampled rows, a random kappa = 40 graph and
    random labels (about 41 distinct candidates per sample, as at 10^7 x 512, k = 10^6); --precision (default
    4 with 4 candidates per group, the tuned setting there); two calls, the second the one to capture."""
    import torch

    from paper_1705_01813_gb300 import gkm
    ap = argparse.ArgumentParser(prog="benchlib.cases assign_large_table")
    ap.add_argument("--precision", type=int, default=4 | (4 << 8))
    a = ap.parse_args(argv)
    n, d, k, kappa = 1_000_000, 512, 1_000_000, 40
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.nn.functional.normalize(torch.randn((n, d), generator=g, device="cuda"), dim=1).to(torch.bfloat16)
    gi = torch.randint(0, n, (n, kappa), generator=g, device="cuda", dtype=torch.int32)
    L = torch.randint(0, k, (n,), generator=g, device="cuda", dtype=torch.int32)
    C = X[torch.randint(0, n, (k,), generator=g, device="cuda")].float()
    ws = gkm.workspace(gkm.workspace_size(gkm.GK_OP_ASSIGN, n, d, k, kappa), X.device)
    out = torch.empty_like(L)
    for _ in range(2):
        gkm.assign_step(X, gi, C, L, out, None, None, None, a.precision, None, ws=ws)
    torch.cuda.synchronize()
    print(json.dumps({"changed": int((out != L).sum()), "status": gkm.read_status(ws)}))


def tree(argv):
    import torch

    from paper_1705_01813_gb300 import gkm
    ap = argparse.ArgumentParser(prog="benchlib.cases tree")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--d", type=int, default=128)
    ap.add_argument("--k", type=int, default=10_000)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--data-seed", type=int, default=1)
    ap.add_argument("--calls", type=int, default=2)
    ap.add_argument("--bf16", action="store_true")
    a = ap.parse_args(argv)
    X = torch.randn((a.n, a.d), device="cuda", generator=torch.Generator(device="cuda").manual_seed(a.data_seed))
    if a.bf16:
        X = X.to(torch.bfloat16)
    ws = gkm.workspace(gkm.workspace_size(gkm.GK_OP_TREE, a.n, a.d, a.k), X.device)
    lab = torch.empty(a.n, dtype=torch.int32, device="cuda")
    gkm.two_means_tree(X, a.k, iters=a.iters, seed=a.seed, out=lab, ws=ws)
    torch.cuda.synchronize()
    ms = None
    if a.calls > 1:
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(a.calls - 1):
            gkm.two_means_tree(X, a.k, iters=a.iters, seed=a.seed, out=lab, ws=ws)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (a.calls - 1)
    print(json.dumps({"n": a.n, "d": a.d, "k": a.k, "iters": a.iters, "bf16": a.bf16, "ms_per_call": ms,
                      "status": gkm.read_status(ws)}))


def boost(argv):
    """The boost form (Eq. 3 gains, Alg. 2 move step) on the SIFT-shaped workload's sizes: 10^6 x 128 FP32
    samples (datagen.sift_like), the library's graph (kappa = 50, xi = 50, tau = 10) and its fit's partition
    (k = 10^4, 10 iterations from seeded labels), then --calls epochs over the first --visits entries of seeded
    permutations; prints one JSON line with the last call's time per visit."""
    import torch

    from paper_1705_01813_gb300 import datagen, gkm
    ap = argparse.ArgumentParser(prog="benchlib.cases boost")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--d", type=int, default=128)
    ap.add_argument("--k", type=int, default=10_000)
    ap.add_argument("--kappa", type=int, default=50)
    ap.add_argument("--visits", type=int, default=20_000)
    ap.add_argument("--calls", type=int, default=2)
    a = ap.parse_args(argv)
    X = torch.from_numpy(datagen.sift_like(a.n, a.d)).cuda()
    gi = gkm.build_knn_graph(X, a.kappa, xi=50, tau=10, seed=1, want_log=False)[0]
    lab = gkm.kmeans_fit(X, a.k, gi, 10, seed=2, want_log=False)[0].clone()
    ws = gkm.workspace(gkm.workspace_size(gkm.GK_OP_BOOST, a.n, a.d, a.k, a.kappa), X.device)
    D, cnt, S = gkm.boost_init(X, lab, a.k, ws=ws)
    g = torch.Generator().manual_seed(3)
    ms = None
    for _ in range(a.calls):
        order = torch.randperm(a.n, generator=g)[:a.visits].to(torch.int32).cuda()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mv = gkm.boost_epoch(X, gi, order, lab, a.k, D, cnt, S, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    print(json.dumps({"n": a.n, "d": a.d, "k": a.k, "kappa": a.kappa, "visits": a.visits,
                      "us_per_visit": 1e3 * ms / a.visits, "moves": int(mv.item()), "status": gkm.read_status(ws)}))


CASES = {"deep_assign_bf16": deep_assign_bf16, "gist_refine": gist_refine, "deep_refine_rounds": deep_refine_rounds,
         "sift_assign_levels": sift_assign_levels, "assign_large_table": assign_large_table, "tree": tree,
         "boost": boost}


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    if not argv or argv[0] not in CASES:
        raise SystemExit("usage: python -m benchlib.cases {" + ",".join(CASES) + "} [options]")
    from paper_1705_01813_gb300 import gkm
    gkm.load()
    CASES[argv[0]](argv[1:])


if __name__ == "__main__":
    main()
