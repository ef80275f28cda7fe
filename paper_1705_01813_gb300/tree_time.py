"""Time the two-means tree (Alg. 1) on seeded Gaussian samples generated on the device.

    python -m paper_1705_01813_gb300.tree_time --n 1000000 --d 128 --k 10000 --iters 2 --calls 2

X = N(0, 1)^(n x d) from a CUDA torch generator seeded with --data-seed (BF16 with --bf16); --calls tree calls on
one workspace, the first a warm-up; prints one JSON line: the mean time of the other calls (CUDA events on the
current stream) and the device status word.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import gkm


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--d", type=int, default=128)
    ap.add_argument("--k", type=int, default=10_000)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--data-seed", type=int, default=1)
    ap.add_argument("--calls", type=int, default=2)
    ap.add_argument("--bf16", action="store_true")
    a = ap.parse_args(argv)
    gkm.load()
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


if __name__ == "__main__":
    main()
