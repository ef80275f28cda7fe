"""Workloads behind the kernel-counter summaries: each case makes the library calls that its summary's ncu
command captured, on seeded synthetic samples generated here.

    python -m paper_1705_01813_gb300.profile_cases deep_assign_bf16
    python -m paper_1705_01813_gb300.profile_cases gist_refine

deep_assign_bf16  10^6 x 512 BF16 deep-feature-shaped samples (200,000 vMF directions, kappa_vMF = 50, seed 11);
                  graph construction with kappa = 40, tau = 1 at precision 2, then two fit iterations at
                  k = 100,000 (a centroid table far larger than L2, like the 10^7 x 512 workload's).
gist_refine       3 x 10^5 x 960 GIST-shaped samples (1,000 latent centres, seed 5); graph construction with
                  kappa = 50, xi = 50, tau = 3 at precision 1 (the FP32 tile refinement at this width).
"""
from __future__ import annotations

import sys

import torch

from . import datagen, gkm


def deep_assign_bf16():
    X = datagen.deep_like_device(1_000_000, 512, 200_000, 50.0, seed=11, device="cuda")
    torch.cuda.empty_cache()
    gi, _, _, _ = gkm.build_knn_graph(X, 40, xi=50, tau=1, seed=1, precision=2)
    _, _, _, log = gkm.kmeans_fit(X, 100_000, gi, 2, seed=2, precision=2)
    torch.cuda.synchronize()
    return log[-1]


def gist_refine():
    X = torch.from_numpy(datagen.gist_like(300_000, 960, 1000, seed=5)).cuda()
    _, _, _, log = gkm.build_knn_graph(X, 50, xi=50, tau=3, seed=1, precision=1)
    torch.cuda.synchronize()
    return log[-1]


CASES = {"deep_assign_bf16": deep_assign_bf16, "gist_refine": gist_refine}


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    if len(argv) != 1 or argv[0] not in CASES:
        raise SystemExit("usage: python -m paper_1705_01813_gb300.profile_cases {" + ",".join(CASES) + "}")
    gkm.load()
    print(argv[0], "final distortion", CASES[argv[0]]())


if __name__ == "__main__":
    main()
