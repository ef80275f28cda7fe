"""Autotuner over the library's precision levels and the assignment's tile shape.

Every level gives the same labels, centroids, distortions and graph bit for bit (the GPU tests assert it), so
the fastest one for a workload can be chosen by measurement alone: one assignment per level (0 to 4; 3 only
for FP32 samples) and one refinement per refinement path (level 0: the FP32 tiles; levels 1 to 4: the
tensor-core Gram where d allows it) are timed with CUDA events on the caller's samples and graph, and each
level is scored by the time the whole path would spend in those calls (the assignment runs tau + iters times
per graph construction and fit, the refinement tau times).  At the levels whose assignment runs the row kernels
(all but 3) the assignment is also timed with 4 and with 8 candidates per group (bits 8-15 of the precision
argument; the kernels' summation tree is the same for both, so the results are too), and the faster width goes
with the level.  Choices are cached per shape key.
"""
from __future__ import annotations

import torch

from . import gkm

_CACHE: dict = {}


def _bucket(v: int) -> int:
    """Powers of two: shapes within a factor of two share a tuning."""
    return max(1, int(v)).bit_length()


def shape_key(X: torch.Tensor, k: int, kappa: int) -> tuple:
    props = torch.cuda.get_device_properties(X.device)
    return (props.name, str(X.dtype), int(X.shape[1]), int(kappa), _bucket(X.shape[0]), _bucket(k))


def _time(fn, reps: int) -> float:
    fn()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_precision(X: torch.Tensor, g_idx: torch.Tensor, g_dist: torch.Tensor, labels: torch.Tensor, k: int,
                   tau: int = 10, iters: int = 10, max_cluster: int = 128, reps: int = 3,
                   use_cache: bool = True) -> dict:
    """Fastest precision level for the samples X with graph (g_idx, g_dist) and labels at k clusters.

    The graph and labels are read, never changed (the refinement is timed on copies).  Returns
    {"precision": p, "assign_ms": {p: ms}, "refine_ms": {path: ms}, "score_ms": {p: ms}, "key": key}."""
    kappa = g_idx.shape[1]
    key = shape_key(X, k, kappa)
    if use_cache and key in _CACHE:
        return _CACHE[key]
    n, d = X.shape
    dev = X.device
    levels = [0, 1, 2, 4] if X.dtype == torch.bfloat16 else [0, 1, 2, 3, 4]
    off, mem, cnt = gkm.group_by_label(labels, k)
    C = torch.zeros((k, d), dtype=torch.float32, device=dev)
    gkm.update_from_groups(X, off, mem, k, C, cnt)
    ws = gkm.workspace(max(gkm.workspace_size(gkm.GK_OP_ASSIGN, n, d, k, kappa),
                           gkm.workspace_size(gkm.GK_OP_REFINE, n, d, k, kappa)), dev)
    out = torch.empty_like(labels)
    assign_ms, group_width = {}, {}
    widths = [8, 4] if d <= 512 else [4]  # rows of more than 512 values take groups of 4
    for p in levels:
        best_w, best_t = 0, float("inf")
        for gw in (widths if p != 3 else [0]):
            code = p | (gw << 8)
            t = _time(lambda: gkm.assign_step(X, g_idx, C, labels, out, None, None, None, code, mem, ws=ws), reps)
            if t < best_t:
                best_w, best_t = gw, t
        assign_ms[p], group_width[p] = best_t, best_w
    gi, gd = g_idx.clone(), g_dist.clone()

    def refine(p):
        gi.copy_(g_idx)
        gd.copy_(g_dist)
        gkm.graph_refine_groups(X, off, mem, k, gi, gd, max_cluster, p, ws=ws)

    refine_ms = {"fp32_tiles": _time(lambda: refine(0), reps), "precision_ge_1": _time(lambda: refine(1), reps)}
    copy_ms = _time(lambda: (gi.copy_(g_idx), gd.copy_(g_dist)), reps)
    score = {p: assign_ms[p] * (tau + iters) +
             (refine_ms["fp32_tiles"] if p == 0 else refine_ms["precision_ge_1"]) * tau - copy_ms * tau
             for p in levels}
    best = min(levels, key=lambda p: (score[p], p))
    res = {"precision": best | (group_width[best] << 8), "level": best, "group_width": group_width[best],
           "assign_ms": assign_ms, "group_width_by_level": group_width, "refine_ms": refine_ms, "score_ms": score,
           "key": list(key)}
    _CACHE[key] = res
    return res
