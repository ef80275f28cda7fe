"""Measured ceilings beside the HBM copy and GEMM peaks: the bandwidth of warp-per-row gathers of table rows
(from L2 for a centroid-sized table, from HBM for one larger than L2) and packed FP32x2 FMA throughput, all
through this library's probe kernels (gk_probe_gather, gk_probe_fma), timed with CUDA events on the
launching stream.  The assignment gathers one centroid row per candidate; these are its ceilings where
HBM bandwidth is not the bound."""
from __future__ import annotations

import torch

from . import gkm


def _best(fn, reps: int, stream) -> float:
    """Shortest of `reps` timed runs of fn() (seconds), after one untimed run."""
    fn()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b) / 1e3)
    return best


def measure(device=None, reps: int = 5, seed: int = 7) -> dict:
    """{'l2_gather_gbs', 'hbm_gather_gbs', 'fp32_ffma2_tflops', ...} on the current device."""
    dev = torch.device(device or "cuda")
    stream = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    sink = torch.empty(gkm.PROBE_SINK, dtype=torch.float32, device=dev)
    out = {}
    # SIFT-shaped centroid table: 10,000 rows of 128 FP32 (5.1 MB, L2-resident)
    t_l2 = torch.randn((10_000, 128), generator=g, device=dev)
    i_l2 = torch.randint(0, t_l2.shape[0], (16_000_000,), generator=g, device=dev, dtype=torch.int32)
    nb = i_l2.numel() * t_l2.shape[1] * 4
    out["l2_gather_gbs"] = nb / _best(lambda: gkm.probe_gather(t_l2, i_l2, sink, stream), reps, stream) / 1e9
    out["l2_gather_table"] = "10,000 x 128 FP32 rows (5.1 MB), 16M random rows of 512 B"
    del t_l2, i_l2
    # deep-feature-shaped centroid table: 1,000,000 rows of 512 FP32 (2 GB, far above L2)
    t_hbm = torch.randn((1_000_000, 512), generator=g, device=dev)
    i_hbm = torch.randint(0, t_hbm.shape[0], (4_000_000,), generator=g, device=dev, dtype=torch.int32)
    nb = i_hbm.numel() * t_hbm.shape[1] * 4
    out["hbm_gather_gbs"] = nb / _best(lambda: gkm.probe_gather(t_hbm, i_hbm, sink, stream), reps, stream) / 1e9
    out["hbm_gather_table"] = "1,000,000 x 512 FP32 rows (2 GB), 4M random rows of 2 KB"
    del t_hbm, i_hbm
    iters = 20_000
    fl = 32 * iters * 152 * 8 * 256
    out["fp32_ffma2_tflops"] = fl / _best(lambda: gkm.probe_fma(sink, iters, stream), reps, stream) / 1e12
    torch.cuda.empty_cache()
    return out
