"""Measured ceilings beside the HBM copy and GEMM peaks, for the benchmark: the bandwidth of warp-per-row
gathers of table rows (from L2 for a centroid-sized table, from HBM for one larger than L2) and packed FP32x2
FMA throughput, through the probe kernels of ``benchlib/probes.cu`` (their own library, libgkm_probes.so,
not part of libgkm), timed with CUDA events on the launching stream.  The assignment gathers one centroid
row per candidate; these are its ceilings where HBM bandwidth is not the bound."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "probes.cu")
LIB = os.path.join(HERE, "_build", "libgkm_probes.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile libgkm_probes.so for sm_103a (one translation unit)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
                           "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "-shared", "-cudart",
                           "static", "-o", tmp, SRC])
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            L.gkb_probe_sink_floats.restype = ctypes.c_int
            L.gkb_probe_gather.argtypes = [P, I64, I32, P, I64, P, P]
            L.gkb_probe_gather.restype = ctypes.c_int
            L.gkb_probe_fma.argtypes = [P, I64, P]
            L.gkb_probe_fma.restype = ctypes.c_int
            _lib = L
    return _lib


def sink_floats() -> int:
    return int(load().gkb_probe_sink_floats())


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what}: {'bad argument' if rc == 1 else 'CUDA launch error'}")


def probe_gather(table, idx, sink, stream):
    """Warp-per-row gather of table rows idx[j]; returns the bytes it reads."""
    _check(load().gkb_probe_gather(ctypes.c_void_p(table.data_ptr()), table.shape[0], table.shape[1],
                                   ctypes.c_void_p(idx.data_ptr()), idx.numel(), ctypes.c_void_p(sink.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream)), "probe_gather")
    return idx.numel() * table.shape[1] * 4


def probe_fma(sink, iters: int, stream):
    """Packed FP32x2 FMA chains; returns the FLOP count."""
    _check(load().gkb_probe_fma(ctypes.c_void_p(sink.data_ptr()), iters, ctypes.c_void_p(stream.cuda_stream)),
           "probe_fma")
    return 32 * iters * sink.numel() * 32


def _best(fn, reps: int, stream) -> float:
    """Shortest of `reps` timed runs of fn() (seconds), after one untimed run."""
    import torch
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
    import torch
    dev = torch.device(device or "cuda")
    stream = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    sink = torch.empty(sink_floats(), dtype=torch.float32, device=dev)
    out = {}
    # SIFT-shaped centroid table: 10,000 rows of 128 FP32 (5.1 MB, L2-resident)
    t_l2 = torch.randn((10_000, 128), generator=g, device=dev)
    i_l2 = torch.randint(0, t_l2.shape[0], (16_000_000,), generator=g, device=dev, dtype=torch.int32)
    nb = i_l2.numel() * t_l2.shape[1] * 4
    out["l2_gather_gbs"] = nb / _best(lambda: probe_gather(t_l2, i_l2, sink, stream), reps, stream) / 1e9
    out["l2_gather_table"] = "10,000 x 128 FP32 rows (5.1 MB), 16M random rows of 512 B"
    del t_l2, i_l2
    # deep-feature-shaped centroid table: 1,000,000 rows of 512 FP32 (2 GB, far above L2)
    t_hbm = torch.randn((1_000_000, 512), generator=g, device=dev)
    i_hbm = torch.randint(0, t_hbm.shape[0], (4_000_000,), generator=g, device=dev, dtype=torch.int32)
    nb = i_hbm.numel() * t_hbm.shape[1] * 4
    out["hbm_gather_gbs"] = nb / _best(lambda: probe_gather(t_hbm, i_hbm, sink, stream), reps, stream) / 1e9
    out["hbm_gather_table"] = "1,000,000 x 512 FP32 rows (2 GB), 4M random rows of 2 KB"
    del t_hbm, i_hbm
    iters = 20_000
    fl = 32 * iters * sink.numel() * 32
    out["fp32_ffma2_tflops"] = fl / _best(lambda: probe_fma(sink, iters, stream), reps, stream) / 1e12
    torch.cuda.empty_cache()
    return out
