#!/usr/bin/env python
"""Benchmark of the graph-guided k-means hot path on GB300.

One step is one pass of the whole path over the workload (default: the
deep-feature-shaped n = 10,000,000, d = 512 (BF16 samples), k = 1,000,000,
kappa = 40 workload, the paper's largest scale; --workload picks another):
  graph construction (Alg. 3): random graph and labels at k0 = n / xi, then
      tau = 10 rounds of {graph-guided assignment, grouping, update, pair refinement}
  graph-guided k-means (Alg. 2, closest-centroid rule): seeded labels at k,
      then 10 iterations of {assignment, grouping, update}
The step is driven through the library's step entry points (the same kernels
the one-call API runs): once launched call by call with CUDA events between the
calls (the per-kernel durations of the roofline), then captured into a CUDA
graph whose replay time is `value`.  `e2e` times the one-call API
(gk_build_knn_graph + gk_kmeans_fit) with the samples copied from pinned host
memory and the labels and centroids copied back inside the timed region.  By
default the precision level is chosen by the autotuner (tune.py) after the
first warm-up step.  Outside the timed region the line also reports the
constructed graph's top-1 recall (Sec. 5), the probe-measured gather and FMA
ceilings, the serving passes, the boost form (Eq. 3 gains, Alg. 2 move step)
from the fit's partition over a prefix of one epoch's visits, and the oracle's
timing on a bounded sample with the library's results on that sample compared
to the oracle's (graph and fit; the boost epoch bit for bit).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gkm|reference]
Under torchrun (N > 1) every rank runs an independent replica on its GPU
(the path needs no exchange between GPUs); value = samples of all ranks / the
slowest rank's time.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1705_01813_gb300 import datagen  # noqa: E402

# `value` is samples per second of the whole path (one graph construction + one fit per step); the assign-step
# rate, the fit time against the plain FP32 path and the serving figures of the headline metric ride beside it
METRIC = ("whole-path samples/s (graph construction + fit per step); beside it: assign-step samples/s, fit time vs "
          "plain FP32, serve jobs/s and p50/p99")
DEFAULT_WORKLOAD = "deep_n10000000_d512_k1000000"
CPU_SAMPLE = 100_000        # cpu_baseline: oracle on the first 100k samples at d = 128 (about 10-30 s)
REF_SAMPLE = 100_000        # --impl reference: oracle per step on the first 100k samples at d = 128 (fewer for wider rows)


L2_BYTES = 129 << 20  # GB300 L2


def oracle_sample(w, base):
    """Samples the oracle runs on: `base` at d = 128, fewer for wider rows (its time grows with d)."""
    return min(w.n, max(2000, base * 128 // max(w.d, 1)))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gkm", "reference"], default="gkm")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(datagen.WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", type=int, choices=[0, 1, 2, 3, 4], default=None,
                    help="0 FP32 SIMT throughout; 1 tensor-core Gram + FP32 rerank in the refinement; 2 also "
                         "BF16 screening in the assignment (SIMT); 3 the screening on the tensor cores; 4 int8 "
                         "screening (SIMT) (all give the same results).  Default: chosen by the autotuner (tune.py) on "
                         "the workload's own "
                         "graph and labels after the first warm-up step")
    ap.add_argument("--group-width", type=int, choices=[0, 4, 8], default=0,
                    help="with --precision: the assignment's candidates per group (0: the kernels' default)")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-boost", action="store_true",
                    help="skip the timing of the boost form (Eq. 3 gains, Alg. 2 move step) on the fit's partition")
    ap.add_argument("--boost-visits", type=int, default=100_000,
                    help="visits of the timed boost epoch (a prefix of a seeded permutation of the samples)")
    ap.add_argument("--no-tree", action="store_true",
                    help="skip the timing of the two-means tree (Alg. 1) at the workload's n, d and k")
    ap.add_argument("--no-ceilings", action="store_true",
                    help="skip the probe kernels that measure the L2 / HBM gather and FP32 FMA ceilings")
    ap.add_argument("--no-replay", action="store_true",
                    help="e2e: launch the one-call API's kernels one by one (default: repeated requests replay the "
                         "CUDA graph captured on their first call, gk_set_replay)")
    ap.add_argument("--no-graph", action="store_true",
                    help="time the step launched op by op only (default: also captured into a CUDA graph, whose "
                         "replay time is the value)")
    ap.add_argument("--serve-jobs", type=int, default=512,
                    help="jobs of the serving stream to run after the step measurement (0: none; 512: all)")
    ap.add_argument("--compare-steps", type=int, default=2,
                    help="steps of the plain FP32 path timed for the comparison (after one untimed step)")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="requests timed through the one-call API with host buffers (at most --steps)")
    ap.add_argument("--traffic-from", metavar="CSV",
                    help="no GPU run: read an ncu --csv log with dram__bytes_read.sum, dram__bytes_write.sum and "
                         "gpu__time_duration.sum of this workload's kernels and record the per-launch means in "
                         "profiles/traffic.json, tagged with the current kernel sources")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def reduce_max(value: float, dist, device) -> float:
    """Largest value over the ranks of the default process group (the slowest replica's time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(samples_per_rank: int, steps: int, world: int, slowest_s: float) -> float:
    """Samples of all replicas per second of the slowest replica (weak scaling: each rank runs the workload)."""
    return world * samples_per_rank * steps / slowest_s


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), float(j["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", self.gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        load = [v for v in sm if mx and v > 0.3 * mx] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- GPU path --

class Path:
    """Device buffers and the step sequence of one replica."""

    def __init__(self, gkm, torch, w, X, precision=1):
        self.gkm, self.torch, self.w = gkm, torch, w
        self.precision = precision
        dev = X.device
        n, d = X.shape
        self.X, self.n, self.d = X, n, d
        self.k0 = w.k0
        i32, f32, f64 = torch.int32, torch.float32, torch.float64
        self.gi = torch.empty((n, w.kappa), dtype=i32, device=dev)
        self.gd = torch.empty((n, w.kappa), dtype=f32, device=dev)
        self.la = torch.empty(n, dtype=i32, device=dev)
        self.lb = torch.empty(n, dtype=i32, device=dev)
        kmax = max(self.k0, w.k)
        self.off = torch.empty(kmax + 1, dtype=i32, device=dev)
        self.mem = torch.empty(n, dtype=i32, device=dev)
        self.cnt = torch.empty(kmax, dtype=i32, device=dev)
        self.C0 = torch.empty((self.k0, d), dtype=f32, device=dev)
        self.C = torch.empty((w.k, d), dtype=f32, device=dev)
        self.s = torch.empty(4, dtype=f64, device=dev)
        self.ws = gkm.Workspace(max(gkm.workspace_size(gkm.GK_OP_FIT, n, d, kmax, w.kappa),
                                    gkm.workspace_size(gkm.GK_OP_REFINE, n, d, kmax, w.kappa),
                                    gkm.workspace_size_build(n, d, w.kappa, w.xi, w.tau, w.max_cluster)), dev)

    def _ev(self):
        return self.torch.cuda.Event(enable_timing=True)

    def step(self, rec=None, probe=None):
        """Whole path once; rec (list) receives (tag, start_event, end_event) per call; probe(phase,
        labels) is called with the labels the last assignment of each phase produced."""
        g, w, torch = self.gkm, self.w, self.torch

        def call(tag, fn, *a, **kw):
            if rec is None:
                return fn(*a, **kw)
            e0, e1 = self._ev(), self._ev()
            e0.record()
            out = fn(*a, **kw)
            e1.record()
            rec.append((tag, e0, e1))
            return out

        n, ws = self.n, self.ws
        # --- Alg. 3: KNN graph by repeated fast k-means at k0
        call("init_graph", g.init_graph, self.X, w.kappa, w.seed, self.gi, self.gd, ws=ws)
        g.init_labels(n, self.k0, w.seed, out=self.la)
        self.C0.zero_()
        call("group", g.group_by_label, self.la, self.k0, self.off, self.mem, self.cnt, ws=ws)
        call("update", g.update_from_groups, self.X, self.off, self.mem, self.k0, self.C0, self.cnt, self.s[0:1], ws=ws)
        cur, nxt = self.la, self.lb
        for _ in range(w.tau):
            call("assign", g.assign_step, self.X, self.gi, self.C0, cur, nxt, None, self.s[1:2], None,
                 self.precision, self.mem, ws=ws)
            call("group", g.group_by_label, nxt, self.k0, self.off, self.mem, self.cnt, ws=ws)
            call("update", g.update_from_groups, self.X, self.off, self.mem, self.k0, self.C0, self.cnt,
                 self.s[0:1], ws=ws)
            call("refine", g.graph_refine_groups, self.X, self.off, self.mem, self.k0, self.gi, self.gd,
                 w.max_cluster, self.precision, ws=ws)
            cur, nxt = nxt, cur
        if probe:
            probe("build", cur)
        # --- Alg. 2 (closest-centroid rule) at k on the constructed graph
        g.init_labels(n, w.k, w.seed + 1, out=self.la)
        self.C.zero_()
        cur, nxt = self.la, self.lb
        call("group", g.group_by_label, cur, w.k, self.off, self.mem, self.cnt, ws=ws)
        call("update", g.update_from_groups, self.X, self.off, self.mem, w.k, self.C, self.cnt, self.s[2:3], ws=ws)
        for _ in range(w.iters):
            call("assign", g.assign_step, self.X, self.gi, self.C, cur, nxt, None, self.s[3:4], None,
                 self.precision, self.mem, ws=ws)
            call("group", g.group_by_label, nxt, w.k, self.off, self.mem, self.cnt, ws=ws)
            call("update", g.update_from_groups, self.X, self.off, self.mem, w.k, self.C, self.cnt, self.s[2:3],
                 ws=ws)
            cur, nxt = nxt, cur
        if probe:
            probe("fit", cur)

    def mean_candidates(self, labels):
        """u: mean number of distinct candidate clusters per sample ({L[i]} and the neighbours' labels)."""
        torch = self.torch
        labs = torch.cat([labels[:, None], labels[self.gi.long()]], 1)
        srt, _ = torch.sort(labs, 1)
        return float((1 + (srt[:, 1:] != srt[:, :-1]).sum(1)).double().mean())


def _radix_passes(k):
    # 8-bit passes over the sort keys 0..k (k: the key of an out-of-range label)
    return (int(k).bit_length() + 7) // 8


def launches_per_step(w, precision):
    """Kernels of this library launched by one step (mirrors the library's launch sequence)."""
    grp = lambda k: 1 + 3 + 5 * _radix_passes(k)  # noqa: E731
    # update: the warp-per-cluster kernel for clusters of at most 32 members (16-byte rows of at most 512 values),
    # the block kernel for the others, the FP64 sum
    upd = 3 if (w.d % 4 == 0 and w.d <= 512) else 2

    def asg(k):
        # (then reduce and finish): kernel (0, 1); shadow copy + screening kernel (2, 4); BF16 copy, tensor-core
        # tiles, SIMT leftovers (3)
        return 3 if precision < 2 else (4 if precision in (2, 4) or w.d > 128 else 5)
    # refine: run count, scan, run clusters, then cluster-sorted copy + Gram + exact recompute + merge (tensor
    # cores) or the two FP32 tile widths
    ref = 1 + 3 + 1 + (4 if tc_refine(precision, w.d, w.storage) else 2)
    graph = 1 + 1 + grp(w.k0) + upd + w.tau * (asg(w.k0) + grp(w.k0) + upd + ref)
    fit = 1 + grp(w.k) + upd + w.iters * (asg(w.k) + grp(w.k) + upd)
    return graph + fit


def algorithmic_bytes(tag, w, k):
    """HBM bytes one launch of a step's kernel must move (per-unit figures x units; L2-resident
    label gathers not counted)."""
    n, d, kappa = w.n, w.d, w.kappa
    s = 2 if w.storage == "bf16" else 4  # bytes per stored sample element
    if tag == "assign":
        return n * (s * d + 4 * kappa + 4 + 4) + k * d * 4
    if tag == "update":
        return n * (s * d + 4) + k * (d * 4 + 8)
    if tag == "group":
        return n * 12 + 4 * (k + 1)
    if tag == "refine":
        return n * (s * d + 16 * kappa + 4) + 4 * (k + 1)
    return 0


def tc_refine(precision, d, storage="f32"):
    """The library's dispatch of the refinement to the tensor-core Gram (the same for both storage types)."""
    return precision >= 1 and 64 <= d <= 128


def kernel_of(tag, precision=1, d=128, storage="f32"):
    if tag == "refine" and tc_refine(precision, d, storage):
        return "k_refine_gram"
    if tag == "assign" and precision in (2, 4):
        return "k_assign_rows_scr"
    if tag == "assign" and precision == 3:
        return "k_assign_tc"
    return {"assign": "k_assign_rows", "update": "k_update", "group": "k_radix_scatter", "refine": "k_refine",
            "init_graph": "k_init_graph"}[tag]


# source file of each kernel whose DRAM traffic is recorded
KERNEL_SOURCE = {"k_assign_rows": "assign.cu", "k_assign_rows_scr": "assign.cu", "k_assign_tc": "assign_tc.cu",
                 "k_update": "update.cu",
                 "k_radix_scatter": "group.cu", "k_refine": "refine.cu", "k_refine_gram": "refine_tc.cu",
                 "k_refine_merge": "refine_tc.cu", "k_refine_exact": "refine_tc.cu", "k_init_graph": "init.cu"}


def file_sha(f):
    with open(os.path.join(ROOT, "paper_1705_01813_gb300", "csrc", f), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def source_sha(tag, precision=1, d=128, storage="f32"):
    return file_sha(KERNEL_SOURCE[kernel_of(tag, precision, d, storage)])


def write_traffic(csv_path, workload):
    """Per-launch DRAM bytes and ncu durations of the listed kernels from an ncu --csv log."""
    import csv
    import io
    import re
    with open(csv_path, errors="replace") as f:
        lines = [ln for ln in f.read().splitlines() if ln.startswith('"')]
    rows = list(csv.reader(io.StringIO("\n".join(lines))))
    h = rows[0]
    ki, ii, mi, ui, vi = (h.index(c) for c in ("Kernel Name", "ID", "Metric Name", "Metric Unit", "Metric Value"))
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "ns": 1e-3, "us": 1, "usecond": 1,
             "nsecond": 1e-3, "ms": 1e3, "msecond": 1e3}
    per = {}
    for r in rows[1:]:
        m = re.match(r"(?:void )?(?:gkm::)?(\w+)", r[ki])
        name = m.group(1) if m else r[ki]
        if name not in KERNEL_SOURCE:
            continue
        v = float(r[vi].replace(",", "")) * scale.get(r[ui], 1)
        per.setdefault(name, {}).setdefault(r[ii], {})[r[mi]] = v
    p = os.path.join(ROOT, "profiles", "traffic.json")
    j = {}
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
    for name, launches in per.items():
        ls = [m for m in launches.values() if "dram__bytes_read.sum" in m and "dram__bytes_write.sum" in m]
        if not ls:
            continue
        rd = sum(m["dram__bytes_read.sum"] for m in ls) / len(ls)
        wr = sum(m["dram__bytes_write.sum"] for m in ls) / len(ls)
        us = [m["gpu__time_duration.sum"] for m in ls if "gpu__time_duration.sum" in m]
        j[f"{name}:{workload}"] = {"dram_bytes_per_launch": int(rd + wr), "read": int(rd), "write": int(wr),
                                   "launches": len(ls),
                                   "ncu_us_per_launch": round(sum(us) / len(us), 1) if us else None,
                                   "source_sha": file_sha(KERNEL_SOURCE[name])}
    with open(p, "w") as f:
        json.dump(j, f, indent=1)
        f.write("\n")
    print(json.dumps({k: v["dram_bytes_per_launch"] for k, v in j.items() if not k.startswith("_")}, indent=1))


def ncu_traffic(tag, workload, precision=1, d=128, storage="f32"):
    """DRAM bytes per launch from the committed ncu summary, if it is for the current source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    e = j.get(f"{kernel_of(tag, precision, d, storage)}:{workload}")
    if not e or e.get("source_sha") != source_sha(tag, precision, d, storage):
        return None
    return e.get("dram_bytes_per_launch")


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1705_01813_gb300 import gkm

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    w = datagen.WORKLOADS[args.workload]
    X, Xh = workload_samples(w, torch)
    gkm.load()

    tuning = None
    if args.precision is not None:
        args.precision |= args.group_width << 8
    path = Path(gkm, torch, w, X, 1 if args.precision is None else args.precision)
    u = {}
    for q in range(args.warmup):  # the last warm-up step also measures u (outside the timed region)
        path.step(probe=(lambda ph, lab: u.__setitem__(ph, round(path.mean_candidates(lab), 2)))
                  if q == args.warmup - 1 else None)
        if q == 0 and args.precision is None:
            # the autotuner on this replica's graph and fit labels (all levels give the same results)
            from paper_1705_01813_gb300 import tune
            torch.cuda.synchronize()
            tuning = tune.tune_precision(path.X, path.gi, path.gd, path.la if w.iters % 2 == 0 else path.lb, w.k,
                                         tau=w.tau, iters=w.iters, max_cluster=w.max_cluster)
            args.precision = path.precision = tuning["precision"]
    torch.cuda.synchronize()
    if gkm.read_status(path.ws) != gkm.GK_OK:
        raise RuntimeError("device status error during warm-up")

    props = torch.cuda.get_device_properties(local_rank)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local_rank)
    clocks = ClockSampler(gpu_id)
    rec = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record()
    for _ in range(args.steps):
        path.step(rec)
    t_end.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed_stream = t_start.elapsed_time(t_end) / 1e3
    # the same step captured once into a CUDA graph and replayed (no launch gaps between kernels)
    elapsed_graph, graph_note = None, None
    if not args.no_graph:
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                path.step()
            graph.replay()  # one untimed replay
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record()
            for _ in range(args.steps):
                graph.replay()
            g1.record()
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            elapsed_graph = g0.elapsed_time(g1) / 1e3
        except Exception as e:  # reported in the line; the stream-launched time stands
            graph_note = f"capture failed: {str(e)[:160]}"
    ck = clocks.stop()
    elapsed = elapsed_graph if elapsed_graph is not None else elapsed_stream
    if world > 1:
        elapsed = reduce_max(elapsed, dist, "cuda")
        elapsed_stream = reduce_max(elapsed_stream, dist, "cuda")
    per_tag = {}
    for tag, e0, e1 in rec:
        per_tag.setdefault(tag, []).append(e0.elapsed_time(e1) / 1e3)
    status = gkm.read_status(path.ws)

    # the plain FP32 path (SIMT pair distances) on the same workload, for comparison
    fp32_ms = None
    lvl = args.precision & 0xff  # the level; bits 8-15 carry the assignment's candidates per group
    if lvl != 0 and not args.no_fp32_compare:
        path.precision = 0
        path.step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(max(1, args.compare_steps)):
            path.step()
        b.record()
        torch.cuda.synchronize()
        fp32_ms = a.elapsed_time(b) / max(1, args.compare_steps)
        path.precision = args.precision

    # e2e through the one-call API with host buffers
    e2e = None
    if not args.no_e2e:
        Xpin = Xh.pin_memory()
        Xdev = torch.empty_like(X)
        lab_h = torch.empty(w.n, dtype=torch.int32).pin_memory()
        C_h = torch.empty((w.k, w.d), dtype=torch.float32).pin_memory()
        gi = torch.empty((w.n, w.kappa), dtype=torch.int32, device="cuda")
        gd = torch.empty((w.n, w.kappa), dtype=torch.float32, device="cuda")
        lab0 = torch.empty(w.n, dtype=torch.int32, device="cuda")
        lab = torch.empty(w.n, dtype=torch.int32, device="cuda")
        C = torch.empty((w.k, w.d), dtype=torch.float32, device="cuda")
        cnt = torch.empty(w.k, dtype=torch.int32, device="cuda")

        def e2e_step():
            Xdev.copy_(Xpin, non_blocking=True)
            gkm.build_knn_graph(Xdev, w.kappa, w.xi, w.tau, w.max_cluster, w.seed, labels_out=lab0, g_idx=gi,
                                g_dist=gd, want_log=False, precision=args.precision, ws=path.ws)
            gkm.kmeans_fit(Xdev, w.k, gi, w.iters, seed=w.seed + 1, labels_out=lab, C_out=C, counts_out=cnt,
                           want_log=False, precision=args.precision, ws=path.ws)
            lab_h.copy_(lab, non_blocking=True)
            C_h.copy_(C, non_blocking=True)

        # the repeated request is replayed as the CUDA graph captured on its first call (gk_set_replay), on a
        # stream of its own (the legacy default stream is never captured)
        gkm.set_replay(not args.no_replay)
        e2e_stream = torch.cuda.Stream()
        with torch.cuda.stream(e2e_stream):
            for _ in range(max(1, args.warmup)):
                e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        t0 = time.perf_counter()
        with torch.cuda.stream(e2e_stream):
            a.record()
            for _ in range(e2e_steps):
                e2e_step()
            b.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        gkm.set_replay(False)
        t_e2e = max(a.elapsed_time(b) / 1e3, wall)
        if world > 1:
            t_e2e = reduce_max(t_e2e, dist, "cuda")
        e2e = {"value": whole_job_rate(w.n, e2e_steps, world, t_e2e), "unit": "samples/s",
               "h2d_bytes_per_step": int(Xh.numel() * Xh.element_size()),
               "d2h_bytes_per_step": int(lab_h.numel() * 4 + C_h.numel() * 4),
               "ms_per_step": 1e3 * t_e2e / e2e_steps, "steps": e2e_steps, "replay": not args.no_replay}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # graph quality: top-1 recall of the constructed graph on seeded sampled queries (Sec. 5), timed apart
    gq = torch.Generator(device="cuda")
    gq.manual_seed(w.seed + 7)
    n_q = min(w.n, 1000)
    queries = torch.randint(0, w.n, (n_q,), generator=gq, device="cuda", dtype=torch.int32)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record()
    hits, _, _ = gkm.graph_recall(path.X, path.gi, queries)
    r1.record()
    torch.cuda.synchronize()
    recall = {"value": int(hits.item()) / n_q, "queries": n_q, "ms": r0.elapsed_time(r1),
              "note": "top-1 recall of the graph after the step's construction (tau rounds), exact neighbours by "
                      "brute force on seeded random queries"}

    tree = None if args.no_tree else time_tree(gkm, torch, path.X, w)
    boost = None if args.no_boost else time_boost(gkm, torch, path.X, w, path.gi,
                                                 path.la if w.iters % 2 == 0 else path.lb, args.boost_visits)

    hbm, bf16, peak_src = load_peaks()
    ceilings = None
    if not args.no_ceilings:
        from benchlib import probes
        ceilings = probes.measure()
    # dominant kernel: the call with the largest share of the step
    totals = {t: sum(v) for t, v in per_tag.items()}
    dom = max(totals, key=totals.get)
    n_graph = w.tau + 1
    # per-launch algorithmic bytes: graph rounds run at k0, fit iterations at k
    if dom in ("assign", "update", "group"):
        ks = [w.k0] * (w.tau + (0 if dom == "assign" else 1)) + [w.k] * (w.iters + (0 if dom == "assign" else 1))
        alg = sum(algorithmic_bytes(dom, w, k) for k in ks) / len(ks)
    else:
        alg = algorithmic_bytes(dom, w, w.k0)
    avg = statistics.mean(per_tag[dom])
    achieved = alg / avg / 1e9
    assign_times = per_tag.get("assign", [])
    fit_assign = assign_times[w.tau::w.tau + w.iters] if assign_times else []
    step_s = elapsed / args.steps
    res = {
        "metric": METRIC,
        "value": whole_job_rate(w.n, args.steps, world, elapsed),
        "unit": "samples/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * step_s,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "d": w.d, "k": w.k, "kappa": w.kappa, "k0": w.k0, "xi": w.xi,
                   "tau": w.tau, "iters": w.iters, "max_cluster": w.max_cluster,
                   "step": "graph construction (tau rounds at k0) + fit (iters at k), whole path",
                   "storage": w.storage,
                   "l2": "inputs larger than L2 (X is %d MB)" % ((Xh.numel() * Xh.element_size()) >> 20),
                   "parallelism": f"replicas x{world}"},
        "fit_s": step_s,
        "precision": {0: "fp32 throughout",
                      1: "bf16 tcgen05 gram in the refinement with exact fp32 recompute inside its error bound",
                      2: "1 plus bf16 screening of assignment candidates (simt) with exact fp32 recompute",
                      3: "1 plus bf16 tcgen05 screening of assignment candidates with exact fp32 recompute",
                      4: "1 plus int8 (per-row scale) screening of assignment candidates (simt) with exact fp32 "
                         "recompute"}
                     [lvl],
        "assign_group_width": (args.precision >> 8) & 0xff or None,
        "plain_fp32_ms_per_step": fp32_ms,
        "assign_samples_per_s": w.n / statistics.mean(assign_times) if assign_times else None,
        "per_call_ms": {t: round(1e3 * statistics.mean(v), 4) for t, v in per_tag.items()},
        "per_step_share": {t: round(v / sum(totals.values()), 4) for t, v in totals.items()},
        "roofline": {"kernel": kernel_of(dom, lvl, w.d, w.storage), "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": int(alg),
                     "traffic": ncu_traffic(dom, w.name, lvl, w.d, w.storage)},
        "gpu_launches": launches_per_step(w, lvl) * args.steps,
        "measured_ceilings": ceilings,
        "precision_tuning": tuning,
        "graph_recall_top1": recall,
        "two_means_tree": tree,
        "boost_form": boost,
        "candidates_u": u or None,
        "clocks": ck,
        "device_status": status,
        "cuda_graph": {"used": elapsed_graph is not None, "ms_per_step_graph": None if elapsed_graph is None else
                       1e3 * elapsed_graph / args.steps, "ms_per_step_launched": 1e3 * elapsed_stream / args.steps,
                       "note": graph_note},
        "e2e": e2e,
    }
    # roofline of every call type, for context
    # The assignment gathers one centroid row per candidate: n u d (BF16 rows at precision >= 2, FP32 rows
    # otherwise) bytes per call beyond the algorithmic ones, u the measured mean candidate count of the phase
    # (graph rounds at k0, fit iterations at k).  They come from L2 while the centroid table fits it and from
    # HBM otherwise; the probe kernels measure both gather ceilings on this GPU.
    if dom == "assign" and u:
        row_b = {2: 2, 3: 2, 4: 1}.get(lvl, 4)
        per = [(w.k0, u.get("build"), w.tau), (w.k, u.get("fit"), w.iters)]
        g_l2 = sum(w.n * uu * w.d * row_b * c for kk, uu, c in per if uu and kk * w.d * 4 <= L2_BYTES)
        g_hbm = sum(w.n * uu * w.d * row_b * c for kk, uu, c in per if uu and kk * w.d * 4 > L2_BYTES)
        g_l2, g_hbm = g_l2 / (w.tau + w.iters), g_hbm / (w.tau + w.iters)
        gath = {"bytes_per_launch": int(g_l2 + g_hbm), "from_l2": int(g_l2), "from_hbm": int(g_hbm),
                "achieved_gbs": (g_l2 + g_hbm) / avg / 1e9,
                "note": "candidate centroid rows, one per candidate (exact second-pass rows at precision 2 not "
                        "counted)"}
        if ceilings:
            # time the gathers would take at the measured ceilings, against the call's time
            t_min = g_l2 / (ceilings["l2_gather_gbs"] * 1e9) + g_hbm / (ceilings["hbm_gather_gbs"] * 1e9)
            gath["ceiling"] = "measured warp-per-row gather (" + ("L2" if g_hbm == 0 else "HBM" if g_l2 == 0
                                                                   else "L2 and HBM") + ")"
            gath["frac_of_gather_ceiling"] = t_min / avg
        res["roofline"]["centroid_gathers"] = gath
    res["roofline_all"] = {}
    for t, v in per_tag.items():
        if t == "init_graph":
            continue
        a = algorithmic_bytes(t, w, w.k0 if t == "refine" else w.k)
        res["roofline_all"][t] = round(a / statistics.mean(v) / 1e9 / hbm, 4)
    if world == 1 and args.serve_jobs > 0:
        res["serving"] = serving(args)
    if world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(w, Xh[:oracle_sample(w, CPU_SAMPLE)].float().numpy(), args.precision)
    print(json.dumps(res), flush=True)
    if world > 1:
        dist.destroy_process_group()


def serving(args):
    """The serving workload (Poisson stream of clustering jobs, n log-uniform in [1e4, 1e6], d in
    {64, 128, 256}, k = n / 100, kappa = 20, HBM budget 120 GB), bounded to its first jobs: the stream
    at its arrival times (latency), all jobs at once (throughput), and the same jobs one at a time on
    the FP32 path (the per-job form), with the largest relative difference of final distortion."""
    import torch

    from paper_1705_01813_gb300 import serve
    specs = serve.job_specs(datagen.serving_jobs()[:args.serve_jobs])
    p = serve.ServeParams(budget_bytes=120 << 30, slots=8, precision=args.precision)
    srv = serve.Server(p)
    srv.run(specs[:2], realtime=False)  # warm-up: library load, allocator, first launches
    torch.cuda.synchronize()
    live = serve.summarize(srv.run(specs, realtime=True))
    sat_res = srv.run(specs, realtime=False)
    sat = serve.summarize(sat_res)
    pb = serve.ServeParams(budget_bytes=p.budget_bytes, slots=p.slots, precision=args.precision, batching=True)
    bsrv = serve.Server(pb)
    # warm-up of the batched form on jobs that make multi-job batches (first-use costs of its launches, about
    # 5 s on a fresh box, would otherwise land on the stream's first jobs)
    bsrv.run(specs[:16], realtime=False)
    torch.cuda.synchronize()
    blive = serve.summarize(bsrv.run(specs, realtime=True))
    bsat_res = bsrv.run(specs, realtime=False)
    bsat = serve.summarize(bsat_res)
    ser_res = serve.run_serial(specs, serve.ServeParams(budget_bytes=p.budget_bytes, slots=1, precision=0))
    ser = serve.summarize(ser_res)
    dE = max(abs(a.distortion - b.distortion) / max(abs(b.distortion), 1e-300)
             for res in (sat_res, bsat_res) for a, b in zip(res, ser_res))
    r3 = lambda d: {k: round(v, 3) if isinstance(v, float) else v for k, v in d.items()}  # noqa: E731
    return {"jobs": len(specs), "rate_per_s": 20.0, "slots": p.slots, "budget_gb": 120,
            "stream": r3(live), "saturation": r3(sat),
            "batched_stream": r3(blive), "batched_saturation": r3(bsat),
            "per_job_fp32_serial": r3(ser),
            "max_rel_distortion_diff": dE,
            "workload": "first jobs of the seeded Poisson stream (rate 20/s): n log-uniform in [1e4, 1e6], "
                        "d in {64, 128, 256}, k = n/100, kappa = 20, Gaussian mixtures generated on the device"}


def workload_samples(w, torch):
    """(X on the device, the same samples in host memory) for a workload: FP32 recipes are drawn on the
    host; the BF16-stored deep-feature recipe is drawn on the device (its host generator would take hours
    at 10^7 rows) and copied back for the end-to-end leg and the oracle's sample."""
    if w.storage == "bf16":
        X = datagen.deep_like_device(w.n, w.d, w.extra["n_dirs"], 50.0, w.seed, device="cuda")
        torch.cuda.empty_cache()
        return X, X.cpu()
    if w.name.startswith("gist"):  # 10^9 Beta draws: a minute on the host, a second on the device
        X = datagen.gist_like_device(w.n, w.d, w.extra.get("n_latent", 1000), w.seed, device="cuda")
        torch.cuda.empty_cache()
        return X, X.cpu()
    Xh = torch.from_numpy(w.data())
    return Xh.cuda(), Xh


def _oracle_step(O, w, X):
    """Graph construction and fit of the oracle on the samples X; returns (k, graph ids, final labels, final
    distortion)."""
    ns = X.shape[0]
    k = max(1, int(round(w.k * ns / w.n)))
    gi, _, _, _ = O.build_graph(X, w.kappa, xi=w.xi, tau=w.tau, max_cluster=w.max_cluster, seed=w.seed)
    L0 = O.init_labels(ns, k, w.seed + 1)
    Lf, _, _, E = O.fit(X, k, gi, w.iters, L0)
    return k, gi, Lf, float(np.asarray(E)[-1])


def gpu_vs_oracle(w, X, k, ora, precision):
    """The library's graph construction and fit on the oracle's sample (same seeds, the workload's storage
    type), against the oracle's results: relative difference of the final distortion, and the fractions of
    equal final labels and of equal graph rows (differences come from near ties, decided in FP32 here and
    in FP64 there, and what follows from them in a free-running fit)."""
    import torch

    from paper_1705_01813_gb300 import gkm
    gi_o, L_o, E_o = ora
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    if w.storage == "bf16":
        Xd = Xd.to(torch.bfloat16)  # the sample holds widened BF16 values: exact
    gi, _, _, _ = gkm.build_knn_graph(Xd, w.kappa, w.xi, w.tau, w.max_cluster, w.seed, want_log=False,
                                      precision=precision)
    lab, _, _, log = gkm.kmeans_fit(Xd, k, gi, w.iters, seed=w.seed + 1, precision=precision)
    gi_h, lab_h = gi.cpu().numpy(), lab.cpu().numpy()
    return {"final_distortion_rel_diff": abs(log[-1] - E_o) / E_o,
            "labels_equal": float((lab_h == L_o).mean()),
            "graph_rows_equal": float((gi_h == gi_o).all(1).mean()),
            "precision": precision}


def host_cpu():
    """(model name, logical CPUs) of the host from lscpu, with os.cpu_count() as the fallback."""
    model, cpus = None, os.cpu_count()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and model is None:
                model = v.strip()
            elif k.strip() == "CPU(s)":
                cpus = int(v.strip())
    except (OSError, ValueError, subprocess.SubprocessError):
        pass
    return model, cpus


def time_oracle(O, w, X, threads):
    """The oracle's graph construction + fit on X with `threads` host threads: (seconds, k, results)."""
    used = O.set_threads(threads)
    t0 = time.perf_counter()
    out = _oracle_step(O, w, X)
    return time.perf_counter() - t0, used, out


def cpu_baseline(w, Xh, precision=1):
    """The oracle on the leading rows Xh (FP32; BF16 samples widened) of the workload's samples, timed on all host
    cores and on one (the paper's own setting); then the library on the same rows against the oracle's
    results."""
    from oracle import oracle as O
    ns = Xh.shape[0]
    X = np.ascontiguousarray(Xh, dtype=np.float32)
    model, cpus = host_cpu()
    dt_all, used_all, (k, gi_o, L_o, E_o) = time_oracle(O, w, X, cpus or 1)
    dt_one, _, out_one = time_oracle(O, w, X, 1)
    O.set_threads(cpus or 1)
    assert np.array_equal(out_one[2], L_o)  # the thread count does not change the oracle's results
    dt_b, order_b, state_b, out_b = oracle_boost(O, w, X, gi_o, L_o, k)
    return {"value": ns / dt_all, "unit": "samples/s", "cores": used_all, "kind": "oracle",
            "sample": f"first {ns} samples of {w.name}, k = {k}, k0 = {ns // w.xi}, kappa = {w.kappa}, "
                      f"tau = {w.tau}, iters = {w.iters}: graph construction + fit, FP64 C with OpenMP",
            "seconds": dt_all, "cpu_model": model, "host_cpus": cpus,
            "single_thread": {"value": ns / dt_one, "unit": "samples/s", "cores": 1, "seconds": dt_one},
            "gpu_vs_oracle": gpu_vs_oracle(w, X, k, (gi_o, L_o, E_o), precision),
            "boost_form": {"us_per_visit": round(1e6 * dt_b / ns, 3), "visits": ns, "seconds": dt_b, "cores": 1,
                           "moves": out_b[4],
                           "sample": "one epoch of the move step over a seeded permutation of the sample, from the "
                                     "oracle fit's partition on the oracle's graph (FP64 C, sequential)",
                           "gpu_vs_oracle": gpu_boost_vs_oracle(w, X, gi_o, L_o, k, order_b, state_b, out_b)}}


def run_reference(args):
    """The reference arm: the FP64 oracle (all host cores, OpenMP) on a bounded sample of the workload per step."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    w = datagen.WORKLOADS[args.workload]
    ns = oracle_sample(w, REF_SAMPLE)
    if w.storage == "bf16":  # the recipe drawn on the host for the sample only (BF16 values widened)
        X = datagen.bf16_bits_to_f32(datagen.deep_like(ns, w.d, w.extra["n_dirs"], 50.0, w.seed))
    elif w.name.startswith("gist"):
        X = datagen.gist_like(ns, w.d, w.extra.get("n_latent", 1000), w.seed)
    else:
        X = np.ascontiguousarray(w.data()[:ns])
    model, cpus = host_cpu()
    used = O.set_threads(cpus or 1)
    for _ in range(args.warmup):
        _oracle_step(O, w, X)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        k = _oracle_step(O, w, X)[0]
    dt = time.perf_counter() - t0
    v = ns * args.steps / dt
    drawn = (f"{ns} samples of the {w.name} recipe drawn on the host" if w.storage == "bf16" or
             w.name.startswith("gist") else f"first {ns} samples of {w.name}")
    sample = (f"{drawn} per step, k = {k}, k0 = {ns // w.xi}: graph construction + fit, "
              f"FP64 C oracle with OpenMP on {used} threads ({model})")
    res = {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "n": w.n, "d": w.d, "k": w.k, "kappa": w.kappa, "sample_n": ns},
           "cpu_baseline": {"value": v, "unit": "samples/s", "cores": used, "kind": "oracle", "sample": sample,
                            "cpu_model": model},
           "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def time_tree(gkm, torch, X, w, iters=2, reps=3):
    """The two-means tree (Alg. 1) at the workload's n, d and k: mean time of `reps` calls after one warm-up,
    and the rate of its reads of X ((iters + 1) passes per complete depth).  It is the paper's initial
    partition; the timed step starts from seeded random labels, as the workloads state."""
    n, d = X.shape
    ws = gkm.workspace(gkm.workspace_size(gkm.GK_OP_TREE, n, d, w.k), X.device)
    lab = torch.empty(n, dtype=torch.int32, device=X.device)
    gkm.two_means_tree(X, w.k, iters=iters, seed=w.seed, out=lab, ws=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s = torch.cuda.current_stream()
    e0.record(s)
    for _ in range(reps):
        gkm.two_means_tree(X, w.k, iters=iters, seed=w.seed, out=lab, ws=ws)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    depths = max(w.k, 1).bit_length() - 1  # complete depths; a partial one follows when k is not a power of two
    x_bytes = depths * (iters + 1) * n * d * X.element_size()
    status = gkm.read_status(ws)
    del ws
    return {"ms": round(ms, 3), "k": w.k, "iters": iters, "complete_depths": depths,
            "x_read_GB": round(x_bytes / 1e9, 3), "x_read_GBs": round(x_bytes / ms / 1e6, 1),
            "device_status": status,
            "note": "Alg. 1 initial partition (equal halves, Lloyd 2-means per bisection, FP64 sums); "
                    "not part of the timed step"}


def time_boost(gkm, torch, X, w, gi, labels, visits=100_000):
    """The boost form (Eq. 2 state, Alg. 2's move step with Eq. 3 gains) from the fit's final partition on the
    step's graph: gk_boost_init, then one epoch over the first `visits` entries of a seeded permutation of the
    samples (the visits are sequential by definition, so a prefix gives the per-visit rate of a whole epoch).
    Not part of the timed step."""
    n, d = X.shape
    k, dev = w.k, X.device
    visits = min(visits, n)
    ws = gkm.workspace(gkm.workspace_size(gkm.GK_OP_BOOST, n, d, k, gi.shape[1]), dev)
    L = labels.clone()
    D = torch.empty((k, d), dtype=torch.float64, device=dev)
    cnt = torch.empty(k, dtype=torch.int32, device=dev)
    S = torch.empty(k, dtype=torch.float64, device=dev)
    order = torch.randperm(n, generator=torch.Generator().manual_seed(w.seed + 11))[:visits].to(torch.int32).to(dev)
    gkm.boost_init(X, L, k, D, cnt, S, ws=ws)
    gkm.boost_epoch(X, gi, order[:0], L, k, D, cnt, S, ws=ws)  # first launch: the cluster shape is queried once
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    s = torch.cuda.current_stream()
    e0.record(s)
    gkm.boost_init(X, L, k, D, cnt, S, ws=ws)
    e1.record(s)
    ne = cnt > 0
    I0 = float((S[ne] / cnt[ne]).sum())
    e1b = torch.cuda.Event(enable_timing=True)
    e1b.record(s)
    mv = gkm.boost_epoch(X, gi, order, L, k, D, cnt, S, ws=ws)
    e2.record(s)
    torch.cuda.synchronize()
    ms = e1b.elapsed_time(e2)
    ne = cnt > 0
    I1 = float((S[ne] / cnt[ne]).sum())
    status = gkm.read_status(ws)
    out = {"visits": visits, "epoch_prefix_ms": round(ms, 3), "us_per_visit": round(1e3 * ms / visits, 3),
           "visits_per_s": round(visits / ms * 1e3, 1), "moves": int(mv.item()),
           "init_ms": round(e0.elapsed_time(e1), 3), "projected_epoch_s": round(n * ms / visits / 1e3, 2),
           "objective_I_gain_per_sample": (I1 - I0) / n, "device_status": status,
           "note": "one thread-block cluster walks the visits in order (FP64, bit-equal to the oracle); the "
                   "partition is the fit's final one and the graph the step's; not part of the timed step"}
    del ws, D, S, cnt, L
    return out


def oracle_boost(O, w, X, gi, L, k):
    """The oracle's boost form on a sample (its graph and its fit's labels), one epoch over a seeded permutation
    of the sample: (seconds of the epoch, visits, the final state)."""
    ns = X.shape[0]
    order = np.random.default_rng(w.seed + 11).permutation(ns).astype(np.int32)
    D, cnt, S = O.boost_init(X, L, k)
    t0 = time.perf_counter()
    out = O.boost_epoch(X, gi, order, L, k, D, cnt, S)
    return time.perf_counter() - t0, order, (D, cnt, S), out


def gpu_boost_vs_oracle(w, X, gi, L, k, order, state0, ora_out):
    """The library's boost epoch on the oracle's sample from the same state and visits: equal bit for bit?"""
    import torch

    from paper_1705_01813_gb300 import gkm
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    if w.storage == "bf16":
        Xd = Xd.to(torch.bfloat16)  # the sample holds widened BF16 values: exact
    Ld = torch.from_numpy(np.ascontiguousarray(L, dtype=np.int32)).cuda()
    D, cnt, S = gkm.boost_init(Xd, Ld, k)
    init_equal = all(np.array_equal(a.cpu().numpy(), b) for a, b in zip((D, cnt, S), state0))
    mv = gkm.boost_epoch(Xd, torch.from_numpy(np.ascontiguousarray(gi, dtype=np.int32)).cuda(),
                         torch.from_numpy(order).cuda(), Ld, k, D, cnt, S)
    Lo, Do, co, So, mo, _ = ora_out
    equal = (np.array_equal(Ld.cpu().numpy(), Lo) and np.array_equal(D.cpu().numpy(), Do)
             and np.array_equal(cnt.cpu().numpy(), co) and np.array_equal(S.cpu().numpy(), So))
    return {"init_state_equal": init_equal, "epoch_state_equal": equal, "moves": int(mv.item()), "oracle_moves": mo}


def main():
    args = parse()
    if args.traffic_from:
        write_traffic(args.traffic_from, args.workload)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
