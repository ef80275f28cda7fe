"""Serving loop for clustering jobs: each job builds its KNN graph by the fast
k-means itself (Alg. 3) and then runs the graph-guided k-means (Alg. 2 with the
closest-centroid rule of Sec. 4.2) on it.

Jobs arrive over time with their own n, d, k.  A job is admitted in arrival
order as soon as a slot is free and its device footprint (samples, graph,
labels, centroids and the library's workspace) fits in the HBM budget; it then
runs on its own CUDA stream, so admitted jobs overlap on the GPU (continuous
batching: a job that arrives while others run starts as soon as memory and a
slot free up).  Everything a job touches stays resident on the device for its
life; the host only issues the two library calls (each a whole pipeline of
kernels) and reads back the distortion log at the end.  Results do not depend
on what else runs: every kernel is deterministic and each job has its own
workspace and stream.

The loop itself is host code over the C ABI: one host thread per slot, each
blocked in a library call (the ctypes call releases the interpreter lock)
while its stream runs.
"""
from __future__ import annotations

import dataclasses
import threading
import time

import torch

from . import datagen, gkm


@dataclasses.dataclass
class JobSpec:
    jid: int
    arrival: float  # seconds after the start of the run
    n: int
    d: int
    k: int
    kappa: int
    seed: int


@dataclasses.dataclass
class JobResult:
    jid: int
    arrival: float
    start: float      # admission time
    end: float        # completion time (host saw the job's stream finish)
    n: int
    d: int
    k: int
    distortion: float  # final distortion of the fit (Eq. 4, mean squared distance)
    labels: torch.Tensor | None = None
    centroids: torch.Tensor | None = None

    @property
    def latency(self) -> float:
        return self.end - self.arrival


@dataclasses.dataclass
class ServeParams:
    budget_bytes: int = 120 << 30  # HBM the jobs may hold at once
    slots: int = 8                 # jobs in flight at most (streams / host threads)
    precision: int = 1
    xi: int = 50
    tau: int = 10
    iters: int = 10
    max_cluster: int = 128
    keep_results: bool = False     # keep each job's labels and centroids (device) in its result


def job_specs(jobs: list[dict]) -> list[JobSpec]:
    """JobSpec list from datagen.serving_jobs-style dicts, in arrival order."""
    out = [JobSpec(i, j["arrival"], j["n"], j["d"], j["k"], j["kappa"], j["seed"]) for i, j in enumerate(jobs)]
    return sorted(out, key=lambda s: (s.arrival, s.jid))


def job_bytes(s: JobSpec, p: ServeParams) -> int:
    """Device bytes a job holds while it runs."""
    f32 = 4
    data = s.n * s.d * f32
    graph = s.n * s.kappa * 8
    labels = 2 * s.n * 4
    cent = s.k * s.d * f32 + s.k * 4
    ws_build = gkm.workspace_size_build(s.n, s.d, s.kappa, p.xi, p.tau, p.max_cluster)
    ws_fit = gkm.workspace_size(gkm.GK_OP_FIT, s.n, s.d, s.k, s.kappa)
    return data + graph + labels + cent + max(ws_build, ws_fit) + (1 << 20)


def job_data(s: JobSpec, device) -> torch.Tensor:
    """The job's samples: a mixture of n/100 unit Gaussians in [-10, 10]^d (seeded, generated on the device)."""
    return datagen.gauss_mixture_device(s.n, s.d, max(1, s.n // 100), s.seed, device)


def _device(device) -> torch.device:
    dev = torch.device(device or "cuda")
    return dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())


def run_job(s: JobSpec, p: ServeParams, device, stream: torch.cuda.Stream):
    """One job on `stream`: samples, graph (Alg. 3), fit (Alg. 2); returns (final distortion, labels, centroids)."""
    with torch.cuda.stream(stream):
        X = job_data(s, device)
        gi, _, _, _ = gkm.build_knn_graph(X, s.kappa, xi=p.xi, tau=p.tau, max_cluster=p.max_cluster, seed=s.seed,
                                          want_log=False, precision=p.precision, stream=stream)
        L0 = gkm.init_labels(s.n, s.k, s.seed + 1, stream=stream)
        labels, C, _, log = gkm.kmeans_fit(X, s.k, gi, p.iters, init_labels=L0, precision=p.precision,
                                           stream=stream)
        del X, gi, L0
    return log[-1], labels, C


class Server:
    """Admits jobs by HBM budget and slots, runs each on its own stream, records latencies."""

    def __init__(self, params: ServeParams | None = None, device=None):
        self.p = params or ServeParams()
        self.device = _device(device)
        gkm.load()

    def run(self, specs: list[JobSpec], realtime: bool = True) -> list[JobResult]:
        """Serve `specs` (arrival-ordered).  realtime: jobs become eligible at their arrival times;
        otherwise all are eligible at once (a saturation run).  Returns one result per job."""
        p = self.p
        for s in specs:
            if job_bytes(s, p) > p.budget_bytes:
                raise ValueError(f"job {s.jid} needs {job_bytes(s, p)} bytes, more than the budget")
        lock = threading.Condition()
        state = {"used": 0, "inflight": 0, "error": None}
        results: dict[int, JobResult] = {}
        streams = [torch.cuda.Stream(device=self.device) for _ in range(p.slots)]
        free_streams = list(range(p.slots))
        t0 = time.perf_counter()

        def worker(s: JobSpec, si: int, start: float, nbytes: int):
            try:
                torch.cuda.set_device(self.device)
                E, labels, C = run_job(s, p, self.device, streams[si])
                end = time.perf_counter() - t0
                res = JobResult(s.jid, s.arrival if realtime else 0.0, start, end, s.n, s.d, s.k, E,
                                labels if p.keep_results else None, C if p.keep_results else None)
                del labels, C
            except BaseException as e:  # reported by run(); the slot and budget are released
                res = None
                with lock:
                    state["error"] = state["error"] or e
            with lock:
                if res is not None:
                    results[s.jid] = res
                state["used"] -= nbytes
                state["inflight"] -= 1
                free_streams.append(si)
                lock.notify_all()

        threads = []
        queue = list(specs)
        with lock:
            while queue:
                if state["error"] is not None:
                    break
                s = queue[0]
                now = time.perf_counter() - t0
                if realtime and s.arrival > now:
                    lock.wait(timeout=s.arrival - now)
                    continue
                nbytes = job_bytes(s, p)
                if state["inflight"] >= p.slots or state["used"] + nbytes > p.budget_bytes:
                    lock.wait(timeout=0.05)
                    continue
                queue.pop(0)
                state["used"] += nbytes
                state["inflight"] += 1
                si = free_streams.pop()
                th = threading.Thread(target=worker, args=(s, si, now, nbytes), daemon=True)
                th.start()
                threads.append(th)
        for th in threads:
            th.join()
        if state["error"] is not None:
            raise state["error"]
        return [results[s.jid] for s in specs]


def summarize(results: list[JobResult]) -> dict:
    """p50 / p99 latency (ms), jobs/s over the span from the first arrival to the last completion."""
    lat = sorted(r.latency for r in results)

    def pct(q):
        i = min(len(lat) - 1, max(0, int(round(q * (len(lat) - 1)))))
        return lat[i] * 1e3

    span = max(r.end for r in results) - min(r.arrival for r in results)
    return {"jobs": len(results), "jobs_per_s": len(results) / span, "p50_ms": pct(0.50), "p99_ms": pct(0.99),
            "samples": int(sum(r.n for r in results)), "span_s": span}


def run_serial(specs: list[JobSpec], params: ServeParams, device=None) -> list[JobResult]:
    """The per-job form: one job at a time on one stream, all eligible at t = 0."""
    device = _device(device)
    stream = torch.cuda.Stream(device=device)
    out = []
    t0 = time.perf_counter()
    for s in specs:
        start = time.perf_counter() - t0
        E, labels, C = run_job(s, params, device, stream)
        end = time.perf_counter() - t0
        out.append(JobResult(s.jid, 0.0, start, end, s.n, s.d, s.k, E,
                             labels if params.keep_results else None, C if params.keep_results else None))
    return out
