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

With batching, the jobs waiting at a dispatch that share the head job's row
width and kappa run together as one concatenated problem (run_batch): each
kernel launch then serves all of them, which amortises launches over small
jobs; a batch's jobs complete together.

Each slot owns an arena (one device buffer, as large as the largest job or
batch the slot has run) from which a job takes all its tensors, so serving
makes no device allocation per job.  The loop itself is host code over the C
ABI: one host thread per slot, each blocked in a library call (the ctypes call
releases the interpreter lock) while its stream runs.
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
    batching: bool = False         # run eligible jobs of one (d, kappa) together (run_batch)
    max_batch_jobs: int = 64
    max_batch_samples: int = 4_000_000


def job_specs(jobs: list[dict]) -> list[JobSpec]:
    """JobSpec list from datagen.serving_jobs-style dicts, in arrival order."""
    out = [JobSpec(i, j["arrival"], j["n"], j["d"], j["k"], j["kappa"], j["seed"]) for i, j in enumerate(jobs)]
    return sorted(out, key=lambda s: (s.arrival, s.jid))


def job_ws_bytes(s: JobSpec, p: ServeParams) -> int:
    return max(gkm.workspace_size_build(s.n, s.d, s.kappa, p.xi, p.tau, p.max_cluster),
               gkm.workspace_size(gkm.GK_OP_FIT, s.n, s.d, s.k, s.kappa))


def job_bytes(s: JobSpec, p: ServeParams) -> int:
    """Device bytes a job holds while it runs (what run_job takes from its slot's arena)."""
    f32 = 4
    data = s.n * s.d * f32 + 8 * s.n  # samples, mixture components while they are drawn
    graph = s.n * s.kappa * 8
    labels = 2 * s.n * 4
    cent = s.k * s.d * f32 + s.k * 4
    return data + graph + labels + cent + job_ws_bytes(s, p) + 16 * 256


class Arena:
    """A slot's device memory: one byte buffer, allocated when the slot first needs it (and grown when a
    larger job comes), from which a job takes its tensors with a bump pointer reset for every job.  A
    serving run thus makes no device allocation per job (allocations and frees of the caching allocator
    can synchronise the whole device)."""

    def __init__(self, device):
        self.device = device
        self.buf = None
        self.off = 0

    @property
    def capacity(self) -> int:
        """Bytes this arena holds on the device."""
        return 0 if self.buf is None else int(self.buf.numel())

    def release(self):
        """Give the buffer up (the caller returns it to the device with torch.cuda.empty_cache())."""
        self.buf = None
        self.off = 0

    def reset(self, nbytes: int):
        if self.buf is None or self.buf.numel() < nbytes:
            replaced = self.buf is not None
            self.buf = None
            if replaced:  # the smaller buffer goes back to the device, not to the allocator's cache
                torch.cuda.empty_cache()
            self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        self.off = 0

    def take(self, shape, dtype) -> torch.Tensor:
        numel = 1
        for v in shape:
            numel *= int(v)
        nb = numel * torch.empty((), dtype=dtype).element_size()
        off = (self.off + 255) & ~255
        if off + nb > self.buf.numel():
            raise MemoryError(f"arena of {self.buf.numel()} bytes cannot hold {nb} more at {off}")
        self.off = off + nb
        return self.buf[off:off + nb].view(dtype).view(tuple(int(v) for v in shape))

    def workspace(self, nbytes: int, stream) -> gkm.Workspace:
        return gkm.Workspace.from_buffer(self.take((max(256, int(nbytes)),), torch.uint8), stream)


def job_data(s: JobSpec, device, out=None, z_out=None) -> torch.Tensor:
    """The job's samples: a mixture of n/100 unit Gaussians in [-10, 10]^d (seeded, generated on the device)."""
    return datagen.gauss_mixture_device(s.n, s.d, max(1, s.n // 100), s.seed, device, out=out, z_out=z_out)


def _device(device) -> torch.device:
    dev = torch.device(device or "cuda")
    return dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())


def run_job(s: JobSpec, p: ServeParams, device, stream: torch.cuda.Stream, arena: Arena | None = None):
    """One job on `stream`: samples, graph (Alg. 3), fit (Alg. 2); returns (final distortion, labels, centroids).
    With an arena every tensor of the job comes from it (the results too: copy them before the arena's next
    job); without one they come from torch's allocator."""
    i32, f32 = torch.int32, torch.float32
    with torch.cuda.stream(stream):
        if arena is None:
            X = job_data(s, device)
            gi, _, _, _ = gkm.build_knn_graph(X, s.kappa, xi=p.xi, tau=p.tau, max_cluster=p.max_cluster,
                                              seed=s.seed, want_log=False, precision=p.precision, stream=stream)
            L0 = gkm.init_labels(s.n, s.k, s.seed + 1, stream=stream)
            labels, C, _, log = gkm.kmeans_fit(X, s.k, gi, p.iters, init_labels=L0, precision=p.precision,
                                               stream=stream)
            return log[-1], labels, C
        arena.reset(job_bytes(s, p))
        X = arena.take((s.n, s.d), f32)
        job_data(s, device, out=X, z_out=arena.take((s.n,), torch.int64))
        gi, gd = arena.take((s.n, s.kappa), i32), arena.take((s.n, s.kappa), f32)
        lab0, labels = arena.take((s.n,), i32), arena.take((s.n,), i32)
        C, cnt = arena.take((s.k, s.d), f32), arena.take((s.k,), i32)
        ws = arena.workspace(job_ws_bytes(s, p), stream)
        gkm.build_knn_graph(X, s.kappa, xi=p.xi, tau=p.tau, max_cluster=p.max_cluster, seed=s.seed,
                            labels_out=lab0, g_idx=gi, g_dist=gd, want_log=False, precision=p.precision, ws=ws,
                            stream=stream)
        gkm.init_labels(s.n, s.k, s.seed + 1, out=lab0, stream=stream)
        _, _, _, log = gkm.kmeans_fit(X, s.k, gi, p.iters, init_labels=lab0, labels_out=labels, C_out=C,
                                      counts_out=cnt, precision=p.precision, ws=ws, stream=stream)
    return log[-1], labels, C


def build_k0(n: int, xi: int) -> int:
    """Clusters of the graph construction (the library's rule): floor(n / xi), at least 1."""
    return max(1, n // xi)


def _batch_jobs(specs: list[JobSpec]) -> list[tuple]:
    """gk_batch_fit's job table: (n, k, graph seed, fit seed); a job's fit starts from init_labels(seed + 1) as in
    run_job."""
    return [(s.n, s.k, s.seed, s.seed + 1) for s in specs]


def _batch_ws_bytes(specs: list[JobSpec], p: ServeParams) -> int:
    return gkm.workspace_size_batch(specs[0].d, _batch_jobs(specs), specs[0].kappa, p.xi, p.tau, p.max_cluster,
                                    p.precision)


def batch_bytes(specs: list[JobSpec], p: ServeParams) -> int:
    """Device bytes of a batch (what run_batch takes from its slot's arena)."""
    N, K = sum(s.n for s in specs), sum(s.k for s in specs)
    d, kappa = specs[0].d, specs[0].kappa
    return (N * d * 4 + 8 * max(s.n for s in specs) + N * kappa * 8 + N * 4 + K * d * 4 + 8 * len(specs)
            + _batch_ws_bytes(specs, p) + 16 * 256)


def run_batch(specs: list[JobSpec], p: ServeParams, device, stream: torch.cuda.Stream, arena: Arena | None = None):
    """Jobs of one row width d and one kappa as one problem, through the library's batched call (gk_batch_fit):
    their samples are concatenated, each kernel launch serves all of them, and each job gets the graph, labels,
    centroids and distortion it gets alone, bit for bit (the library numbers each job's rows and clusters after
    the jobs before it and draws its random start on its own rows).  All tensors come from `arena` (a private
    one when none is given).  Returns [(distortion, labels, centroids)], the last two views into the arena."""
    d, kappa = specs[0].d, specs[0].kappa
    if any(s.d != d or s.kappa != kappa for s in specs):
        raise ValueError("a batch holds jobs of one row width and one kappa")
    if len(specs) > gkm.MAX_BATCH_JOBS:
        raise ValueError(f"a batch holds at most {gkm.MAX_BATCH_JOBS} jobs")
    N, K = sum(s.n for s in specs), sum(s.k for s in specs)
    i32, f32 = torch.int32, torch.float32
    arena = arena or Arena(device)
    with torch.cuda.stream(stream):
        arena.reset(batch_bytes(specs, p))
        X = arena.take((N, d), f32)
        z = arena.take((max(s.n for s in specs),), torch.int64)
        gi, gd = arena.take((N, kappa), i32), arena.take((N, kappa), f32)
        lab = arena.take((N,), i32)
        C = arena.take((K, d), f32)
        dist = arena.take((len(specs),), torch.float64)
        ws = arena.workspace(_batch_ws_bytes(specs, p), stream)
        first = 0
        for s in specs:  # each job's samples, generated on its own rows
            job_data(s, device, out=X[first:first + s.n], z_out=z[:s.n])
            first += s.n
        gkm.batch_fit(X, _batch_jobs(specs), kappa, xi=p.xi, tau=p.tau, max_cluster=p.max_cluster, iters=p.iters,
                      precision=p.precision, g_idx=gi, g_dist=gd, labels_out=lab, C_out=C, distortion=dist, ws=ws,
                      stream=stream)
    stream.synchronize()
    E = dist.cpu().tolist()
    out, first, kfirst = [], 0, 0
    for j, s in enumerate(specs):
        out.append((E[j], lab[first:first + s.n], C[kfirst:kfirst + s.k]))
        first += s.n
        kfirst += s.k
    return out


class Server:
    """Admits jobs by HBM budget and slots, runs each on its own stream, records latencies.

    The budget bounds the device memory the slots' arenas hold, idle or not: a job (or batch) is admitted to a
    free slot only when the arenas, with that slot's grown to the job's size, fit in the budget; idle slots'
    arenas are released (largest first) to make room, and a replaced or released buffer goes back to the
    device.  `max_held` is the most the arenas held at once over the server's runs."""

    def __init__(self, params: ServeParams | None = None, device=None):
        self.p = params or ServeParams()
        self.device = _device(device)
        self.arenas: list[Arena] = []  # one per slot, kept across runs
        self.max_held = 0
        gkm.load()

    def run(self, specs: list[JobSpec], realtime: bool = True) -> list[JobResult]:
        """Serve `specs` (arrival-ordered).  realtime: jobs become eligible at their arrival times;
        otherwise all are eligible at once (a saturation run).  Returns one result per job."""
        p = self.p
        for s in specs:
            need = batch_bytes([s], p) if p.batching else job_bytes(s, p)
            if need > p.budget_bytes:
                raise ValueError(f"job {s.jid} needs {need} bytes, more than the budget")
        lock = threading.Condition()
        state = {"inflight": 0, "error": None}
        results: dict[int, JobResult] = {}
        streams = [torch.cuda.Stream(device=self.device) for _ in range(p.slots)]
        while len(self.arenas) < p.slots:
            self.arenas.append(Arena(self.device))
        held = [a.capacity for a in self.arenas]  # bytes each slot's arena holds or is about to hold
        free_streams = list(range(p.slots))
        t0 = time.perf_counter()

        def worker(batch: list[JobSpec], si: int, start: float):
            try:
                torch.cuda.set_device(self.device)
                if p.batching:
                    outs = run_batch(batch, p, self.device, streams[si], self.arenas[si])
                else:
                    outs = [run_job(batch[0], p, self.device, streams[si], self.arenas[si])]
                if p.keep_results:  # out of the slot's arena before its next job
                    with torch.cuda.stream(streams[si]):
                        outs = [(E, lab.clone(), C.clone()) for E, lab, C in outs]
                    streams[si].synchronize()
                end = time.perf_counter() - t0
                res = [JobResult(s.jid, s.arrival if realtime else 0.0, start, end, s.n, s.d, s.k, E,
                                 labels if p.keep_results else None, C if p.keep_results else None)
                       for s, (E, labels, C) in zip(batch, outs)]
                del outs
            except BaseException as e:  # reported by run(); the slot and budget are released
                res = None
                with lock:
                    state["error"] = state["error"] or e
            with lock:
                for r in res or []:
                    results[r.jid] = r
                state["inflight"] -= 1
                free_streams.append(si)
                lock.notify_all()

        def next_batch(now: float) -> list[JobSpec]:
            """The head job, and with batching the eligible jobs of its (d, kappa) after it."""
            head = queue[0]
            if not p.batching:
                return [head]
            out, total = [], 0
            for s in queue:
                if realtime and s.arrival > now:
                    break
                if (s.d, s.kappa) != (head.d, head.kappa):
                    continue
                if out and (len(out) >= p.max_batch_jobs or total + s.n > p.max_batch_samples):
                    break
                out.append(s)
                total += s.n
            return out

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
                batch = next_batch(now)
                nbytes = batch_bytes(batch, p) if p.batching else job_bytes(s, p)
                if state["inflight"] >= p.slots:
                    lock.wait(timeout=0.05)
                    continue
                # the free slot whose arena already holds the job (the smallest such), else the largest one
                fits = [j for j in free_streams if held[j] >= nbytes]
                si = min(fits, key=lambda j: held[j]) if fits else max(free_streams, key=lambda j: held[j])
                need = sum(held) - held[si] + max(held[si], nbytes)
                if need > p.budget_bytes:
                    released = False
                    for sj in sorted((j for j in free_streams if j != si and held[j] > 0), key=lambda j: -held[j]):
                        if need <= p.budget_bytes:
                            break
                        self.arenas[sj].release()
                        need -= held[sj]
                        held[sj] = 0
                        released = True
                    if released:
                        torch.cuda.empty_cache()
                    if need > p.budget_bytes:
                        lock.wait(timeout=0.05)
                        continue
                held[si] = max(held[si], nbytes)
                self.max_held = max(self.max_held, sum(held))
                for b in batch:
                    queue.remove(b)
                state["inflight"] += 1
                free_streams.remove(si)
                th = threading.Thread(target=worker, args=(batch, si, now), daemon=True)
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
    arena = Arena(device)
    out = []
    t0 = time.perf_counter()
    for s in specs:
        start = time.perf_counter() - t0
        E, labels, C = run_job(s, params, device, stream, arena)
        if params.keep_results:
            with torch.cuda.stream(stream):
                labels, C = labels.clone(), C.clone()
            stream.synchronize()
        end = time.perf_counter() - t0
        out.append(JobResult(s.jid, 0.0, start, end, s.n, s.d, s.k, E,
                             labels if params.keep_results else None, C if params.keep_results else None))
    return out
