"""Serving loop: a job's result is the same alone and among others, admission keeps the HBM budget and
the slot count, and the latency summary is what it says."""
import numpy as np
import pytest

from paper_1705_01813_gb300 import serve


def _specs(sizes, arrival_gap=0.0):
    return [serve.JobSpec(i, i * arrival_gap, n, d, max(1, n // 100), 20, 1000 + i) for i, (n, d) in enumerate(sizes)]


def _peak_in_flight(res):
    events = sorted([(r.start, 1) for r in res] + [(r.end, -1) for r in res], key=lambda e: (e[0], e[1]))
    live = peak = 0
    for _, dv in events:
        live += dv
        peak = max(peak, live)
    return peak


def test_summary_percentiles_and_rate():
    res = [serve.JobResult(i, arrival=0.1 * i, start=0.1 * i, end=0.1 * i + 0.01 * (i + 1), n=100, d=8, k=1,
                           distortion=1.0) for i in range(100)]
    s = serve.summarize(res)
    assert s["jobs"] == 100 and s["samples"] == 10000
    # latency of job i is 10 (i + 1) ms; the q-quantile is the entry at index round(q (count - 1))
    assert abs(s["p50_ms"] - 10 * (round(0.5 * 99) + 1)) < 1e-6
    assert abs(s["p99_ms"] - 10 * (round(0.99 * 99) + 1)) < 1e-6
    assert abs(s["span_s"] - (9.9 + 1.0)) < 1e-9 and abs(s["jobs_per_s"] - 100 / 10.9) < 1e-9


def test_job_bytes_grows_with_the_job():
    p = serve.ServeParams()
    a, b, c = _specs([(10000, 64), (20000, 64), (20000, 128)])
    assert serve.job_bytes(a, p) < serve.job_bytes(b, p) < serve.job_bytes(c, p)
    assert serve.job_bytes(b, p) >= 20000 * 64 * 4 + 20000 * 20 * 8  # samples and graph at least


@pytest.mark.gpu
def test_result_alone_equals_result_in_the_mix():
    import torch
    specs = _specs([(12000, 64), (30011, 128), (15000, 256), (20000, 64), (10007, 128), (25000, 256)])
    keep = serve.ServeParams(slots=4, keep_results=True)
    mix = serve.Server(keep).run(specs, realtime=False)
    assert _peak_in_flight(mix) >= 2  # the jobs did overlap
    for s, rm in zip(specs, mix):
        ra = serve.Server(serve.ServeParams(slots=1, keep_results=True)).run([s], realtime=False)[0]
        assert torch.equal(ra.labels, rm.labels) and torch.equal(ra.centroids, rm.centroids)
        assert ra.distortion == rm.distortion
        assert rm.labels.shape == (s.n,) and rm.centroids.shape == (s.k, s.d)
        assert np.isfinite(rm.distortion) and rm.distortion > 0


@pytest.mark.gpu
def test_admission_keeps_budget_and_slots():
    specs = _specs([(20000, 128)] * 6)
    p = serve.ServeParams(slots=4)
    p.budget_bytes = 2 * serve.job_bytes(specs[0], p) + 1  # room for two of them
    res = serve.Server(p).run(specs, realtime=False)
    assert _peak_in_flight(res) <= 2
    with pytest.raises(ValueError):
        serve.Server(serve.ServeParams(budget_bytes=1)).run(specs[:1], realtime=False)


@pytest.mark.gpu
def test_admission_counts_the_arenas_the_slots_hold():
    """The budget bounds what the slots' arenas hold, idle or not: after two big jobs grew two arenas, small jobs
    reuse those or wait, and never make the arenas hold more than the budget."""
    big = _specs([(40000, 128)] * 2)
    small = [serve.JobSpec(10 + i, 0.0, 20000, 64, 200, 20, 2000 + i) for i in range(6)]
    p = serve.ServeParams(slots=4)
    p.budget_bytes = 2 * serve.job_bytes(big[0], p) + serve.job_bytes(small[0], p) // 2
    srv = serve.Server(p)
    srv.run(big, realtime=False)
    assert sum(a.capacity for a in srv.arenas) == 2 * serve.job_bytes(big[0], p)
    res = srv.run(small, realtime=False)
    assert len(res) == 6 and _peak_in_flight(res) <= 2
    assert srv.max_held <= p.budget_bytes
    assert sum(a.capacity for a in srv.arenas) <= p.budget_bytes
    # a job that needs a larger arena makes the server release an idle one first
    p2 = serve.ServeParams(slots=2, budget_bytes=serve.job_bytes(big[0], p) + serve.job_bytes(small[0], p) // 2)
    srv2 = serve.Server(p2)
    srv2.run(small[:2], realtime=False)
    assert sorted(a.capacity for a in srv2.arenas) == [serve.job_bytes(small[0], p)] * 2
    srv2.run(big[:1], realtime=False)
    assert srv2.max_held <= p2.budget_bytes
    assert sorted(a.capacity for a in srv2.arenas) == [0, serve.job_bytes(big[0], p)]


@pytest.mark.gpu
def test_stream_latency_counts_from_arrival():
    specs = _specs([(10000, 64)] * 4, arrival_gap=0.05)
    res = serve.Server(serve.ServeParams(slots=2)).run(specs, realtime=True)
    for s, r in zip(specs, res):
        assert r.start >= s.arrival - 1e-3 and r.end > r.start and abs(r.latency - (r.end - s.arrival)) < 1e-12


@pytest.mark.gpu
def test_batched_jobs_equal_jobs_alone():
    """Jobs of one row width concatenated into one problem (shifted graph ids and labels) give each job
    the labels and centroids it gets alone through the one-call library API."""
    import torch
    specs = _specs([(12000, 64), (15013, 128), (20000, 64), (10007, 128), (9000, 64), (30011, 128)])
    pb = serve.ServeParams(slots=2, keep_results=True, batching=True)
    batched = serve.Server(pb).run(specs, realtime=False)
    assert len({r.end for r in batched}) < len(specs)  # some jobs completed together, in one batch
    for s, rb in zip(specs, batched):
        ra = serve.Server(serve.ServeParams(slots=1, keep_results=True)).run([s], realtime=False)[0]
        assert torch.equal(ra.labels, rb.labels) and torch.equal(ra.centroids, rb.centroids)
        assert abs(rb.distortion - ra.distortion) <= 1e-9 * abs(ra.distortion)


@pytest.mark.gpu
def test_batch_rejects_mixed_widths():
    import torch
    with pytest.raises(ValueError):
        serve.run_batch(_specs([(1000, 64), (1000, 128)]), serve.ServeParams(), torch.device("cuda", 0),
                        torch.cuda.current_stream())


@pytest.mark.gpu
def test_arena_run_equals_allocating_run():
    """A job whose tensors come from a slot arena (reused by an earlier, different job) gives the same
    results as the job with tensors from torch's allocator."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    p = serve.ServeParams()
    arena = serve.Arena(dev)
    first, second = _specs([(30011, 128), (12007, 64)])
    serve.run_job(first, p, dev, stream, arena)  # leaves its contents in the arena
    Ea, la, Ca = serve.run_job(second, p, dev, stream, arena)
    Eb, lb, Cb = serve.run_job(second, p, dev, stream)
    stream.synchronize()
    assert torch.equal(la, lb) and torch.equal(Ca, Cb) and Ea == Eb
    assert arena.buf.numel() >= serve.job_bytes(first, p)


@pytest.mark.gpu
def test_injected_job_failure_is_raised_and_the_server_recovers(monkeypatch):
    """A failure injected on the host into one job (an allocation failure) ends the run with that error; the
    slots and the budget are released, so the same server serves the next run."""
    specs = _specs([(10000, 64)] * 6)
    real = serve.run_job

    def flaky(s, p, device, stream, arena=None):
        if s.jid == 3:
            raise MemoryError("injected allocation failure")
        return real(s, p, device, stream, arena)

    monkeypatch.setattr(serve, "run_job", flaky)
    srv = serve.Server(serve.ServeParams(slots=2))
    with pytest.raises(MemoryError, match="injected"):
        srv.run(specs, realtime=False)
    monkeypatch.setattr(serve, "run_job", real)
    res = srv.run(specs[:3], realtime=False)
    assert [r.jid for r in res] == [0, 1, 2] and all(np.isfinite(r.distortion) for r in res)
