"""Batches of independent jobs (gk_batch_fit): every job's graph rows, labels, centroids and final distortion
equal what the one-call API gives for that job alone, bit for bit; and the host checks refuse bad job tables
before anything reaches a device."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1705_01813_gb300 import build_native, datagen, gkm  # noqa: E402

KAPPA, XI, TAU, CAP, ITERS = 12, 50, 4, 128, 5


def _jobs(sizes, seed0=100):
    return [(n, max(1, n // 40), seed0 + 3 * j, seed0 + 3 * j + 1) for j, n in enumerate(sizes)]


def _data(sizes, d):
    return [datagen.gauss_mixture(n, d, max(2, n // 60), seed=7 + j) for j, n in enumerate(sizes)]


@pytest.mark.gpu
@pytest.mark.parametrize("d,precision", [(24, 0), (64, 1), (128, 1), (40, 2)])
def test_batch_equals_jobs_alone(d, precision):
    sizes = [3001, 517, 12000, 64, 2048]
    jobs = _jobs(sizes)
    Xs = _data(sizes, d)
    X = torch.from_numpy(np.concatenate(Xs)).cuda()
    gi, gd, lab, C, dist = gkm.batch_fit(X, jobs, KAPPA, xi=XI, tau=TAU, max_cluster=CAP, iters=ITERS,
                                         precision=precision)
    torch.cuda.synchronize()
    first = kfirst = 0
    for (n, k, gs, fs), Xj in zip(jobs, Xs):
        xj = torch.from_numpy(Xj).cuda()
        gi1, gd1, _, _ = gkm.build_knn_graph(xj, KAPPA, xi=XI, tau=TAU, max_cluster=CAP, seed=gs, want_log=False,
                                             precision=precision)
        L0 = gkm.init_labels(n, k, fs)
        lab1, C1, _, log = gkm.kmeans_fit(xj, k, gi1, ITERS, init_labels=L0, precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(gi[first:first + n] - first, gi1) and torch.equal(gd[first:first + n], gd1)
        assert torch.equal(lab[first:first + n], lab1)
        assert torch.equal(C[kfirst:kfirst + k], C1)
        assert dist[jobs.index((n, k, gs, fs))].item() == log[-1]
        first += n
        kfirst += k


@pytest.mark.gpu
def test_batch_bf16_samples_and_replay():
    sizes = [2000, 3333]
    jobs = _jobs(sizes, seed0=9)
    X = torch.from_numpy(np.concatenate(_data(sizes, 64))).cuda().to(torch.bfloat16)
    a = gkm.batch_fit(X, jobs, KAPPA, xi=XI, tau=TAU, iters=ITERS, precision=1)
    torch.cuda.synchronize()
    ref = [t.clone() for t in a]
    # the same request replayed as a captured CUDA graph gives the same bits
    gkm.set_replay(True)
    try:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for _ in range(3):
                b = gkm.batch_fit(X, jobs, KAPPA, xi=XI, tau=TAU, iters=ITERS, precision=1, g_idx=a[0], g_dist=a[1],
                                  labels_out=a[2], C_out=a[3], distortion=a[4], stream=s)
        s.synchronize()
    finally:
        gkm.set_replay(False)
    assert all(torch.equal(x, y) for x, y in zip(b, ref))


def test_batch_argument_checks():
    build_native.build()
    if torch.cuda.is_available():
        pytest.skip("argument checks with fake pointers run on CPU-only hosts")
    L = gkm.load()
    P, ws = ctypes.c_void_p(0x10000000), ctypes.c_void_p(0x20000000)
    p = gkm.GraphParams(8, 50, 3, 128, 0, 0, 0)

    def call(jobs, n_jobs=None, iters=2):
        arr = gkm._jobs(jobs)
        return L.gk_batch_fit(P, 16, 16, len(jobs) if n_jobs is None else n_jobs, ctypes.cast(arr, ctypes.c_void_p),
                              ctypes.byref(p), iters, P, P, P, P, P, ws, 1 << 30, None)

    assert call([(100, 4, 1, 2)] * 65) == gkm.GK_ERR_INVALID                 # more than GK_MAX_BATCH_JOBS
    assert call([(100, 4, 1, 2)], n_jobs=0) == gkm.GK_ERR_INVALID
    assert call([(100, 4, 1, 2), (8, 2, 1, 2)]) == gkm.GK_ERR_INVALID        # kappa >= n of the second job
    assert b"job 1" in L.gk_last_error()
    assert call([(100, 0, 1, 2)]) == gkm.GK_ERR_INVALID                      # k < 1
    assert call([(100, 4, 1, 2)], iters=-1) == gkm.GK_ERR_INVALID
    assert gkm.workspace_size_batch(16, [(100, 4, 1, 2)] * 65, 8) == 0
    assert gkm.workspace_size_batch(16, [(100, 4, 1, 2)], 8) < gkm.workspace_size_batch(16, [(100, 4, 1, 2)] * 3, 8)
