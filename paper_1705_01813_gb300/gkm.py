"""Python binding of libgkm (the C ABI in include/gkm.h).

Argument marshalling only: every step runs in the CUDA library.  PyTorch
supplies device memory (tensors, the workspace) and the current CUDA stream.
There is no CPU fallback: if ``libgkm.so`` is missing or fails to load, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build_native

_PKG = os.path.dirname(os.path.abspath(__file__))
_lib = None
_lock = threading.Lock()

GK_OK, GK_ERR_INVALID, GK_ERR_CUDA, GK_ERR_NOMEM, GK_ERR_TIMEOUT, GK_ERR_NUMERIC = range(6)
GK_OP_ASSIGN, GK_OP_UPDATE, GK_OP_REFINE, GK_OP_FIT, GK_OP_BUILD, GK_OP_RECALL, GK_OP_TREE, GK_OP_BOOST = range(8)

#: every entry point the header declares (checked by the tests)
EXPORTS = ["gk_version", "gk_last_error", "gk_workspace_size", "gk_workspace_size_build", "gk_init_labels",
           "gk_init_graph", "gk_assign_step", "gk_update_step", "gk_graph_refine", "gk_build_knn_graph",
           "gk_kmeans_fit", "gk_read_status", "gk_group_by_label", "gk_update_from_groups",
           "gk_graph_refine_groups", "gk_update_step_noalloc", "gk_graph_recall",
           "gk_set_replay", "gk_two_means_tree", "gk_workspace_size_batch", "gk_batch_fit", "gk_boost_init",
           "gk_boost_epoch"]
#: entry points that read the samples and have a BF16-sample twin named <name>_bf16
X_ENTRIES = ["gk_init_graph", "gk_assign_step", "gk_update_step", "gk_graph_refine", "gk_update_from_groups",
             "gk_graph_refine_groups", "gk_build_knn_graph", "gk_kmeans_fit", "gk_graph_recall",
             "gk_two_means_tree", "gk_batch_fit", "gk_boost_init", "gk_boost_epoch"]
EXPORTS += [name + "_bf16" for name in X_ENTRIES]


class GraphParams(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_int32), ("xi", ctypes.c_int32), ("tau", ctypes.c_int32),
                ("max_cluster", ctypes.c_int32), ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Job(ctypes.Structure):
    """One job of a batch (gk_job): n samples, k clusters, the seeds of its graph construction and its fit."""
    _fields_ = [("n", ctypes.c_int64), ("k", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("graph_seed", ctypes.c_uint64), ("fit_seed", ctypes.c_uint64)]


MAX_BATCH_JOBS = 64  # GK_MAX_BATCH_JOBS


class GkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libgkm error {code}: {msg}")
        self.code = code


def lib_path() -> str:
    return build_native.LIB


def load(build_if_missing: bool = True):
    """Load libgkm.so (compiling it first if it is missing and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(build_native.LIB):
                if not build_if_missing:
                    raise RuntimeError(f"libgkm.so not built ({build_native.LIB})")
                build_native.build()
            L = ctypes.CDLL(build_native.LIB)
            P, I64, I32, U64, SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
            L.gk_version.restype = ctypes.c_char_p
            L.gk_version.argtypes = []
            L.gk_last_error.restype = ctypes.c_char_p
            L.gk_last_error.argtypes = []
            L.gk_workspace_size.restype = SZ
            L.gk_workspace_size.argtypes = [I32, I64, I64, I32, I32]
            L.gk_workspace_size_build.restype = SZ
            L.gk_workspace_size_build.argtypes = [I64, I64, ctypes.POINTER(GraphParams)]
            L.gk_init_labels.argtypes = [I64, I32, U64, P, P]
            L.gk_init_graph.argtypes = [P, I64, I64, I64, I32, U64, P, P, P, SZ, P]
            L.gk_assign_step.argtypes = [P, I64, I64, I64, P, I32, P, I32, P, P, P, P, P, I32, P, P, SZ, P]
            L.gk_update_step.argtypes = [P, I64, I64, I64, P, I32, P, P, P, P, P, P, SZ, P]
            L.gk_graph_refine.argtypes = [P, I64, I64, I64, P, I32, I32, I32, I32, P, P, P, SZ, P]
            L.gk_build_knn_graph.argtypes = [P, I64, I64, I64, ctypes.POINTER(GraphParams), P, P, P, P, P, SZ, P]
            L.gk_kmeans_fit.argtypes = [P, I64, I64, I64, I32, P, I32, I32, P, U64, I32, P, P, P, P, P, SZ, P]
            L.gk_read_status.argtypes = [P, P]
            L.gk_group_by_label.argtypes = [P, I64, I32, P, P, P, P, SZ, P]
            L.gk_update_from_groups.argtypes = [P, I64, I64, I64, P, P, I32, P, P, P, P, SZ, P]
            L.gk_graph_refine_groups.argtypes = [P, I64, I64, I64, P, P, I32, I32, I32, I32, P, P, P, SZ, P]
            L.gk_update_step_noalloc.argtypes = [P, I64, I64, I64, P, I32, P, P, P, P]
            L.gk_graph_recall.argtypes = [P, I64, I64, I64, P, I32, P, I32, P, P, P, P, SZ, P]
            L.gk_set_replay.argtypes = [I32]
            L.gk_two_means_tree.argtypes = [P, I64, I64, I64, I32, I32, U64, P, P, SZ, P]
            L.gk_workspace_size_batch.restype = SZ
            L.gk_boost_init.argtypes = [P, I64, I64, I64, P, I32, P, P, P, P, SZ, P]
            L.gk_boost_epoch.argtypes = [P, I64, I64, I64, P, I32, P, I64, P, I32, P, P, P, P, P, SZ, P]
            L.gk_workspace_size_batch.argtypes = [I64, I32, P, ctypes.POINTER(GraphParams)]
            L.gk_batch_fit.argtypes = [P, I64, I64, I32, P, ctypes.POINTER(GraphParams), I32, P, P, P, P, P, P, SZ,
                                       P]
            for name in X_ENTRIES:
                getattr(L, name + "_bf16").argtypes = getattr(L, name).argtypes
            for name in EXPORTS:
                if name not in ("gk_version", "gk_last_error", "gk_workspace_size", "gk_workspace_size_build",
                                "gk_workspace_size_batch"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(rc: int):
    if rc != GK_OK:
        raise GkError(rc, load().gk_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _x(X: torch.Tensor):
    if (X.device.type != "cuda" or X.dtype not in (torch.float32, torch.bfloat16) or X.dim() != 2
            or X.stride(1) != 1):
        raise ValueError("X must be a CUDA float32 or bfloat16 matrix with unit column stride")
    return X.shape[0], X.shape[1], X.stride(0)


def _entry(name: str, X: torch.Tensor):
    """The library entry point for samples of X's type: BF16 samples go to the <name>_bf16 twin, which
    widens every element exactly to FP32 as it reads it."""
    return getattr(load(), name + "_bf16" if X.dtype == torch.bfloat16 else name)


def _dev(t: torch.Tensor, dtype, name: str):
    if t.device.type != "cuda" or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t


class Workspace:
    """Device scratch for the library, allocated by torch's caching allocator."""

    def __init__(self, nbytes: int, device=None):
        self.nbytes = max(256, int(nbytes))
        self.buf = torch.zeros(self.nbytes + 256, dtype=torch.uint8, device=device or "cuda")
        base = self.buf.data_ptr()
        self.off = (-base) % 256
        self.ptr = ctypes.c_void_p(base + self.off)

    @classmethod
    def from_buffer(cls, buf: torch.Tensor, stream=None) -> "Workspace":
        """A workspace over an existing uint8 device tensor (256-byte aligned start); its status word is
        cleared on `stream`."""
        if buf.dtype != torch.uint8 or not buf.is_cuda or buf.data_ptr() % 256 or buf.numel() < 256:
            raise ValueError("workspace buffer: uint8 device tensor, 256-byte aligned, at least 256 bytes")
        ws = cls.__new__(cls)
        ws.nbytes, ws.buf, ws.off = int(buf.numel()), buf, 0
        ws.ptr = ctypes.c_void_p(buf.data_ptr())
        with torch.cuda.stream(stream or torch.cuda.current_stream()):
            buf[:256].zero_()
        return ws

    def status(self, stream=None) -> int:
        return load().gk_read_status(self.ptr, _stream(stream))


_ws_cache: dict = {}


def workspace(nbytes: int, device=None) -> Workspace:
    dev = torch.device(device) if device is not None else torch.device("cuda")
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    key = (str(dev), threading.get_ident())
    ws = _ws_cache.get(key)
    if ws is None or ws.nbytes < nbytes:
        ws = Workspace(max(nbytes, int(ws.nbytes * 1.25) if ws else nbytes), dev)
        _ws_cache[key] = ws
    return ws


def workspace_size(op: int, n: int, d: int, k: int, kappa: int = 0) -> int:
    return int(load().gk_workspace_size(op, n, d, k, kappa))


def workspace_size_build(n: int, d: int, kappa: int, xi: int = 50, tau: int = 10, max_cluster: int = 128,
                         seed: int = 0) -> int:
    p = GraphParams(kappa, xi, tau, max_cluster, seed, 0, 0)
    return int(load().gk_workspace_size_build(n, d, ctypes.byref(p)))


def version() -> str:
    return load().gk_version().decode()


def init_labels(n: int, k: int, seed: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    out = torch.empty(n, dtype=torch.int32, device="cuda") if out is None else _dev(out, torch.int32, "out")
    _check(load().gk_init_labels(n, k, seed, _ptr(out), _stream(stream)))
    return out


def init_graph(X: torch.Tensor, kappa: int, seed: int, g_idx=None, g_dist=None, ws: Workspace | None = None,
               stream=None):
    n, d, ld = _x(X)
    gi = torch.empty((n, kappa), dtype=torch.int32, device=X.device) if g_idx is None else g_idx
    gd = torch.empty((n, kappa), dtype=torch.float32, device=X.device) if g_dist is None else g_dist
    ws = ws or workspace(256, X.device)
    _check(_entry("gk_init_graph", X)(_ptr(X), n, d, ld, kappa, seed, _ptr(gi), _ptr(gd), ws.ptr, ws.nbytes,
                                _stream(stream)))
    return gi, gd


ALLOC = "alloc"


def assign_step(X, g_idx, C, labels_in, labels_out=None, best_d2=ALLOC, sum_d2=ALLOC, n_changed=ALLOC,
                precision: int = 0, members=None, ws: Workspace | None = None, stream=None):
    """Graph-guided assignment; returns (labels_out, best_d2, sum_d2, n_changed).

    The optional outputs are allocated by default; pass a tensor to reuse it or
    None to have the library skip that output."""
    n, d, ld = _x(X)
    _dev(g_idx, torch.int32, "g_idx")
    _dev(C, torch.float32, "C")
    _dev(labels_in, torch.int32, "labels_in")
    k, kappa = C.shape[0], g_idx.shape[1]
    dev = X.device
    labels_out = torch.empty(n, dtype=torch.int32, device=dev) if labels_out is None else labels_out
    best_d2 = torch.empty(n, dtype=torch.float32, device=dev) if best_d2 is ALLOC else best_d2
    sum_d2 = torch.empty(1, dtype=torch.float64, device=dev) if sum_d2 is ALLOC else sum_d2
    n_changed = torch.empty(1, dtype=torch.int64, device=dev) if n_changed is ALLOC else n_changed
    ws = ws or workspace(workspace_size(GK_OP_ASSIGN, n, d, k, kappa), dev)
    _check(_entry("gk_assign_step", X)(_ptr(X), n, d, ld, _ptr(g_idx), kappa, _ptr(C), k, _ptr(labels_in),
                                 _ptr(labels_out), _ptr(best_d2), _ptr(sum_d2), _ptr(n_changed), precision,
                                 _ptr(members), ws.ptr, ws.nbytes, _stream(stream)))
    return labels_out, best_d2, sum_d2, n_changed


def update_step(X, labels, k: int, C, counts=None, sum_d2=None, offsets=None, members=None,
                ws: Workspace | None = None, stream=None):
    """Centroid update in place on C; returns (C, counts, sum_d2, offsets, members)."""
    n, d, ld = _x(X)
    _dev(labels, torch.int32, "labels")
    _dev(C, torch.float32, "C")
    dev = X.device
    counts = torch.empty(k, dtype=torch.int32, device=dev) if counts is None else counts
    sum_d2 = torch.empty(1, dtype=torch.float64, device=dev) if sum_d2 is None else sum_d2
    offsets = torch.empty(k + 1, dtype=torch.int32, device=dev) if offsets is None else offsets
    members = torch.empty(n, dtype=torch.int32, device=dev) if members is None else members
    ws = ws or workspace(workspace_size(GK_OP_UPDATE, n, d, k), dev)
    _check(_entry("gk_update_step", X)(_ptr(X), n, d, ld, _ptr(labels), k, _ptr(C), _ptr(counts), _ptr(sum_d2),
                                 _ptr(offsets), _ptr(members), ws.ptr, ws.nbytes, _stream(stream)))
    return C, counts, sum_d2, offsets, members


def graph_refine(X, labels, k: int, g_idx, g_dist, max_cluster: int = 128, precision: int = 0,
                 ws: Workspace | None = None, stream=None):
    """One refinement of the graph in place (pairs inside each cluster)."""
    n, d, ld = _x(X)
    _dev(labels, torch.int32, "labels")
    _dev(g_idx, torch.int32, "g_idx")
    _dev(g_dist, torch.float32, "g_dist")
    kappa = g_idx.shape[1]
    ws = ws or workspace(workspace_size(GK_OP_REFINE, n, d, k, kappa), X.device)
    _check(_entry("gk_graph_refine", X)(_ptr(X), n, d, ld, _ptr(labels), k, kappa, max_cluster, precision, _ptr(g_idx),
                                  _ptr(g_dist), ws.ptr, ws.nbytes, _stream(stream)))
    return g_idx, g_dist


def build_knn_graph(X, kappa: int, xi: int = 50, tau: int = 10, max_cluster: int = 128, seed: int = 0,
                    labels_out=None, g_idx=None, g_dist=None, want_log: bool = True, precision: int = 0,
                    ws: Workspace | None = None, stream=None):
    """Alg. 3; returns (g_idx, g_dist, labels at k0, distortion log or None)."""
    n, d, ld = _x(X)
    dev = X.device
    p = GraphParams(kappa, xi, tau, max_cluster, seed, precision, 0)
    g_idx = torch.empty((n, kappa), dtype=torch.int32, device=dev) if g_idx is None else g_idx
    g_dist = torch.empty((n, kappa), dtype=torch.float32, device=dev) if g_dist is None else g_dist
    labels_out = torch.empty(n, dtype=torch.int32, device=dev) if labels_out is None else labels_out
    log = (ctypes.c_double * (2 * tau + 1))() if want_log else None
    ws = ws or workspace(int(load().gk_workspace_size_build(n, d, ctypes.byref(p))), dev)
    _check(_entry("gk_build_knn_graph", X)(_ptr(X), n, d, ld, ctypes.byref(p), _ptr(g_idx), _ptr(g_dist),
                                     _ptr(labels_out), log, ws.ptr, ws.nbytes, _stream(stream)))
    return g_idx, g_dist, labels_out, (list(log) if want_log else None)


def kmeans_fit(X, k: int, g_idx, iters: int, init_labels=None, seed: int = 0, labels_out=None, C_out=None,
               counts_out=None, want_log: bool = True, precision: int = 0, ws: Workspace | None = None,
               stream=None):
    """Graph-guided k-means; returns (labels, centroids, counts, distortion log or None)."""
    n, d, ld = _x(X)
    dev = X.device
    _dev(g_idx, torch.int32, "g_idx")
    kappa = g_idx.shape[1]
    labels_out = torch.empty(n, dtype=torch.int32, device=dev) if labels_out is None else labels_out
    C_out = torch.empty((k, d), dtype=torch.float32, device=dev) if C_out is None else C_out
    counts_out = torch.empty(k, dtype=torch.int32, device=dev) if counts_out is None else counts_out
    log = (ctypes.c_double * (2 * iters + 1))() if want_log else None
    ws = ws or workspace(workspace_size(GK_OP_FIT, n, d, k, kappa), dev)
    _check(_entry("gk_kmeans_fit", X)(_ptr(X), n, d, ld, k, _ptr(g_idx), kappa, iters, _ptr(init_labels), seed,
                                precision, _ptr(labels_out), _ptr(C_out), _ptr(counts_out), log, ws.ptr, ws.nbytes,
                                _stream(stream)))
    return labels_out, C_out, counts_out, (list(log) if want_log else None)


def _jobs(jobs) -> "ctypes.Array":
    """A gk_job array from (n, k, graph_seed, fit_seed) tuples."""
    arr = (Job * len(jobs))()
    for a, (n, k, gs, fs) in zip(arr, jobs):
        a.n, a.k, a.reserved, a.graph_seed, a.fit_seed = int(n), int(k), 0, int(gs), int(fs)
    return arr


def workspace_size_batch(d: int, jobs, kappa: int, xi: int = 50, tau: int = 10, max_cluster: int = 128,
                         precision: int = 0) -> int:
    p = GraphParams(kappa, xi, tau, max_cluster, 0, precision, 0)
    return int(load().gk_workspace_size_batch(d, len(jobs), ctypes.cast(_jobs(jobs), ctypes.c_void_p),
                                              ctypes.byref(p)))


def batch_fit(X, jobs, kappa: int, xi: int = 50, tau: int = 10, max_cluster: int = 128, iters: int = 10,
              precision: int = 0, g_idx=None, g_dist=None, labels_out=None, C_out=None, distortion=None,
              ws: Workspace | None = None, stream=None):
    """Independent jobs as one batch (gk_batch_fit): X holds the jobs' samples concatenated, jobs is a list of
    (n, k, graph_seed, fit_seed).  Returns (g_idx, g_dist, labels (each job's own numbering), centroids (jobs'
    rows stacked), distortion [njobs] FP64 on the device)."""
    N, d, ld = _x(X)
    if sum(int(j[0]) for j in jobs) != N:
        raise ValueError("the jobs' sample counts must add up to X's rows")
    dev = X.device
    K = sum(int(j[1]) for j in jobs)
    p = GraphParams(kappa, xi, tau, max_cluster, 0, precision, 0)
    arr = _jobs(jobs)
    g_idx = torch.empty((N, kappa), dtype=torch.int32, device=dev) if g_idx is None else g_idx
    g_dist = torch.empty((N, kappa), dtype=torch.float32, device=dev) if g_dist is None else g_dist
    labels_out = torch.empty(N, dtype=torch.int32, device=dev) if labels_out is None else labels_out
    C_out = torch.empty((K, d), dtype=torch.float32, device=dev) if C_out is None else C_out
    distortion = torch.empty(len(jobs), dtype=torch.float64, device=dev) if distortion is None else distortion
    ws = ws or workspace(workspace_size_batch(d, jobs, kappa, xi, tau, max_cluster, precision), dev)
    _check(_entry("gk_batch_fit", X)(_ptr(X), d, ld, len(jobs), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(p),
                                     iters, _ptr(g_idx), _ptr(g_dist), _ptr(labels_out), _ptr(C_out),
                                     _ptr(distortion), ws.ptr, ws.nbytes, _stream(stream)))
    return g_idx, g_dist, labels_out, C_out, distortion


def group_by_label(labels, k: int, offsets=None, members=None, counts=None, ws: Workspace | None = None,
                   stream=None):
    """CSR of the clusters: (offsets [k+1], members [n], counts [k])."""
    _dev(labels, torch.int32, "labels")
    n = labels.shape[0]
    dev = labels.device
    offsets = torch.empty(k + 1, dtype=torch.int32, device=dev) if offsets is None else offsets
    members = torch.empty(n, dtype=torch.int32, device=dev) if members is None else members
    counts = torch.empty(k, dtype=torch.int32, device=dev) if counts is None else counts
    ws = ws or workspace(workspace_size(GK_OP_UPDATE, n, 1, k), dev)
    _check(load().gk_group_by_label(_ptr(labels), n, k, _ptr(offsets), _ptr(members), _ptr(counts), ws.ptr,
                                    ws.nbytes, _stream(stream)))
    return offsets, members, counts


def update_from_groups(X, offsets, members, k: int, C, counts=None, sum_d2=None, ws: Workspace | None = None,
                       stream=None):
    """Segmented mean over a CSR grouping, in place on C."""
    n, d, ld = _x(X)
    ws = ws or workspace(workspace_size(GK_OP_UPDATE, n, d, k), X.device)
    _check(_entry("gk_update_from_groups", X)(_ptr(X), n, d, ld, _ptr(offsets), _ptr(members), k, _ptr(C),
                                        _ptr(counts), _ptr(sum_d2), ws.ptr, ws.nbytes, _stream(stream)))
    return C


def graph_refine_groups(X, offsets, members, k: int, g_idx, g_dist, max_cluster: int = 128, precision: int = 0,
                        ws: Workspace | None = None, stream=None):
    """Graph refinement over a CSR grouping, in place on (g_idx, g_dist)."""
    n, d, ld = _x(X)
    ws = ws or workspace(workspace_size(GK_OP_REFINE, n, d, k, g_idx.shape[1]), X.device)
    _check(_entry("gk_graph_refine_groups", X)(_ptr(X), n, d, ld, _ptr(offsets), _ptr(members), k, g_idx.shape[1],
                                         max_cluster, precision, _ptr(g_idx), _ptr(g_dist), ws.ptr, ws.nbytes,
                                         _stream(stream)))
    return g_idx, g_dist


def graph_recall(X, g_idx, queries, nn_idx=None, nn_dist=None, ws: Workspace | None = None, stream=None):
    """Top-1 recall of the graph on the sampled queries (Sec. 5); returns (hits tensor [1] int64, nn_idx,
    nn_dist): each query's exact nearest neighbour and its distance."""
    n, d, ld = _x(X)
    _dev(g_idx, torch.int32, "g_idx")
    _dev(queries, torch.int32, "queries")
    m, dev = queries.numel(), X.device
    nn_idx = torch.empty(m, dtype=torch.int32, device=dev) if nn_idx is None else nn_idx
    nn_dist = torch.empty(m, dtype=torch.float32, device=dev) if nn_dist is None else nn_dist
    hits = torch.empty(1, dtype=torch.int64, device=dev)
    ws = ws or workspace(workspace_size(GK_OP_RECALL, n, d, m, g_idx.shape[1]), dev)
    _check(_entry("gk_graph_recall", X)(_ptr(X), n, d, ld, _ptr(g_idx), g_idx.shape[1], _ptr(queries), m,
                                        _ptr(nn_idx), _ptr(nn_dist), _ptr(hits), ws.ptr, ws.nbytes,
                                        _stream(stream)))
    return hits, nn_idx, nn_dist


def two_means_tree(X, k: int, iters: int = 2, seed: int = 0, out: torch.Tensor | None = None,
                   ws: Workspace | None = None, stream=None) -> torch.Tensor:
    """Alg. 1: labels int32[n] of k clusters made by bisecting the largest cluster into equal halves (see
    gk_two_means_tree); clusters are numbered left to right in the tree."""
    n, d, ld = _x(X)
    out = torch.empty(n, dtype=torch.int32, device=X.device) if out is None else out
    _dev(out, torch.int32, "out")
    ws = ws or workspace(workspace_size(GK_OP_TREE, n, d, k), X.device)
    _check(_entry("gk_two_means_tree", X)(_ptr(X), n, d, ld, k, iters, seed, _ptr(out), ws.ptr, ws.nbytes,
                                          _stream(stream)))
    return out


def boost_init(X, labels, k: int, D=None, counts=None, S=None, ws: Workspace | None = None, stream=None):
    """Eq. 2 state of the partition `labels` (see gk_boost_init): D (k x d FP64 composite vectors), counts
    (int32[k]) and S (FP64[k], D_r'D_r)."""
    n, d, ld = _x(X)
    dev = X.device
    D = torch.empty((k, d), dtype=torch.float64, device=dev) if D is None else D
    counts = torch.empty(k, dtype=torch.int32, device=dev) if counts is None else counts
    S = torch.empty(k, dtype=torch.float64, device=dev) if S is None else S
    _dev(labels, torch.int32, "labels")
    _dev(D, torch.float64, "D")
    _dev(counts, torch.int32, "counts")
    _dev(S, torch.float64, "S")
    if tuple(D.shape) != (k, d):
        raise ValueError("D must be k x d")
    ws = ws or workspace(workspace_size(GK_OP_BOOST, n, d, k), dev)
    _check(_entry("gk_boost_init", X)(_ptr(X), n, d, ld, _ptr(labels), k, _ptr(D), _ptr(counts), _ptr(S), ws.ptr,
                                      ws.nbytes, _stream(stream)))
    return D, counts, S


def boost_epoch(X, g_idx, order, labels, k: int, D, counts, S, n_moved=None, ws: Workspace | None = None,
                stream=None) -> torch.Tensor:
    """One epoch of the boost form's move step (Eq. 3 gains, Alg. 2) over the visits `order` (int32 sample ids);
    labels, D, counts and S are updated in place.  Returns n_moved (device int64[1])."""
    n, d, ld = _x(X)
    dev = X.device
    for t, dt, name in ((g_idx, torch.int32, "g_idx"), (order, torch.int32, "order"), (labels, torch.int32, "labels"),
                        (D, torch.float64, "D"), (counts, torch.int32, "counts"), (S, torch.float64, "S")):
        _dev(t, dt, name)
    if tuple(D.shape) != (k, d):
        raise ValueError("D must be k x d")
    n_moved = torch.empty(1, dtype=torch.int64, device=dev) if n_moved is None else n_moved
    _dev(n_moved, torch.int64, "n_moved")
    kappa = g_idx.shape[1]
    ws = ws or workspace(workspace_size(GK_OP_BOOST, n, d, k, kappa), dev)
    _check(_entry("gk_boost_epoch", X)(_ptr(X), n, d, ld, _ptr(g_idx), kappa, _ptr(order), order.numel(),
                                       _ptr(labels), k, _ptr(D), _ptr(counts), _ptr(S), _ptr(n_moved), ws.ptr,
                                       ws.nbytes, _stream(stream)))
    return n_moved


def set_replay(enable: bool):
    """Replay repeated build_knn_graph / kmeans_fit calls with equal arguments as one captured CUDA graph (see
    gk_set_replay); off by default."""
    _check(load().gk_set_replay(1 if enable else 0))


def read_status(ws: Workspace, stream=None) -> int:
    """Synchronise and return (and clear) the device status word of a workspace."""
    return int(load().gk_read_status(ws.ptr, _stream(stream)))
