"""Python face of the GK-means FP64 oracle (``gkm_oracle.c``).

TEST INFRASTRUCTURE ONLY: this module and the C file it compiles are the
independent checker of the CUDA library.  Only the test suite, the smoke check
and the benchmark's CPU-baseline / reference leg may import it; the library's
own code path never does.  It shares no code with the CUDA side: it compiles
its own C file with gcc and marshals numpy arrays through ctypes.

Every function restates the paper (Deng & Zhao, arXiv 1705.01813):
  init_labels / init_graph   seeded start (Alg. 3 starts from random neighbour lists; SplitMix64 by its published definition)
  assign                     Alg. 2 with the closest-centroid rule of Sec. 4.2 (GK-means^-)
  assign_exhaustive          Lloyd's assignment after Eq. 1 (every centroid a candidate)
  assign_margin              near-tie report: relative gap of each sample's two best candidate clusters
  update                     centroid = mean (Sec. 1), Eq. 2 objective I, Eq. 4 distortion
  fit                        C0 = update(L0), then T x {assign, update}
  graph_refine(_rows)        Alg. 3 exhaustive pairs inside each cluster
  build_graph                Alg. 3 with one GK-means iteration per round (Sec. 4.5)
  brute_knn                  exact KNN graph by all pairs
  two_means_tree             Alg. 1: k clusters by bisecting the largest cluster into equal halves
  boost_init / boost_epoch   the boost form: Eq. 2 state (D_r, n_r, S_r) and Alg. 2's move step by Eq. 3 gains
  fold_sq                    the fixed-order FP64 squared norm the boost form uses

Parity status: every function above is pinned by tests/test_oracle_pins.py
(brute force, closed forms, invariants, published SplitMix64 outputs); the
paper prints no worked example, so no function is pinned to a printed value.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gkm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgkm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no vector intrinsics, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


def _bind(lib):
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I32 = ctypes.c_int32
    U64 = ctypes.c_uint64
    lib.or_set_threads.argtypes = [ctypes.c_int]
    lib.or_set_threads.restype = ctypes.c_int
    lib.or_splitmix64_next.argtypes = [P]
    lib.or_splitmix64_next.restype = U64
    lib.or_draw.argtypes = [U64, U64]
    lib.or_draw.restype = U64
    lib.or_init_labels.argtypes = [I64, I32, U64, P]
    lib.or_init_graph.argtypes = [P, I64, I64, I64, I32, U64, P, P]
    lib.or_init_graph_rows.argtypes = [P, I64, I64, I64, I32, U64, P, I64, P, P]
    lib.or_assign.argtypes = [P, I64, I64, I64, P, I32, P, I32, P, P, P, P, P, I64]
    lib.or_assign_exhaustive.argtypes = [P, I64, I64, I64, P, I32, P, P]
    lib.or_assign_margin.argtypes = [P, I64, I64, I64, P, I32, P, P, P]
    lib.or_update.argtypes = [P, I64, I64, I64, P, I32, P, P, P, P]
    lib.or_fit.argtypes = [P, I64, I64, I64, I32, P, I32, I32, P, P, P, P, P]
    lib.or_graph_refine.argtypes = [P, I64, I64, I64, P, I32, I32, I32, P, P]
    lib.or_graph_refine_rows.argtypes = [P, I64, I64, I64, P, I32, I32, I32, P, I64, P, P]
    lib.or_group_csr.argtypes = [P, I64, I32, P, P]
    lib.or_build_graph.argtypes = [P, I64, I64, I64, I32, I32, I32, I32, U64, ctypes.c_int, P, P, P, P]
    lib.or_build_graph.restype = ctypes.c_int
    lib.or_brute_knn.argtypes = [P, I64, I64, I64, I32, P, P]
    lib.or_two_means_tree.argtypes = [P, I64, I64, I64, I32, I32, U64, P]
    lib.or_two_means_tree.restype = ctypes.c_int
    lib.or_fold_sq.argtypes = [P, I64]
    lib.or_fold_sq.restype = ctypes.c_double
    lib.or_boost_init.argtypes = [P, I64, I64, I64, P, I32, P, P, P]
    lib.or_boost_init.restype = ctypes.c_int
    lib.or_boost_epoch.argtypes = [P, I64, I64, I64, P, I32, P, I64, P, I32, P, P, P, P]
    lib.or_boost_epoch.restype = I64
    return lib


def compile_source(src: str, lib_path: str) -> str:
    """Compile an oracle source file to a shared library (used by build() and by
    the tests that plant a mistake in a copy of the oracle)."""
    os.makedirs(os.path.dirname(lib_path), exist_ok=True)
    tmp = lib_path + f".{os.getpid()}.tmp"
    subprocess.check_call(
        ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-std=c11",
         "-o", tmp, src, "-lm"])
    os.replace(tmp, lib_path)
    return lib_path


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _x(X):
    X = np.asarray(X)
    if X.dtype != np.float32:
        raise TypeError("oracle reads X as stored FP32")
    X = np.ascontiguousarray(X)
    return X, X.shape[0], X.shape[1]


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Oracle:
    """The oracle's functions bound to one compiled copy of gkm_oracle.c."""

    def __init__(self, lib_path: str | None = None):
        self._lib = _load() if lib_path is None else _bind(ctypes.CDLL(lib_path))

    def set_threads(self, threads: int) -> int:
        """Host threads of the oracle's parallel loops (1: single-threaded; 0: leave as is); returns the count in
        effect.  Results do not depend on it."""
        return int(self._lib.or_set_threads(int(threads)))

    def splitmix64_stream(self, seed: int, count: int) -> list[int]:
        """The published SplitMix64 sequence: ``count`` outputs from state ``seed``."""
        lib = self._lib
        st = ctypes.c_uint64(seed)
        return [int(lib.or_splitmix64_next(ctypes.byref(st))) for _ in range(count)]

    def draw(self, key: int, counter: int) -> int:
        return int(self._lib.or_draw(key, counter))

    def init_labels(self, n: int, k: int, seed: int) -> np.ndarray:
        out = np.empty(n, np.int32)
        self._lib.or_init_labels(n, k, seed, _p(out))
        return out

    def init_graph(self, X, kappa: int, seed: int):
        X, n, d = _x(X)
        idx = np.empty((n, kappa), np.int32)
        dist = np.empty((n, kappa), np.float64)
        self._lib.or_init_graph(_p(X), n, d, d, kappa, seed, _p(idx), _p(dist))
        return idx, dist

    def init_graph_rows(self, X, kappa: int, seed: int, rows):
        """The initial graph's rows for the listed samples only (the same draws and distances)."""
        X, n, d = _x(X)
        r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        idx = np.empty((r.shape[0], kappa), np.int32)
        dist = np.empty((r.shape[0], kappa), np.float64)
        self._lib.or_init_graph_rows(_p(X), n, d, d, kappa, seed, _p(r), r.shape[0], _p(idx), _p(dist))
        return idx, dist

    def assign(self, X, G, C, labels, rows=None):
        """Graph-guided assignment; returns (labels', best d2, |Q|) for all rows or the listed rows."""
        X, n, d = _x(X)
        G = _i32(G)
        kappa = G.shape[1]
        C = _f64(C)
        k = C.shape[0]
        L = _i32(labels)
        if rows is None:
            m, r = n, None
        else:
            r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
            m = r.shape[0]
        Lo = np.empty(m, np.int32)
        best = np.empty(m, np.float64)
        uniq = np.empty(m, np.int32)
        self._lib.or_assign(_p(X), n, d, d, _p(G), kappa, _p(C), k, _p(L), _p(Lo), _p(best), _p(uniq),
                          _p(r), 0 if r is None else m)
        return Lo, best, uniq

    def assign_margin(self, X, G, C, labels):
        """Near-tie report of the assignment: per sample (d2 - d1) / d1 over its two best distinct candidate
        clusters (0: exact tie, inf: one candidate cluster or d1 = 0 < d2)."""
        X, n, d = _x(X)
        G = _i32(G)
        C = _f64(C)
        L = _i32(labels)
        out = np.empty(n, np.float64)
        self._lib.or_assign_margin(_p(X), n, d, d, _p(G), G.shape[1], _p(C), _p(L), _p(out))
        return out

    def assign_exhaustive(self, X, C):
        X, n, d = _x(X)
        C = _f64(C)
        Lo = np.empty(n, np.int32)
        best = np.empty(n, np.float64)
        self._lib.or_assign_exhaustive(_p(X), n, d, d, _p(C), C.shape[0], _p(Lo), _p(best))
        return Lo, best

    def update(self, X, labels, k: int, C_old=None):
        """Returns (C [k x d] FP64, counts [k], E after the update, I of Eq. 2)."""
        X, n, d = _x(X)
        L = _i32(labels)
        C = np.zeros((k, d), np.float64) if C_old is None else _f64(C_old).copy()
        counts = np.empty(k, np.int64)
        E = ctypes.c_double()
        I = ctypes.c_double()
        self._lib.or_update(_p(X), n, d, d, _p(L), k, _p(C), _p(counts), ctypes.byref(E), ctypes.byref(I))
        return C, counts, E.value, I.value

    def fit(self, X, k: int, G, iters: int, L0):
        X, n, d = _x(X)
        G = _i32(G)
        L0 = _i32(L0)
        L = np.empty(n, np.int32)
        C = np.empty((k, d), np.float64)
        counts = np.empty(k, np.int64)
        E = np.empty(2 * iters + 1, np.float64)
        self._lib.or_fit(_p(X), n, d, d, k, _p(G), G.shape[1], iters, _p(L0), _p(L), _p(C), _p(counts), _p(E))
        return L, C, counts, E

    def graph_refine(self, X, labels, k: int, g_idx, g_dist, max_cluster: int):
        X, n, d = _x(X)
        L = _i32(labels)
        gi = _i32(g_idx).copy()
        gd = _f64(g_dist).copy()
        self._lib.or_graph_refine(_p(X), n, d, d, _p(L), k, gi.shape[1], max_cluster, _p(gi), _p(gd))
        return gi, gd

    def graph_refine_rows(self, X, labels, k: int, rows, rows_idx, rows_dist, max_cluster: int):
        X, n, d = _x(X)
        L = _i32(labels)
        r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        gi = _i32(rows_idx).copy()
        gd = _f64(rows_dist).copy()
        self._lib.or_graph_refine_rows(_p(X), n, d, d, _p(L), k, gi.shape[1], max_cluster, _p(r), r.shape[0],
                                     _p(gi), _p(gd))
        return gi, gd

    def group_csr(self, labels, k: int):
        L = _i32(labels)
        off = np.empty(k + 1, np.int64)
        mem = np.empty(L.shape[0], np.int32)
        self._lib.or_group_csr(_p(L), L.shape[0], k, _p(off), _p(mem))
        return off, mem

    def build_graph(self, X, kappa: int, xi: int = 50, tau: int = 10, max_cluster: int = 128, seed: int = 0,
                    use_visited: bool = False):
        """Alg. 3; returns (g_idx, g_dist, final labels at k0, E log of 2*tau+1 entries)."""
        X, n, d = _x(X)
        gi = np.empty((n, kappa), np.int32)
        gd = np.empty((n, kappa), np.float64)
        L = np.empty(n, np.int32)
        E = np.empty(2 * tau + 1, np.float64)
        rc = self._lib.or_build_graph(_p(X), n, d, d, kappa, xi, tau, max_cluster, seed, int(use_visited),
                                    _p(gi), _p(gd), _p(L), _p(E))
        if rc:
            raise MemoryError("visited-pair set does not fit")
        return gi, gd, L, E

    def brute_knn(self, X, kappa: int):
        X, n, d = _x(X)
        gi = np.empty((n, kappa), np.int32)
        gd = np.empty((n, kappa), np.float64)
        self._lib.or_brute_knn(_p(X), n, d, d, kappa, _p(gi), _p(gd))
        return gi, gd

    def two_means_tree(self, X, k: int, iters: int = 2, seed: int = 0) -> np.ndarray:
        """Alg. 1 (readings T1-T6 in gkm_oracle.c); labels in [0, k), numbered left to right in the tree."""
        X, n, d = _x(X)
        out = np.empty(n, np.int32)
        if self._lib.or_two_means_tree(_p(X), n, d, d, k, iters, seed, _p(out)):
            raise ValueError("two_means_tree: need 1 <= k <= n and iters >= 0")
        return out

    def fold_sq(self, v) -> float:
        """Squared norm of v in FP64 by halving folds over v zero-padded to a power of two (the boost form's
        order of summation, reading B4 in gkm_oracle.c)."""
        v = _f64(v).ravel()
        return float(self._lib.or_fold_sq(_p(v), v.shape[0]))

    def boost_init(self, X, labels, k: int):
        """Eq. 2 state of a partition: (D k x d FP64 composite vectors, counts int32[k], S FP64[k] = D_r'D_r)."""
        X, n, d = _x(X)
        L = _i32(labels)
        D = np.empty((k, d), np.float64)
        cnt = np.empty(k, np.int32)
        S = np.empty(k, np.float64)
        if self._lib.or_boost_init(_p(X), n, d, d, _p(L), k, _p(D), _p(cnt), _p(S)):
            raise MemoryError("boost_init")
        return D, cnt, S

    def boost_epoch(self, X, g_idx, order, labels, k: int, D, counts, S):
        """Alg. 2's move step (Eq. 3 gains) over the visits `order`; returns new (labels, D, counts, S, moves,
        gains) where gains[s] is the gain of the move made at visit s (0 if the sample stayed)."""
        X, n, d = _x(X)
        G = _i32(g_idx)
        kappa = G.shape[1]
        od = _i32(order)
        L = _i32(labels).copy()
        D = _f64(D).copy()
        cnt = _i32(counts).copy()
        S = _f64(S).copy()
        gains = np.empty(od.shape[0], np.float64)
        moves = self._lib.or_boost_epoch(_p(X), n, d, d, _p(G), kappa, _p(od), od.shape[0], _p(L), k, _p(D),
                                         _p(cnt), _p(S), _p(gains))
        if moves < 0:
            raise MemoryError("boost_epoch")
        return L, D, cnt, S, int(moves), gains


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def __getattr__(name):
    # module-level access to the default oracle's functions: oracle.assign(...)
    if name.startswith("_"):
        raise AttributeError(name)
    return getattr(default(), name)
