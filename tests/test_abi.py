"""The C ABI without a GPU: the library loads, exports every entry point the
header declares, sizes workspaces, and rejects bad arguments before it
enqueues anything (these calls never reach a CUDA call)."""
import ctypes
import os
import re

import pytest

from paper_1705_01813_gb300 import build_native, gkm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gkm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gk_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build_native.build()
    return gkm.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert names == sorted(gkm.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name
    assert "sm_103a" in gkm.version()


def test_workspace_sizes(lib):
    for op in (gkm.GK_OP_ASSIGN, gkm.GK_OP_UPDATE, gkm.GK_OP_REFINE, gkm.GK_OP_FIT):
        a = gkm.workspace_size(op, 20000, 32, 200, 20)
        b = gkm.workspace_size(op, 1_000_000, 128, 10000, 50)
        assert 256 <= a <= b
    assert gkm.workspace_size(99, 10, 2, 2) == 0
    assert gkm.workspace_size_build(20000, 32, 20) > gkm.workspace_size(gkm.GK_OP_FIT, 20000, 32, 400)


def _fake(addr=0x10000000):
    return ctypes.c_void_p(addr)


def test_argument_errors(lib):
    # fake pointers: every call below must be refused by the host-side checks before any CUDA
    # call; run only where no GPU is visible so that a missed check can never reach a device
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("argument checks with fake pointers run on CPU-only hosts")
    P = _fake()
    ws = _fake(0x20000000)
    # n too small, kappa >= n, kappa > 128, ld < d, misaligned workspace, NULL arrays
    assert lib.gk_assign_step(P, 1, 4, 4, P, 1, P, 2, P, _fake(0x30000000), None, None, None, 0, None, ws, 1 << 20,
                              None) == gkm.GK_ERR_INVALID
    assert lib.gk_assign_step(P, 10, 4, 4, P, 10, P, 2, P, _fake(0x30000000), None, None, None, 0, None, ws, 1 << 20,
                              None) == gkm.GK_ERR_INVALID
    assert b"kappa" in lib.gk_last_error()
    assert lib.gk_assign_step(P, 1000, 4, 4, P, 129, P, 2, P, _fake(0x30000000), None, None, None, 0, None, ws, 1 << 20,
                              None) == gkm.GK_ERR_INVALID
    assert lib.gk_assign_step(P, 10, 4, 3, P, 2, P, 2, P, _fake(0x30000000), None, None, None, 0, None, ws, 1 << 20,
                              None) == gkm.GK_ERR_INVALID
    assert b"ld" in lib.gk_last_error()
    assert lib.gk_assign_step(P, 10, 4, 4, P, 2, P, 2, P, P, None, None, None, 0, None, ws, 1 << 20,
                              None) == gkm.GK_ERR_INVALID
    assert b"alias" in lib.gk_last_error()
    assert lib.gk_assign_step(P, 10, 4, 4, P, 2, P, 2, P, _fake(0x30000000), None, None, None, 0, None, _fake(0x20000010),
                              1 << 20, None) == gkm.GK_ERR_INVALID
    assert b"aligned" in lib.gk_last_error()
    assert lib.gk_assign_step(P, 10, 4, 4, P, 2, P, 2, P, _fake(0x30000000), None, None, None, 0, None, ws, 16,
                              None) == gkm.GK_ERR_INVALID
    assert b"too small" in lib.gk_last_error()
    assert lib.gk_assign_step(P, 10, 4, 4, P, 2, P, 2, P, _fake(0x30000000), None, None, None, 5, None, ws, 1 << 20,
                              None) == gkm.GK_ERR_INVALID
    assert b"precision" in lib.gk_last_error()
    for bad in (2 | (3 << 8), 1 | (16 << 8), 1 << 16, -1):  # group width not 0, 4 or 8; bits above 15; negative
        assert lib.gk_assign_step(P, 10, 4, 4, P, 2, P, 2, P, _fake(0x30000000), None, None, None, bad, None, ws,
                                  1 << 20, None) == gkm.GK_ERR_INVALID
    assert lib.gk_update_step(None, 10, 4, 4, P, 2, P, None, None, None, None, ws, 1 << 20,
                              None) == gkm.GK_ERR_INVALID
    assert lib.gk_update_step(P, 10, 4, 4, P, 0, P, None, None, None, None, ws, 1 << 20,
                              None) == gkm.GK_ERR_INVALID
    assert lib.gk_graph_refine(P, 10, 4, 4, P, 2, 3, 1, 0, P, P, ws, 1 << 20, None) == gkm.GK_ERR_INVALID
    assert b"max_cluster" in lib.gk_last_error()
    assert lib.gk_graph_refine(P, 10, 4, 4, P, 2, 3, 8, 5, P, P, ws, 1 << 20, None) == gkm.GK_ERR_INVALID
    assert b"precision" in lib.gk_last_error()
    assert lib.gk_kmeans_fit(P, 10, 4, 4, 2, P, 3, 5000, None, 0, 0, P, P, None, None, ws, 1 << 20,
                             None) == gkm.GK_ERR_INVALID
    assert lib.gk_init_labels(0, 3, 0, P, None) == gkm.GK_ERR_INVALID
    assert lib.gk_init_labels(10, 0, 0, P, None) == gkm.GK_ERR_INVALID
    p = gkm.GraphParams(5, 0, 10, 128, 0, 0, 0)
    assert lib.gk_build_knn_graph(P, 100, 4, 4, ctypes.byref(p), P, P, None, None, ws, 1 << 30,
                                  None) == gkm.GK_ERR_INVALID
    p = gkm.GraphParams(5, 50, 10, 128, 0, 7, 0)
    assert lib.gk_build_knn_graph(P, 100, 4, 4, ctypes.byref(p), P, P, None, None, ws, 1 << 30,
                                  None) == gkm.GK_ERR_INVALID
    assert lib.gk_graph_recall(P, 10, 4, 4, P, 2, P, 0, None, None, P, ws, 1 << 20, None) == gkm.GK_ERR_INVALID
    assert b"m = 0" in lib.gk_last_error()
    assert lib.gk_graph_recall(P, 10, 4, 4, P, 2, P, 5, None, None, None, ws, 1 << 20, None) == gkm.GK_ERR_INVALID
    assert gkm.workspace_size(gkm.GK_OP_RECALL, 1000, 4, 100) > gkm.workspace_size(gkm.GK_OP_RECALL, 1000, 4, 1)
    assert gkm.workspace_size(gkm.GK_OP_BUILD, 1000, 4, 100) == 0  # the build has its own query
    assert lib.gk_two_means_tree(P, 10, 4, 4, 0, 2, 0, P, ws, 1 << 20, None) == gkm.GK_ERR_INVALID
    assert b"k = 0" in lib.gk_last_error()
    assert lib.gk_two_means_tree(P, 10, 4, 4, 11, 2, 0, P, ws, 1 << 20, None) == gkm.GK_ERR_INVALID
    assert lib.gk_two_means_tree(P, 10, 4, 4, 3, -1, 0, P, ws, 1 << 20, None) == gkm.GK_ERR_INVALID
    assert b"iters" in lib.gk_last_error()
    assert lib.gk_two_means_tree(P, 10, 4, 4, 3, 2, 0, None, ws, 1 << 20, None) == gkm.GK_ERR_INVALID
    assert lib.gk_two_means_tree(P, 10, 4, 4, 3, 2, 0, P, ws, 16, None) == gkm.GK_ERR_INVALID
    assert b"too small" in lib.gk_last_error()
    # the tree's scratch: two permutations and the keys (16 bytes per sample) plus 2 d floats per cluster of the
    # deepest complete depth
    big, small = (gkm.workspace_size(gkm.GK_OP_TREE, 100000, 64, k) for k in (4096, 2))
    assert big - small >= (4096 - 2) * 2 * 64 * 4 and small >= 100000 * 16
    assert lib.gk_read_status(None, None) == gkm.GK_ERR_INVALID
    # the boost form: d up to 1024, 1 <= k <= n, the state arrays, kappa, the visit count and sequence
    big = 1 << 30
    assert gkm.workspace_size(gkm.GK_OP_BOOST, 100000, 64, 100) > gkm.workspace_size(gkm.GK_OP_BOOST, 1000, 64, 100)
    assert lib.gk_boost_init(P, 10, 1025, 1025, P, 2, P, P, P, ws, big, None) == gkm.GK_ERR_INVALID
    assert b"1024" in lib.gk_last_error()
    assert lib.gk_boost_init(P, 10, 4, 4, P, 0, P, P, P, ws, big, None) == gkm.GK_ERR_INVALID
    assert lib.gk_boost_init(P, 10, 4, 4, P, 11, P, P, P, ws, big, None) == gkm.GK_ERR_INVALID
    assert b"k = 11" in lib.gk_last_error()
    assert lib.gk_boost_init(P, 10, 4, 4, P, 2, None, P, P, ws, big, None) == gkm.GK_ERR_INVALID
    assert lib.gk_boost_init(P, 10, 4, 4, None, 2, P, P, P, ws, big, None) == gkm.GK_ERR_INVALID
    assert b"labels" in lib.gk_last_error()
    assert lib.gk_boost_init(P, 10, 4, 4, P, 2, P, P, P, ws, 16, None) == gkm.GK_ERR_INVALID
    assert b"too small" in lib.gk_last_error()
    assert lib.gk_boost_epoch(P, 10, 4, 4, P, 10, P, 5, P, 2, P, P, P, None, ws, big, None) == gkm.GK_ERR_INVALID
    assert b"kappa" in lib.gk_last_error()
    assert lib.gk_boost_epoch(P, 10, 4, 4, P, 3, P, -1, P, 2, P, P, P, None, ws, big, None) == gkm.GK_ERR_INVALID
    assert b"m = -1" in lib.gk_last_error()
    assert lib.gk_boost_epoch(P, 10, 4, 4, P, 3, None, 5, P, 2, P, P, P, None, ws, big, None) == gkm.GK_ERR_INVALID
    assert lib.gk_boost_epoch(P, 10, 4, 4, None, 3, P, 5, P, 2, P, P, P, None, ws, big, None) == gkm.GK_ERR_INVALID
    assert lib.gk_boost_epoch_bf16(P, 10, 2000, 2000, P, 3, P, 5, P, 2, P, P, P, None, ws, big,
                                   None) == gkm.GK_ERR_INVALID
