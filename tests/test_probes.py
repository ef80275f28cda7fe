"""The benchmark's measurement probes (benchlib/probes.cu, their own library) read what they claim: the gather
probe's per-warp sums add up to the sum of the indexed table rows (indices outside the table read nothing),
and the argument checks refuse bad shapes."""
import ctypes

import pytest

torch = pytest.importorskip("torch")


def test_probe_library_builds_and_checks_arguments():
    from benchlib import probes
    probes.build()
    if torch.cuda.is_available():
        pytest.skip("argument checks with fake pointers run on CPU-only hosts")
    L = probes.load()
    P = ctypes.c_void_p(0x10000000)
    assert L.gkb_probe_gather(P, 10, 6, P, 4, P, None) == 1  # row_floats not a multiple of 4
    assert L.gkb_probe_gather(P, 10, 1024, P, 4, P, None) == 1
    assert L.gkb_probe_gather(None, 10, 8, P, 4, P, None) == 1
    assert L.gkb_probe_gather(ctypes.c_void_p(0x10000004), 10, 8, P, 4, P, None) == 1
    assert L.gkb_probe_fma(None, 10, None) == 1
    assert probes.sink_floats() == 152 * 8 * 8


def test_probes_are_not_in_the_clustering_library():
    from paper_1705_01813_gb300 import build_native, gkm
    build_native.build()
    L = gkm.load()
    for name in ("gk_probe_gather", "gk_probe_fma"):
        assert not hasattr(L, name)


@pytest.mark.gpu
@pytest.mark.parametrize("rows,width,count", [(1000, 128, 100_003), (257, 512, 9_999), (64, 4, 50_000)])
def test_probe_gather_reads_the_indexed_rows(rows, width, count):
    from benchlib import probes
    g = torch.Generator(device="cuda")
    g.manual_seed(rows)
    table = torch.rand((rows, width), generator=g, device="cuda")
    idx = torch.randint(-5, rows + 5, (count,), generator=g, device="cuda", dtype=torch.int32)
    sink = torch.zeros(probes.sink_floats(), device="cuda")
    nb = probes.probe_gather(table, idx, sink, torch.cuda.current_stream())
    assert nb == count * width * 4
    ok = (idx >= 0) & (idx < rows)
    want = table.double().sum(1)[idx[ok].long()].sum().item()
    assert abs(sink.double().sum().item() - want) <= 1e-4 * want


@pytest.mark.gpu
def test_probe_fma_runs():
    from benchlib import probes
    sink = torch.full((probes.sink_floats(),), float("nan"), device="cuda")
    probes.probe_fma(sink, 1000, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.isfinite(sink).all()
    m = probes.measure(reps=2)
    assert m["l2_gather_gbs"] > 0 and m["hbm_gather_gbs"] > 0 and m["fp32_ffma2_tflops"] > 0
