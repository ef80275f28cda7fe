"""The precision autotuner: it times every level on the caller's data without changing the graph or the
labels, picks the level with the smallest weighted time, and caches the choice per shape."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_tuner_picks_a_level_and_leaves_inputs_alone():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01813_gb300 import gkm, tune
    g = np.random.default_rng(3)
    X = torch.from_numpy((g.uniform(-10, 10, (40, 64))[g.integers(0, 40, 30000)]
                          + g.standard_normal((30000, 64))).astype(np.float32)).cuda()
    gi, gd, lab, _ = gkm.build_knn_graph(X, 16, xi=50, tau=2, seed=1)
    gi0, gd0, lab0 = gi.clone(), gd.clone(), lab.clone()
    r = tune.tune_precision(X, gi, gd, lab, 600, tau=2, iters=3, use_cache=False)
    assert torch.equal(gi, gi0) and torch.equal(gd, gd0) and torch.equal(lab, lab0)
    assert r["level"] in (0, 1, 2, 3, 4) and r["group_width"] in (0, 4, 8)
    assert r["precision"] == r["level"] | (r["group_width"] << 8)
    assert r["score_ms"][r["level"]] == min(r["score_ms"].values())
    assert set(r["assign_ms"]) == {0, 1, 2, 3, 4}
    r2 = tune.tune_precision(X, gi, gd, lab, 600, tau=2, iters=3)
    assert tune.tune_precision(X, gi, gd, lab, 700, tau=2, iters=3) is r2  # same shape bucket: cached
    rb = tune.tune_precision(X.to(torch.bfloat16), gi, gd, lab, 600, tau=2, iters=3, use_cache=False)
    assert set(rb["assign_ms"]) == {0, 1, 2, 4}  # no tensor-core screening for BF16 samples
