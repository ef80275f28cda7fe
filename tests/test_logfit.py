"""The logged step-by-step driver: the one-call API's results bit for bit, and one sensible JSONL record per graph
round and per fit iteration."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_logged_driver_equals_one_call_api(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_01813_gb300 import datagen, gkm, logfit
    X = torch.from_numpy(datagen.gauss_mixture(20000, 32, 200, seed=11)).cuda()
    kappa, k, tau, iters = 20, 200, 5, 6
    path = tmp_path / "fit.jsonl"
    gi, gd, lab, C, cnt, recs = logfit.build_and_fit(X, kappa, k, tau=tau, iters=iters, seed=3, precision=1,
                                                     log_path=str(path))
    gi1, gd1, _, blog = gkm.build_knn_graph(X, kappa, 50, tau, 128, 3, precision=1)
    lab1, C1, cnt1, flog = gkm.kmeans_fit(X, k, gi1, iters, seed=4, precision=1)
    assert torch.equal(gi, gi1) and torch.equal(gd, gd1)
    assert torch.equal(lab, lab1) and torch.equal(C, C1) and torch.equal(cnt, cnt1)
    build = [r for r in recs if r["phase"] == "build"]
    fit = [r for r in recs if r["phase"] == "fit"]
    assert len(build) == tau and len(fit) == iters
    assert [r["E_assign"] for r in build] == blog[1::2] and [r["E_update"] for r in build] == blog[2::2]
    assert [r["E_assign"] for r in fit] == flog[1::2] and [r["E_update"] for r in fit] == flog[2::2]
    for r in recs:
        assert 0 <= r["changed"] <= 20000 and 0 <= r["empty"] <= r["k"] and 1.0 <= r["u"] <= kappa + 1
    assert all(0.0 <= r["recall"] <= 1.0 for r in build)
    assert build[-1]["recall"] >= build[0]["recall"]  # the graph improves over the rounds (Sec. 4.3)
    E = [r["E_update"] for r in fit]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(E, E[1:]))
    lines = [json.loads(s) for s in path.read_text().splitlines()]
    assert lines == recs
