"""Free-running parity: the library's one-call graph construction (Alg. 3) and fit (Alg. 2, closest-centroid
rule) against the FP64 oracle run from the same seeds, each side on its own state from start to end.

Where floating point decides an argmin, the two sides may part at a near tie (two candidate clusters within
1e-5 relative), and a k-means run that parts once goes on differently.  These inputs are chosen so that the
oracle meets no near tie at any assignment of the path (its margin report says so; the test asserts it), and
they are SIFT-shaped integers, whose pair distances are exact in FP32 and in the BF16 Gram: so every label,
every graph row and the whole distortion log must agree, element by element, with no exemption."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1705_01813_gb300 import datagen
from tests import parity as P
from tests.freerun import oracle_path

torch = pytest.importorskip("torch")

KAPPA, XI, TAU, CAP, ITERS = 50, 50, 10, 128, 10
# (n, seed): SIFT-shaped samples on which the oracle's smallest assignment margin over the whole path is >= 1e-5
CASES = [(1000, 1), (3000, 11)]


def _inputs(n, seed):
    X = datagen.sift_like(n, 128, n_latent=max(10, n // 100), seed=seed)
    return X, n // 100


def test_stepwise_oracle_equals_its_one_call_functions():
    n, seed = CASES[0]
    X, k = _inputs(n, seed)
    r = oracle_path(O, X, KAPPA, XI, TAU, CAP, seed, k, ITERS, seed + 1)
    gi, gd, lb, eb = O.build_graph(X, KAPPA, xi=XI, tau=TAU, max_cluster=CAP, seed=seed)
    assert np.array_equal(gi, r["g_idx"]) and np.array_equal(gd, r["g_dist"])
    assert np.array_equal(lb, r["labels_build"]) and np.array_equal(eb, np.asarray(r["e_build"]))
    L, C, _, E = O.fit(X, k, gi, ITERS, O.init_labels(n, k, seed + 1))
    assert np.array_equal(L, r["labels"]) and np.array_equal(C, r["C"]) and np.array_equal(E, np.asarray(r["e_fit"]))


@pytest.mark.parametrize("n,seed", CASES)
def test_cases_meet_no_near_tie(n, seed):
    X, k = _inputs(n, seed)
    r = oracle_path(O, X, KAPPA, XI, TAU, CAP, seed, k, ITERS, seed + 1)
    assert min(r["margins"]) >= 1e-5, r["margins"]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n,seed", CASES)
def test_free_running_path_equals_oracle(n, seed, precision):
    from paper_1705_01813_gb300 import gkm
    X, k = _inputs(n, seed)
    ref = oracle_path(O, X, KAPPA, XI, TAU, CAP, seed, k, ITERS, seed + 1)
    assert min(ref["margins"]) >= 1e-5  # the precondition of element-wise equality
    Xd = torch.from_numpy(X).cuda()
    gi, gd, lb, eb = gkm.build_knn_graph(Xd, KAPPA, xi=XI, tau=TAU, max_cluster=CAP, seed=seed, precision=precision)
    lab, C, cnt, ef = gkm.kmeans_fit(Xd, k, gi, ITERS, seed=seed + 1, precision=precision)
    torch.cuda.synchronize()
    # graph: ids and distances bit for bit (integer samples: every pair distance is an exact integer)
    assert np.array_equal(gi.cpu().numpy(), ref["g_idx"])
    assert np.array_equal(gd.cpu().numpy().astype(np.float64), ref["g_dist"])
    # labels element by element, at k0 after the construction and at k after the fit
    assert np.array_equal(lb.cpu().numpy(), ref["labels_build"])
    assert np.array_equal(lab.cpu().numpy(), ref["labels"])
    assert np.array_equal(cnt.cpu().numpy(), np.bincount(ref["labels"], minlength=k))
    # centroids per cluster and every distortion of both logs within 1e-5 relative
    P.check_centroids(C.cpu().numpy(), ref["C"], np.bincount(ref["labels"], minlength=k))
    for got, want in zip(eb + ef, ref["e_build"] + ref["e_fit"]):
        P.check_rel(got, want, rel=1e-5, what="distortion")
