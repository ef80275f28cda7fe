"""The oracle's graph construction (Alg. 3) and fit (Alg. 2, closest-centroid rule) driven step by step from
Python, recording the near-tie margin of every assignment (test helper, no GPU).  The steps are the
oracle's own functions in the order of or_build_graph and or_fit, so the results equal those one-call
functions' (a CPU test checks it)."""
from __future__ import annotations

import numpy as np


def oracle_path(O, X, kappa, xi, tau, max_cluster, seed, k, iters, fit_seed):
    """Returns a dict: g_idx, g_dist (after the construction), labels_build (at k0), labels, C (after the fit),
    e_build (2 tau + 1 entries), e_fit (2 iters + 1 entries) and margins: the smallest near-tie margin of each
    assignment (tau of the construction, then iters of the fit)."""
    n = X.shape[0]
    k0 = max(1, n // xi)
    gi, gd = O.init_graph(X, kappa, seed)
    L = O.init_labels(n, k0, seed)
    C, _, E, _ = O.update(X, L, k0)
    e_build, margins = [E], []
    for _ in range(tau):
        margins.append(float(O.assign_margin(X, gi, C, L).min()))
        L2, best, _ = O.assign(X, gi, C, L)
        e_build.append(float(np.cumsum(best)[-1]) / n)  # summed in index order, as the C functions do
        C, _, E, _ = O.update(X, L2, k0, C_old=C)
        e_build.append(E)
        gi, gd = O.graph_refine(X, L2, k0, gi, gd, max_cluster)
        L = L2
    labels_build = L
    L = O.init_labels(n, k, fit_seed)
    C, _, E, _ = O.update(X, L, k)
    e_fit = [E]
    for _ in range(iters):
        margins.append(float(O.assign_margin(X, gi, C, L).min()))
        L2, best, _ = O.assign(X, gi, C, L)
        e_fit.append(float(np.cumsum(best)[-1]) / n)
        C, _, E, _ = O.update(X, L2, k, C_old=C)
        e_fit.append(E)
        L = L2
    return {"g_idx": gi, "g_dist": gd, "labels_build": labels_build, "labels": L, "C": C,
            "e_build": e_build, "e_fit": e_fit, "margins": margins}
