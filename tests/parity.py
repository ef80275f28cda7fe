"""Comparison rules between the CUDA path and the FP64 oracle.

Tolerances (relative, FP32 path):
  labels         equal, except where the oracle's distance to the GPU's label is
                 within REL of the oracle's best (the two best differ by < REL)
  graph rows     equal ids in equal order, except where the FP64 keys of the
                 differing entries are within REL (near ties)
  centroids      ||C_gpu - C_oracle|| <= REL ||C_oracle|| per centroid
  distortion     within REL
REL = 1e-5.  On integer-valued data every FP32 pair distance is exact, so graph
rows must match bit for bit with no exemption.
"""
import numpy as np

REL = 1e-5


def d2_rows(X, rows, C):
    """FP64 squared distances ||X[rows] - C[...]||^2 (C indexed per row)."""
    return ((X[rows].astype(np.float64) - np.asarray(C, np.float64)) ** 2).sum(-1)


def check_labels(X, C64, gpu_labels, ora_labels, ora_best, rows=None, rel=REL):
    """Labels equal except near ties; returns the number of exempted samples."""
    gl = np.asarray(gpu_labels)
    ol = np.asarray(ora_labels)
    idx = np.arange(gl.shape[0]) if rows is None else np.asarray(rows)
    bad = np.nonzero(gl != ol)[0]
    if bad.size == 0:
        return 0
    dg = d2_rows(X, idx[bad], np.asarray(C64)[gl[bad]])
    ob = np.asarray(ora_best)[bad]
    ok = dg <= ob * (1 + rel) + 1e-30
    assert ok.all(), f"{(~ok).sum()} label mismatches beyond near ties, e.g. sample {idx[bad][~ok][:5]}"
    return int(bad.size)


def check_centroids(C_gpu, C_ora, counts=None, rel=REL):
    Cg = np.asarray(C_gpu, np.float64)
    Co = np.asarray(C_ora, np.float64)
    num = np.linalg.norm(Cg - Co, axis=1)
    den = np.linalg.norm(Co, axis=1)
    sel = np.ones(Cg.shape[0], bool) if counts is None else np.asarray(counts) > 0
    worst = (num[sel] / np.maximum(den[sel], 1e-30)).max() if sel.any() else 0.0
    assert worst <= rel, f"centroid relative error {worst:.3e} > {rel}"
    return float(worst)


def check_rel(a, b, rel=REL, what="value"):
    a, b = float(a), float(b)
    err = abs(a - b) / max(abs(b), 1e-300)
    assert err <= rel, f"{what}: {a!r} vs {b!r} (rel {err:.3e} > {rel})"
    return err


def row_invariants(X, gi, gd, rows=None):
    """GPU rows: sorted by (dist, id), no self, no repeats, stored FP32 distance == recomputed."""
    gi = np.asarray(gi)
    gd = np.asarray(gd)
    n, kappa = gi.shape
    rows = np.arange(n) if rows is None else np.asarray(rows)
    for q, i in enumerate(rows):
        r = gi[q]
        assert (r >= 0).all() and (r < X.shape[0]).all()
        assert i not in r, f"row {i} holds itself"
        assert len(set(r.tolist())) == kappa, f"row {i} repeats an id"
        keys = list(zip(gd[q].tolist(), r.tolist()))
        assert keys == sorted(keys), f"row {i} not sorted"
    # FP32 distance recomputed in FP64 agrees within the FP32 summation bound (d + 2) u
    ref = ((X[rows][:, None, :].astype(np.float64) - X[gi].astype(np.float64)) ** 2).sum(-1)
    bound = (X.shape[1] + 2) * 2.0 ** -24 * 1.01
    err = np.abs(gd - ref) / np.maximum(ref, 1e-30)
    assert ((err <= bound) | (np.abs(gd - ref) <= 1e-30)).all(), f"stored distance off by {err.max():.2e}"


def check_graph(X, gi_gpu, gd_gpu, gi_ora, gd_ora, rows=None, exact=False, rel=REL):
    """Rows equal to the oracle's, except near ties (none allowed when exact)."""
    gi_gpu = np.asarray(gi_gpu)
    gi_ora = np.asarray(gi_ora)
    gd_ora = np.asarray(gd_ora, np.float64)
    rows = np.arange(gi_gpu.shape[0]) if rows is None else np.asarray(rows)
    diff = np.nonzero((gi_gpu != gi_ora).any(1))[0]
    if exact:
        assert diff.size == 0, f"{diff.size} rows differ on exact data, e.g. {rows[diff[:5]]}"
        assert np.array_equal(np.asarray(gd_gpu, np.float64), gd_ora)
        return 0
    for q in diff:
        i = rows[q]
        dg = np.sort(((X[gi_gpu[q]].astype(np.float64) - X[i].astype(np.float64)) ** 2).sum(-1))
        do = gd_ora[q]
        assert np.all(np.abs(dg - do) <= rel * np.maximum(do, 1e-30)), \
            f"row {i}: gpu {gi_gpu[q].tolist()} vs oracle {gi_ora[q].tolist()}"
    return int(diff.size)
