"""Graph construction and fit driven step by step, with one JSONL record per round and per iteration.

The steps are the library's step entry points in the order of gk_build_knn_graph and gk_kmeans_fit (so labels,
centroids, graph and distortions equal the one-call API's bit for bit); between steps the loop reads, per graph
round (Alg. 3) and per fit iteration (Alg. 2):

  E_assign   distortion after the assignment (mean best squared distance, Eq. 4)
  E_update   distortion after the update (Eq. 2 identity)
  changed    samples whose label changed
  empty      clusters without members
  u          mean number of distinct candidate clusters per sample (own label and the neighbours' labels)
  recall     (graph rounds) top-1 recall of the graph on sampled queries (Sec. 5), through gk_graph_recall

Reading them synchronises the stream once per step, so this loop is for monitoring, not for timing.
"""
from __future__ import annotations

import json

import torch

from . import gkm


def _u(labels, g_idx):
    labs = torch.cat([labels[:, None], labels[g_idx.long()]], 1)
    srt, _ = torch.sort(labs, 1)
    return float((1 + (srt[:, 1:] != srt[:, :-1]).sum(1)).double().mean())


def build_and_fit(X, kappa: int, k: int, xi: int = 50, tau: int = 10, iters: int = 10, max_cluster: int = 128,
                  seed: int = 0, fit_seed: int | None = None, precision: int = 1, recall_queries: int = 100,
                  with_u: bool = True, log_path: str | None = None):
    """Alg. 3 then Alg. 2 with per-step records.  Returns (g_idx, g_dist, labels, C, counts, records); records
    are also appended to log_path as JSON lines when given.  fit_seed defaults to seed + 1."""
    n, d = X.shape
    dev = X.device
    fit_seed = seed + 1 if fit_seed is None else fit_seed
    k0 = max(1, n // xi)
    kmax = max(k0, k)
    ws = gkm.workspace(max(gkm.workspace_size(gkm.GK_OP_FIT, n, d, kmax, kappa),
                           gkm.workspace_size(gkm.GK_OP_REFINE, n, d, kmax, kappa)), dev)
    i32 = torch.int32
    off = torch.empty(kmax + 1, dtype=i32, device=dev)
    mem = torch.empty(n, dtype=i32, device=dev)
    cnt = torch.empty(kmax, dtype=i32, device=dev)
    la, lb = torch.empty(n, dtype=i32, device=dev), torch.empty(n, dtype=i32, device=dev)
    s_asg = torch.empty(1, dtype=torch.float64, device=dev)
    s_upd = torch.empty(1, dtype=torch.float64, device=dev)
    chg = torch.empty(1, dtype=torch.int64, device=dev)
    gq = torch.Generator(device=dev)
    gq.manual_seed(seed + 7)
    queries = torch.randint(0, n, (min(n, recall_queries),), generator=gq, device=dev, dtype=i32)
    records = []

    def record(phase, step, kk, labels_in, g_idx, with_recall):
        rec = {"phase": phase, "step": step, "k": kk, "E_assign": float(s_asg.item()) / n,
               "E_update": float(s_upd.item()) / n, "changed": int(chg.item()),
               "empty": int((cnt[:kk] == 0).sum().item())}
        if with_u:
            rec["u"] = _u(labels_in, g_idx)
        if with_recall:
            hits, _, _ = gkm.graph_recall(X, g_idx, queries)
            rec["recall"] = int(hits.item()) / queries.numel()
        records.append(rec)
        if log_path:
            with open(log_path, "a") as f:
                f.write(json.dumps(rec) + "\n")

    # Alg. 3: random graph and labels at k0, then tau rounds of {assign, group, update, refine}
    gi, gd = gkm.init_graph(X, kappa, seed, ws=ws)
    gkm.init_labels(n, k0, seed, out=la)
    C0 = torch.zeros((k0, d), device=dev)
    gkm.group_by_label(la, k0, off, mem, cnt, ws=ws)
    gkm.update_from_groups(X, off, mem, k0, C0, cnt, s_upd, ws=ws)
    cur, nxt = la, lb
    for t in range(tau):
        gkm.assign_step(X, gi, C0, cur, nxt, None, s_asg, chg, precision, mem, ws=ws)
        gkm.group_by_label(nxt, k0, off, mem, cnt, ws=ws)
        gkm.update_from_groups(X, off, mem, k0, C0, cnt, s_upd, ws=ws)
        gkm.graph_refine_groups(X, off, mem, k0, gi, gd, max_cluster, precision, ws=ws)
        record("build", t, k0, cur, gi, True)
        cur, nxt = nxt, cur
    # Alg. 2 at k on the constructed graph: seeded labels, then iters of {assign, group, update}
    lab, other = torch.empty(n, dtype=i32, device=dev), torch.empty(n, dtype=i32, device=dev)
    gkm.init_labels(n, k, fit_seed, out=lab)
    C = torch.zeros((k, d), device=dev)
    gkm.group_by_label(lab, k, off, mem, cnt, ws=ws)
    gkm.update_from_groups(X, off, mem, k, C, cnt, s_upd, ws=ws)
    cur, nxt = lab, other
    for t in range(iters):
        gkm.assign_step(X, gi, C, cur, nxt, None, s_asg, chg, precision, mem, ws=ws)
        gkm.group_by_label(nxt, k, off, mem, cnt, ws=ws)
        gkm.update_from_groups(X, off, mem, k, C, cnt, s_upd, ws=ws)
        record("fit", t, k, cur, gi, False)
        cur, nxt = nxt, cur
    status = gkm.read_status(ws)
    if status != gkm.GK_OK:
        raise gkm.GkError(status, gkm.load().gk_last_error().decode())
    return gi, gd, cur, C, cnt[:k].clone(), records
