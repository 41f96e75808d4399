"""Shared test helpers: seeded workloads, the two builds, parity comparisons.

The oracle and the CUDA path receive the same seeded inputs (corpus, queries,
centroids, projections); nothing the CUDA path computes is fed to the oracle.
"""
from __future__ import annotations

import os

import numpy as np

from oracle import lider_oracle as O
from paper_2205_00970_b300 import configs, synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

SCORE_RTOL = 1e-5     # FP32 scores vs FP64 (relative)
SCORE_ATOL = 1e-6     # floor for scores near zero


def workload(name: str, nq: int | None = None):
    cfg = configs.get(name)
    X = synth.corpus(cfg["seed"], cfg["n"], cfg["d"], cfg["n_comp"], cfg["sigma"], cfg["zipf_s"])
    Q = synth.queries(cfg["seed"], cfg["nq"] if nq is None else nq, cfg["d"], cfg["n_comp"], cfg["sigma"],
                      cfg["zipf_s"])
    C = np.load(os.path.join(GOLDEN, f"centroids_{name}.npy"))
    A, b = synth.projections(cfg["seed"], cfg["L"], cfg["m"], cfg["d"], cfg["W"])
    return cfg, X, Q, C, A, b


def oracle_index(cfg, X, C, A, b):
    return O.build_index(X, C, A, b, cfg["L"], cfg["m"], cfg["W"], cfg["leaves"], B=cfg["B"],
                         hash_kind=cfg.get("hash_kind", O.HASH_PSTABLE), raw_keys=bool(cfg.get("raw_keys", 0)))


def gpu_index(cfg, X, C, A, b, device="cuda"):
    import torch
    from paper_2205_00970_b300 import lider
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return lider.Index(t(X), t(C), t(A), t(b), L=cfg["L"], m=cfg["m"], W=cfg["W"],
                       rmi_leaves=cfg["leaves"], r0=cfg["r0"], B=cfg["B"],
                       score_mode=cfg.get("score_mode", lider.SCORE_TENSOR), rerank=cfg.get("rerank", 0),
                       hash_kind=cfg.get("hash_kind", lider.HASH_PSTABLE),
                       route_kind=cfg.get("route_kind", lider.ROUTE_EXACT), raw_keys=bool(cfg.get("raw_keys", 0)))


def check_topk(gpu_ids, gpu_sc, ref_ids, ref_sc, X, Q, rows=None):
    """Top-k parity: at every rank the GPU's exact (FP64) score equals the
    oracle's within the tolerance, ids are identical wherever the oracle's
    score at that rank is not tied (within tolerance) with a neighbour, and the
    GPU's FP32 scores are within tolerance of FP64.  Returns mismatch notes."""
    bad = []
    rows = range(len(ref_ids)) if rows is None else rows
    for i in rows:
        gi, gs, oi, osc = gpu_ids[i], gpu_sc[i], ref_ids[i], ref_sc[i]
        nv = int(np.sum(oi >= 0))
        if int(np.sum(gi >= 0)) != nv:
            bad.append((i, "count", int(np.sum(gi >= 0)), nv))
            continue
        if nv == 0:
            continue
        if np.any(gi[nv:] != -1) or not np.all(np.isneginf(gs[nv:])):
            bad.append((i, "padding"))
        if len(set(gi[:nv].tolist())) != nv:
            bad.append((i, "duplicate ids"))
        q64 = Q[i].astype(np.float64)
        exact = X[gi[:nv]].astype(np.float64) @ q64
        tol = SCORE_RTOL * np.abs(osc[:nv]) + SCORE_ATOL
        if np.any(np.abs(exact - osc[:nv]) > tol):
            bad.append((i, "rank scores", float(np.max(np.abs(exact - osc[:nv])))))
        if np.any(np.abs(gs[:nv].astype(np.float64) - exact) > SCORE_RTOL * np.abs(exact) + SCORE_ATOL):
            bad.append((i, "fp32 score error"))
        for r in range(nv):
            tied = (r > 0 and abs(osc[r] - osc[r - 1]) <= tol[r]) or \
                   (r + 1 < nv and abs(osc[r] - osc[r + 1]) <= tol[r])
            if not tied and gi[r] != oi[r]:
                bad.append((i, "id", r, int(gi[r]), int(oi[r])))
                break
    return bad


def check_trace(trace, ref: "O.SearchResult", rows=None):
    """Per-step parity of one search.  Route and query keys may differ only
    where the oracle marks a near-tie / boundary; a (query, array) whose key
    differs and a query whose route differs are exempt from the later steps.
    Returns (mismatches, exempt query set)."""
    route = trace["route"].cpu().numpy()
    qkeys = trace["qkeys"].cpu().numpy().view(np.uint64)
    pstar = trace["pstar"].cpu().numpy()
    wstart = trace["wstart"].cpu().numpy()
    wlen = trace["wlen"].cpu().numpy()
    ucount = trace["ucount"].cpu().numpy()
    rows = range(route.shape[0]) if rows is None else rows
    bad, exempt = [], set()
    for i in rows:
        if not np.array_equal(route[i], ref.route[i]):
            if ref.route_near[i]:
                exempt.add(i)
                continue
            bad.append((i, "route", route[i].tolist(), ref.route[i].tolist()))
            continue
        kdiff = qkeys[i] != ref.qkeys[i]
        if np.any(kdiff):
            if np.all(ref.qflags[i][kdiff]):
                exempt.add(i)
                continue
            bad.append((i, "qkey"))
            continue
        for name, g, o in (("pstar", pstar, ref.pstar), ("wstart", wstart, ref.wstart), ("wlen", wlen, ref.wlen)):
            if not np.array_equal(g[i], o[i]):
                bad.append((i, name))
        if not np.array_equal(ucount[i], ref.ucount[i]):
            bad.append((i, "ucount", ucount[i].tolist(), ref.ucount[i].tolist()))
    return bad, exempt
