"""The precision workload at full size: 21,000,000 x 768 (Zipf(1.1)
component sizes, 1,024 clusters, c=16, k=100, R=300), indexed with the exact
FP16 mode and with the served BF16 and FP8-e4m3 forms (shortlist 4,000
re-ranked in FP32).  A batch of 2,000 queries is searched per dtype.

Checks against the FP64 oracle on samples (the oracle's full build of 21M
rows does not fit a test): sampled rows' assignment is the FP64 argmax over the
centroids; a probed cluster's sorted arrays hold the oracle's keys of its rows
in (key, id) order; sampled queries' routes and keys equal the oracle's.  The
FP16 mode equals the independent SIMT path bit for bit on a prefix.  Per
dtype, recall@10 and the largest relative score error against FP64 brute
force over the whole corpus, and the served forms' agreement with the exact
top-k, are asserted."""
import numpy as np
import pytest

from oracle import lider_oracle as O
from tests import lider_fixtures as F

pytestmark = pytest.mark.gpu

NQ = 2_000
SAMPLE = [0, 1, 2, 333, 777, 1024, 1500, 1999]


@pytest.fixture(scope="module")
def precision():
    import torch

    import bench
    cfg, X, Q, C, A, b = F.workload("precision", nq=NQ)
    Qd = torch.from_numpy(Q).cuda()
    out = {}
    for mode in (3, 2, 4):
        g = F.gpu_index(dict(cfg, score_mode=mode, rerank=cfg["rerank"]), X, C, A, b)
        ids, sc, st, tr = g.search(Qd, cfg["k"], cfg["c"], stats=True, trace=True)
        out[mode] = dict(ids=ids.cpu().numpy(), sc=sc.cpu().numpy(), st=st,
                         tr={k: v.cpu().numpy() for k, v in tr.items()})
        if mode == 3:
            off = g.cluster_offsets()
            j = int(tr["route"][0, 0])
            arrays = [g.export_array(j, l) for l in range(cfg["L"])]
            asg = g.assignment()
            simt_prefix = None
            g.free()
            g = F.gpu_index(dict(cfg, score_mode=1), X, C, A, b)
            simt_prefix = [a.cpu().numpy() for a in g.search(Qd[:256].contiguous(), cfg["k"], cfg["c"])]
        g.free()
        torch.cuda.empty_cache()
    truth = bench.fp64_knn(X, Q[SAMPLE], 10)
    return dict(cfg=cfg, X=X, Q=Q, C=C, A=A, b=b, out=out, off=off, j=j, arrays=arrays, asg=asg,
                simt_prefix=simt_prefix, truth=truth)


def test_precision_partition_sampled_rows(precision):
    X, C, asg = precision["X"], precision["C"], precision["asg"]
    rows = np.sort(np.random.default_rng(2).choice(len(X), 30_000, replace=False))
    C64 = C.astype(np.float64)
    S = X[rows].astype(np.float64) @ C64.T - 0.5 * np.sum(C64 * C64, axis=1)
    best = np.argmax(S, axis=1)
    wrong = best != asg[rows]
    top, got = S[np.arange(len(rows)), best], S[np.arange(len(rows)), asg[rows]]
    assert not np.any(wrong & ((top - got) > 1e-9 * np.maximum(1.0, np.abs(top))))
    sizes = np.diff(precision["off"])
    assert sizes.sum() == len(X) and sizes.max() > 20 * np.median(sizes[sizes > 0])


def test_precision_sorted_arrays_of_a_probed_cluster(precision):
    """The oracle's keys of the cluster's rows (hashed by the oracle), in
    (key, id) order, are the exported arrays (boundary-flagged keys excepted)."""
    cfg = precision["cfg"]
    for l, (keys, ids) in enumerate(precision["arrays"]):
        assert len(ids) == precision["off"][precision["j"] + 1] - precision["off"][precision["j"]]
        ok, fl, _ = O.hash_keys(precision["X"][np.sort(ids)], precision["A"], precision["b"], cfg["L"], cfg["m"],
                                cfg["W"])
        order = np.lexsort((np.sort(ids), ok[:, l]))
        ref_keys, ref_ids, ref_fl = ok[order, l], np.sort(ids)[order], fl[order, l]
        diff = (keys != ref_keys) | (ids != ref_ids)
        assert not np.any(diff & ~ref_fl), l


def test_precision_routes_and_keys_of_sampled_queries(precision):
    cfg, Q, C = precision["cfg"], precision["Q"], precision["C"]
    rt, near, _ = O.route(Q[SAMPLE], C, cfg["c"])
    qk, qf, _ = O.hash_keys(Q[SAMPLE], precision["A"], precision["b"], cfg["L"], cfg["m"], cfg["W"])
    for mode in (3, 2, 4):
        tr = precision["out"][mode]["tr"]
        for r, i in enumerate(SAMPLE):
            assert near[r] or np.array_equal(tr["route"][i], rt[r]), (mode, i)
            kd = tr["qkeys"][i].view(np.uint64) != qk[r]
            assert np.all(qf[r][kd]), (mode, i)


def test_precision_f16_equals_simt_prefix(precision):
    ids, sc = precision["simt_prefix"]
    f16 = precision["out"][3]
    assert np.array_equal(ids, f16["ids"][:256])
    assert np.array_equal(sc.view(np.uint32), f16["sc"][:256].view(np.uint32))


@pytest.mark.parametrize("mode", [3, 2, 4], ids=["f16", "bf16", "fp8"])
def test_precision_recall_and_score_error(precision, mode):
    """Per dtype on the sampled queries: recall@10 against FP64 brute force
    over all 21M rows is the exact mode's (the served forms re-rank their
    shortlist in FP32), and every returned score is its id's exact inner
    product within 1e-5 relative."""
    X, Q = precision["X"], precision["Q"]
    r = precision["out"][mode]
    rec = np.mean([len(set(r["ids"][i, :10].tolist()) & set(precision["truth"][s].tolist())) / 10
                   for s, i in enumerate(SAMPLE)])
    exact_rec = np.mean([len(set(precision["out"][3]["ids"][i, :10].tolist()) & set(precision["truth"][s].tolist()))
                         / 10 for s, i in enumerate(SAMPLE)])
    assert rec >= exact_rec - 0.05, (rec, exact_rec)
    for i in SAMPLE:
        sel = r["ids"][i][r["ids"][i] >= 0]
        ex = X[sel].astype(np.float64) @ Q[i].astype(np.float64)
        assert np.all(np.abs(r["sc"][i][:len(sel)] - ex) <= F.SCORE_RTOL * np.abs(ex) + F.SCORE_ATOL)
    if mode != 3:
        top = r["ids"][:, :10]
        ref = precision["out"][3]["ids"][:, :10]
        agree = np.mean([len(set(top[i].tolist()) & set(ref[i].tolist())) / 10 for i in range(NQ)])
        assert agree >= 0.995, agree
