"""Fidelity variants on the GPU against the FP64 oracle (tiny workload, all
1,000 queries): hyperplane ESK-LSH hashkeys (Sec. 4.1, one bit per hash,
B = 3), the Layer-1 centroids retriever (Sec. 3.2: a core model over the
centroids routes each query), RMIs learned on raw keys (no re-scaling), and
the OOR/LE diagnostics of Sec. 7.4 in the search counters.

Every step is compared as in the plain parity tests (route, query keys,
lower bounds, windows, candidate counts, top-k); the SIMT and the FP16
tensor-core paths must also agree bit for bit.  The diagnostics counters
must equal the oracle's counts over the same (query, cluster, array)
triples, except on triples of queries the per-step comparison exempts
(their route or keys may differ by a near-tie or a hash boundary)."""
import numpy as np
import pytest

from oracle import lider_oracle as O
from tests import lider_fixtures as F

pytestmark = pytest.mark.gpu

VARIANTS = {
    "hyperplane": dict(hash_kind=O.HASH_HYPERPLANE, m=16, B=3),
    "core_route": dict(route_kind=O.ROUTE_CORE),
    "raw_keys": dict(raw_keys=1),
    "hyperplane_core_route": dict(hash_kind=O.HASH_HYPERPLANE, m=16, B=3, route_kind=O.ROUTE_CORE),
}
MODES = [1, 3]          # SIMT, FP16 tensor cores (tensor-core hashing and routing)


@pytest.fixture(scope="module", params=list(VARIANTS))
def variant(request):
    import torch
    name = request.param
    cfg, X, Q, C, A0, b0 = F.workload("tiny")
    cfg = dict(cfg, **VARIANTS[name])
    if cfg["m"] != F.configs.get("tiny")["m"]:
        A0, b0 = F.synth.projections(cfg["seed"], cfg["L"], cfg["m"], cfg["d"], cfg["W"])
    ref_idx = F.oracle_index(cfg, X, C, A0, b0)
    ref = O.search(ref_idx, Q, cfg["k"], cfg["c"], cfg["R"], route_kind=cfg.get("route_kind", O.ROUTE_EXACT))
    Qd = torch.from_numpy(Q).cuda()
    out = {}
    for mode in MODES:
        g = F.gpu_index(dict(cfg, score_mode=mode), X, C, A0, b0)
        ids, sc, st, tr = g.search(Qd, cfg["k"], cfg["c"], stats=True, trace=True)
        out[mode] = (ids.cpu().numpy(), sc.cpu().numpy(), st, tr)
        g.free()
    return dict(name=name, cfg=cfg, X=X, Q=Q, ref_idx=ref_idx, ref=ref, out=out)


@pytest.mark.parametrize("mode", MODES)
def test_variant_steps_and_topk(variant, mode):
    ids, sc, st, tr = variant["out"][mode]
    bad, exempt = F.check_trace(tr, variant["ref"])
    assert not bad, bad[:10]
    assert len(exempt) <= 5, len(exempt)
    rows = [i for i in range(len(ids)) if i not in exempt]
    bad = F.check_topk(ids, sc, variant["ref"].ids, variant["ref"].scores, variant["X"], variant["Q"], rows=rows)
    assert not bad, bad[:10]
    assert st["qkey_clamped"] == 0


def test_variant_paths_agree_bit_for_bit(variant):
    a, b = variant["out"][1], variant["out"][3]
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))


def test_variant_rmi_diagnostics(variant):
    cfg, ref = variant["cfg"], variant["ref"]
    want = O.rmi_diagnostics(variant["ref_idx"], ref.qkeys, ref.route, cfg["k"])
    for mode in MODES:
        _, _, st, tr = variant["out"][mode]
        _, exempt = F.check_trace(tr, ref)
        slack = len(exempt) * cfg["c"] * cfg["L"]
        got = (st["rmi_oor"], st["rmi_le"], st["rmi_oor_le"])
        for g, w in zip(got, want):
            assert abs(g - w) <= slack, (variant["name"], mode, got, want, slack)
        assert st["rmi_oor_le"] <= min(st["rmi_oor"], st["rmi_le"])


def test_core_route_differs_from_exact_scan_but_stays_close():
    """The centroids retriever is approximate: on tiny (16 clusters, Rc = 8
    positions of 16 per array, L = 4) it must still find most of the exact
    scan's clusters, and its routes must be valid (distinct, in range)."""
    import torch
    cfg, X, Q, C, A, b = F.workload("tiny")
    g = F.gpu_index(dict(cfg, route_kind=O.ROUTE_CORE, score_mode=1), X, C, A, b)
    _, _, _, tr = g.search(torch.from_numpy(Q).cuda(), cfg["k"], cfg["c"], stats=True, trace=True)
    g.free()
    route = tr["route"].cpu().numpy()
    exact, _, _ = O.route(Q, C, cfg["c"])
    assert np.all((route >= 0) & (route < cfg["n_clusters"]))
    assert all(len(set(r)) == cfg["c"] for r in route.tolist())
    overlap = np.mean([len(set(a) & set(e)) / cfg["c"] for a, e in zip(route.tolist(), exact.tolist())])
    assert 0.5 < overlap <= 1.0, overlap


@pytest.mark.parametrize("case", ["core_route_all_clusters", "hyperplane_64_bits"])
def test_variant_edge_cases(case):
    """Edges of the variants on tiny: the Layer-1 route probing every cluster
    (c = n_clusters = 16, each window spans all centroids, so the route is the
    exact scan's order), and hyperplane keys that use all 64 bits (m = 64)."""
    import torch
    cfg, X, Q, C, A, b = F.workload("tiny")
    if case == "core_route_all_clusters":
        cfg = dict(cfg, route_kind=O.ROUTE_CORE, c=cfg["n_clusters"])
    else:
        cfg = dict(cfg, hash_kind=O.HASH_HYPERPLANE, m=64, B=3)
        A, b = F.synth.projections(cfg["seed"], cfg["L"], cfg["m"], cfg["d"], cfg["W"])
    nq = 200
    ref_idx = F.oracle_index(cfg, X, C, A, b)
    ref = O.search(ref_idx, Q[:nq], cfg["k"], cfg["c"], cfg["R"], route_kind=cfg.get("route_kind", O.ROUTE_EXACT))
    out = []
    for mode in MODES:
        g = F.gpu_index(dict(cfg, score_mode=mode), X, C, A, b)
        ids, sc, _, tr = g.search(torch.from_numpy(Q[:nq]).cuda(), cfg["k"], cfg["c"], stats=True, trace=True)
        g.free()
        bad, exempt = F.check_trace(tr, ref)
        assert not bad, (case, mode, bad[:5])
        assert len(exempt) <= 2
        ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
        rows = [i for i in range(nq) if i not in exempt]
        bad = F.check_topk(ids, sc, ref.ids, ref.scores, X, Q[:nq], rows=rows)
        assert not bad, (case, mode, bad[:5])
        out.append((ids, sc))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1].view(np.uint32), out[1][1].view(np.uint32))
    if case == "core_route_all_clusters":
        exact, _, _ = O.route(Q[:nq], C, cfg["c"])
        np.testing.assert_array_equal(ref.route, exact)
