"""Fidelity variants at full bench size (mid: 1,000,000 x 768, 256 clusters,
c=8, L=8, k=100, R=300), searched as one batch of 10,000 queries in the FP16
mode; a spread sample is checked step by step against the FP64 oracle.

- core_route: the Layer-1 centroids retriever routes every query (Sec. 3.2);
- hyperplane: 32-bit hyperplane hashkeys, B = 3 (Sec. 4.1).

The sample is also searched on its own, and its RMI diagnostics (Sec. 7.4:
out-of-range and large-error predictions) must equal the oracle's counts."""
import numpy as np
import pytest

from oracle import lider_oracle as O
from tests import lider_fixtures as F

pytestmark = pytest.mark.gpu

SAMPLE = [0, 1, 2, 3, 977, 4096, 5000, 8191, 9999] + list(range(123, 10000, 997))
VARIANTS = {
    "core_route": dict(route_kind=O.ROUTE_CORE),
    "hyperplane": dict(hash_kind=O.HASH_HYPERPLANE, m=32, B=3),
}


@pytest.fixture(scope="module", params=list(VARIANTS))
def mid_variant(request):
    import torch
    cfg, X, Q, C, A, b = F.workload("mid")
    cfg = dict(cfg, score_mode=3, **VARIANTS[request.param])
    if cfg["m"] != F.configs.get("mid")["m"]:
        A, b = F.synth.projections(cfg["seed"], cfg["L"], cfg["m"], cfg["d"], cfg["W"])
    g = F.gpu_index(cfg, X, C, A, b)
    Qd = torch.from_numpy(Q).cuda()
    ids, sc, _, tr = g.search(Qd, cfg["k"], cfg["c"], stats=True, trace=True)
    _, _, st_sample = g.search(Qd[SAMPLE].contiguous(), cfg["k"], cfg["c"], stats=True)
    g.free()
    ref_idx = F.oracle_index(cfg, X, C, A, b)
    ref = O.search(ref_idx, Q[SAMPLE], cfg["k"], cfg["c"], cfg["R"], route_kind=cfg.get("route_kind", 0))
    return dict(name=request.param, cfg=cfg, X=X, Q=Q, ids=ids.cpu().numpy(), sc=sc.cpu().numpy(),
                tr={k: v[SAMPLE] for k, v in tr.items()}, st_sample=st_sample, ref_idx=ref_idx, ref=ref)


def test_mid_variant_steps_and_topk(mid_variant):
    bad, exempt = F.check_trace(mid_variant["tr"], mid_variant["ref"])
    assert not bad, bad[:10]
    assert len(exempt) <= 1
    rows = [i for i in range(len(SAMPLE)) if i not in exempt]
    bad = F.check_topk(mid_variant["ids"][SAMPLE], mid_variant["sc"][SAMPLE], mid_variant["ref"].ids,
                       mid_variant["ref"].scores, mid_variant["X"], mid_variant["Q"][SAMPLE], rows=rows)
    assert not bad, bad[:10]


def test_mid_variant_rmi_diagnostics(mid_variant):
    cfg, ref = mid_variant["cfg"], mid_variant["ref"]
    _, exempt = F.check_trace(mid_variant["tr"], ref)
    want = O.rmi_diagnostics(mid_variant["ref_idx"], ref.qkeys, ref.route, cfg["k"])
    st = mid_variant["st_sample"]
    got = (st["rmi_oor"], st["rmi_le"], st["rmi_oor_le"])
    slack = len(exempt) * cfg["c"] * cfg["L"]
    assert all(abs(a - b) <= slack for a, b in zip(got, want)), (got, want, slack)
