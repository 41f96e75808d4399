"""GPU search vs the FP64 oracle at full size on the batched workload
(8,800,000 x 768, Zipf(1.1) component sizes, so uneven clusters; 1,024
clusters, c=16, L=8, m=16, k=100, R=300), searched in the benchmark's calls of
6,250 queries with the FP16 score mode.  A spread sample of the first call's
queries is checked step by step against the oracle; the whole call is checked
against the independent SIMT path (bit for bit on a prefix)."""
import numpy as np
import pytest

from oracle import lider_oracle as O
from tests import lider_fixtures as F

pytestmark = pytest.mark.gpu

CALL = 6_250
SAMPLE = [0, 1, 2, 777, 1234, 2500, 3141, 4096, 5000, 6000, 6249]


@pytest.fixture(scope="module")
def batched():
    import torch
    cfg, X, Q, C, A, b = F.workload("batched", nq=CALL)
    gidx = F.gpu_index(dict(cfg, score_mode=3), X, C, A, b)
    Qd = torch.from_numpy(Q).cuda()
    ids, sc, stats, tr = gidx.search(Qd, cfg["k"], cfg["c"], stats=True, trace=True)
    ref_idx = F.oracle_index(cfg, X, C, A, b)
    ref = O.search(ref_idx, Q[SAMPLE], cfg["k"], cfg["c"], cfg["R"])
    return dict(cfg=cfg, X=X, Q=Q, C=C, A=A, b=b, Qd=Qd, gidx=gidx, ids=ids.cpu().numpy(), sc=sc.cpu().numpy(),
                stats=stats, tr={k: v[SAMPLE] for k, v in tr.items()}, ref_idx=ref_idx, ref=ref)


def test_batched_partition(batched):
    sizes = np.diff(batched["gidx"].cluster_offsets())
    ref = np.bincount(batched["ref_idx"].asg, minlength=batched["cfg"]["n_clusters"])
    moved = int(np.abs(sizes - ref).sum()) // 2
    assert moved <= batched["ref_idx"].asg_near_ties, (moved, batched["ref_idx"].asg_near_ties)
    assert sizes.max() > 20 * np.median(sizes[sizes > 0])        # the clusters are uneven


def test_batched_search_steps(batched):
    bad, exempt = F.check_trace(batched["tr"], batched["ref"])
    assert not bad, bad[:10]
    assert len(exempt) <= 1


def test_batched_topk(batched):
    rows = np.array(SAMPLE)
    bad = F.check_topk(batched["ids"][rows], batched["sc"][rows], batched["ref"].ids, batched["ref"].scores,
                       batched["X"], batched["Q"][rows])
    assert not bad, bad[:10]


def test_batched_counters(batched):
    st = batched["stats"]
    assert st["pairs"] == CALL * 16
    assert st["qkey_clamped"] == 0 and st["select_overflow"] == 0


def test_batched_f16_equals_simt(batched):
    """The first 512 queries of the call through the SIMT path (candidates
    gathered, FP32 FMA): the same ids and scores bit for bit."""
    import torch
    cfg = batched["cfg"]
    g = F.gpu_index(dict(cfg, score_mode=1), batched["X"], batched["C"], batched["A"], batched["b"])
    ids, sc = g.search(batched["Qd"][:512].contiguous(), cfg["k"], cfg["c"])
    g.free()
    assert np.array_equal(ids.cpu().numpy(), batched["ids"][:512])
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), batched["sc"][:512].view(np.uint32))
