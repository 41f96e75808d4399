"""GPU search vs the FP64 oracle at full bench size: the mid workload
(1,000,000 x 768, 256 clusters, c=8, L=8, m=16, RMI 1,024 leaves, k=100,
R=300), searched as one batch of 10,000 queries exactly as the benchmark
launches it; a spread sample of queries is checked step by step."""
import numpy as np
import pytest

from oracle import lider_oracle as O
from tests import lider_fixtures as F

pytestmark = pytest.mark.gpu

SAMPLE = [0, 1, 2, 3, 977, 1999, 3333, 4096, 5000, 6789, 7777, 8191, 9000, 9998, 9999] + \
    list(range(123, 10000, 701))


@pytest.fixture(scope="module")
def mid():
    import torch
    cfg, X, Q, C, A, b = F.workload("mid")
    gidx = F.gpu_index(cfg, X, C, A, b)
    ids, sc, stats, tr = gidx.search(torch.from_numpy(Q).cuda(), cfg["k"], cfg["c"], stats=True, trace=True)
    ref_idx = F.oracle_index(cfg, X, C, A, b)
    ref = O.search(ref_idx, Q[SAMPLE], cfg["k"], cfg["c"], cfg["R"])
    return dict(cfg=cfg, X=X, Q=Q, C=C, A=A, b=b, gidx=gidx, ids=ids.cpu().numpy(), sc=sc.cpu().numpy(), stats=stats,
                tr={k: v[SAMPLE] for k, v in tr.items()}, ref_idx=ref_idx, ref=ref)


def test_mid_partition(mid):
    off = mid["gidx"].cluster_offsets()
    np.testing.assert_array_equal(np.diff(off), np.bincount(mid["ref_idx"].asg, minlength=256))


def test_mid_sorted_arrays_of_probed_clusters(mid):
    probed = sorted(set(mid["ref"].route[:4].ravel().tolist()))
    for j in probed:
        cm = mid["ref_idx"].core(j, fit=False)
        for l in range(mid["cfg"]["L"]):
            keys, ids = mid["gidx"].export_array(j, l)
            diff = (keys != cm.keys[l]) | (ids != cm.sorted_ids[l])
            assert not np.any(diff & ~cm.flags[l]), (j, l)


def test_mid_rmi_windows_hold(mid):
    """The GPU-built RMI of a few (cluster, array) pairs keeps every key's
    first position inside its leaf's window."""
    for j, l in [(0, 0), (17, 3), (255, 7)]:
        cm = mid["ref_idx"].core(j, fit=False)
        ks = cm.keys[l]
        g = mid["gidx"].export_rmi(j, l)
        rmi = O.RMI(len(ks), mid["cfg"]["leaves"], g["a0"], g["b0"], g["a"], g["b"], g["e_lo"], g["e_hi"])
        lb = np.searchsorted(ks, ks, side="left")
        for i in range(0, len(ks), 3):
            lf, p = rmi.predict(O.rescale(int(ks[i]), g["x_min"], g["x_max"], len(ks)))
            assert p + g["e_lo"][lf] <= lb[i] <= p + g["e_hi"][lf]


def test_mid_search_steps(mid):
    bad, exempt = F.check_trace(mid["tr"], mid["ref"])
    assert not bad, bad[:10]
    assert len(exempt) <= 1


def test_mid_topk(mid):
    rows = np.array(SAMPLE)
    bad = F.check_topk(mid["ids"][rows], mid["sc"][rows], mid["ref"].ids, mid["ref"].scores, mid["X"],
                       mid["Q"][rows])
    assert not bad, bad[:10]


def test_mid_counters(mid):
    st = mid["stats"]
    assert st["pairs"] == 10_000 * 8 and st["empty_pairs"] == 0
    assert st["candidates"] > 0
    assert st["qkey_clamped"] == 0
    assert st["select_overflow"] == 0


def test_mid_tensor_modes_equal_simt_exactly(mid):
    """At full size, all 10,000 queries: the 3xTF32 and FP16 tensor-core
    paths' results equal the SIMT path's (the exact FP32 top-k of each
    candidate union) bit for bit."""
    import torch
    cfg, X, Q, C, A, b = (mid[n] for n in ("cfg", "X", "Q", "C", "A", "b"))
    Qd = torch.from_numpy(Q).cuda()
    g = F.gpu_index(dict(cfg, score_mode=1), X, C, A, b)
    ids, sc = g.search(Qd, cfg["k"], cfg["c"])
    g.free()
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    diff = np.nonzero(np.any(ids != mid["ids"], axis=1))[0]
    assert diff.size == 0, (diff[:10], diff.size)
    assert np.array_equal(sc.view(np.uint32), mid["sc"].view(np.uint32))
    g = F.gpu_index(dict(cfg, score_mode=3), X, C, A, b)
    fi, fs, st = g.search(Qd, cfg["k"], cfg["c"], stats=True)
    g.free()
    assert st["select_overflow"] == 0 and st["route_fallback"] == 0
    fi, fs = fi.cpu().numpy(), fs.cpu().numpy()
    diff = np.nonzero(np.any(fi != ids, axis=1))[0]
    assert diff.size == 0, (diff[:10], diff.size)
    assert np.array_equal(fs.view(np.uint32), sc.view(np.uint32))
