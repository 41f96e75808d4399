"""A search captured into a CUDA graph and replayed: the captured search takes
its scratch from a graph allocation and makes no host synchronisation, so each
replay on new query contents returns exactly what an eager search returns."""
import numpy as np
import pytest

from tests import lider_fixtures as F

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4], ids=["tensor", "simt", "bf16", "f16", "fp8"])
def test_search_replays_as_cuda_graph(mode):
    import torch
    cfg, X, Q, C, A, b = F.workload("tiny")
    cfg = dict(cfg, score_mode=mode, rerank=2 if mode in (2, 4) else 0)
    ix = F.gpu_index(cfg, X, C, A, b)
    nq, k, c = 256, cfg["k"], cfg["c"]
    Qbuf = torch.from_numpy(Q[:nq].copy()).cuda()
    ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    sc = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    ix.search(Qbuf, k, c, out=(ids, sc))            # eager first: kernel attributes are set once
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ix.search(Qbuf, k, c, out=(ids, sc), stream=s)
    for off in (0, 300, 600, 744):
        Qbuf.copy_(torch.from_numpy(Q[off:off + nq]))
        g.replay()
        torch.cuda.synchronize()
        ei, es = ix.search(torch.from_numpy(Q[off:off + nq]).cuda(), k, c)
        assert np.array_equal(ids.cpu().numpy(), ei.cpu().numpy()), off
        assert np.array_equal(sc.cpu().numpy().view(np.uint32), es.cpu().numpy().view(np.uint32)), off
    del g
    ix.free()
