"""lider_search_noalloc: search without any device allocation.

Callers that cannot allocate device memory while they search (a service that
reserved its whole GPU budget up front, or code running while another
framework owns the CUDA allocator) use this entry point; its scratch is a
fixed device array inside the library.  These tests call it through the C ABI
and check it against lider_search on two calls in a row, so that contents left
in the shared array by one call cannot leak into the next.
"""
import ctypes

import numpy as np
import pytest

from tests import lider_fixtures as F

pytestmark = pytest.mark.gpu


def _noalloc(lider, idx, Qd, k, c):
    import torch
    nq = Qd.shape[0]
    ids = torch.full((nq, k), -7, dtype=torch.int64, device=Qd.device)
    sc = torch.full((nq, k), 7.0, dtype=torch.float32, device=Qd.device)
    st = lider.Stats()
    rc = lider.raw_call("lider_search_noalloc", idx.handle, Qd.data_ptr(), nq, k, c, ids.data_ptr(),
                        sc.data_ptr(), ctypes.byref(st), torch.cuda.current_stream().cuda_stream)
    return rc, ids, sc, st.as_dict()


@pytest.mark.parametrize("mode,rerank", [(0, 0), (1, 0), (2, 4), (4, 4)], ids=["tensor", "simt", "bf16", "fp8"])
def test_noalloc_matches_search_on_two_calls(mode, rerank):
    """Every score mode carves its own regions from the shared array (the
    served forms their shortlists, SIMT its per-pair lists); a second, smaller
    batch runs over the first call's leftovers."""
    import torch
    from paper_2205_00970_b300 import lider
    cfg, X, Q, C, A, b = F.workload("tiny")
    idx = F.gpu_index(dict(cfg, score_mode=mode, rerank=rerank), X, C, A, b)
    k, c = cfg["k"], cfg["c"]
    batches = [torch.from_numpy(Q).cuda(), torch.from_numpy(Q[500:800]).cuda()]
    for Qd in batches:                       # two calls in a row, different batches
        ref_ids, ref_sc, ref_st = idx.search(Qd, k, c, stats=True)
        rc, ids, sc, st = _noalloc(lider, idx, Qd, k, c)
        assert rc == 0, lider.last_error()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids)
        np.testing.assert_allclose(sc.cpu().numpy(), ref_sc.cpu().numpy(),
                                   rtol=F.SCORE_RTOL, atol=F.SCORE_ATOL)
        assert st == ref_st
    idx.free()


def test_noalloc_rejects_batches_beyond_its_scratch():
    import torch
    from paper_2205_00970_b300 import lider
    cfg, X, Q, C, A, b = F.workload("tiny")
    idx = F.gpu_index(cfg, X, C, A, b)
    nq = 200_000                              # needs far more than the fixed scratch
    Qd = torch.zeros((nq, cfg["d"]), dtype=torch.float32, device="cuda")
    rc, ids, sc, _ = _noalloc(lider, idx, Qd, cfg["k"], cfg["c"])
    assert rc == -4 and "LIDER_NOALLOC_SCRATCH_BYTES" in lider.last_error()
    assert int(ids[0, 0]) == -7                  # nothing was launched
    idx.free()
