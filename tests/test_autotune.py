"""The autotuner picks launch shapes from the allowed sets by timing searches;
results are the same bit for bit under every launch shape."""
import itertools

import numpy as np
import pytest

from tests import lider_fixtures as F

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 3], ids=["tensor", "f16"])
def test_launch_shapes_do_not_change_results(mode):
    import torch
    from paper_2205_00970_b300 import lider
    cfg, X, Q, C, A, b = F.workload("tiny")
    ix = F.gpu_index(dict(cfg, score_mode=mode), X, C, A, b)
    Qd = torch.from_numpy(Q).cuda()
    ref_ids, ref_sc = (t.cpu().numpy() for t in ix.search(Qd, cfg["k"], cfg["c"]))
    for sel, res, mark, order in itertools.product((64, 512), (64, 512), (32, 256), (0, 1)):
        ix.set_tuning(select_threads=sel, rescore_threads=res, mark_threads=mark, tile_order=order)
        ids, sc = ix.search(Qd, cfg["k"], cfg["c"])
        assert np.array_equal(ids.cpu().numpy(), ref_ids), (sel, res, mark, order)
        assert np.array_equal(sc.cpu().numpy().view(np.uint32), ref_sc.view(np.uint32))
    with pytest.raises(lider.LiderError):
        ix.set_tuning(select_threads=300)
    tune, ms = ix.autotune(Qd[:512].contiguous(), cfg["k"], cfg["c"], reps=3)
    assert tune["select_threads"] in (64, 128, 256, 512) and tune["tile_order"] in (0, 1)
    assert ms > 0 and ix.tuning() == tune
    ids, sc = ix.search(Qd, cfg["k"], cfg["c"])
    assert np.array_equal(ids.cpu().numpy(), ref_ids)
    ix.free()
