"""GPU search vs the FP64 oracle on the tiny workload (10k x 128, 16 clusters,
c=4, L=4, m=8, RMI 16 leaves, k=10): every query, every step."""
import numpy as np
import pytest

from oracle import lider_oracle as O
from tests import lider_fixtures as F

pytestmark = pytest.mark.gpu


MODES = [0, 1, 3]       # 3xTF32 tensor-core scoring, SIMT scoring, FP16 tensor-core scoring
MODE_IDS = ["tensor", "simt", "f16"]


@pytest.fixture(scope="module", params=MODES, ids=MODE_IDS)
def tiny(request):
    import torch
    cfg, X, Q, C, A, b = F.workload("tiny")
    cfg["score_mode"] = request.param
    ref_idx = F.oracle_index(cfg, X, C, A, b)
    gidx = F.gpu_index(cfg, X, C, A, b)
    ref = O.search(ref_idx, Q, cfg["k"], cfg["c"], cfg["R"])
    Qd = torch.from_numpy(Q).cuda()
    return dict(cfg=cfg, X=X, Q=Q, C=C, A=A, b=b, ref_idx=ref_idx, gidx=gidx, ref=ref, Qd=Qd)


def test_partition_matches_oracle(tiny):
    off = tiny["gidx"].cluster_offsets()
    sizes = np.bincount(tiny["ref_idx"].asg, minlength=tiny["cfg"]["n_clusters"])
    assert tiny["ref_idx"].asg_near_ties == 0
    np.testing.assert_array_equal(np.diff(off), sizes)


def test_sorted_arrays_bit_exact(tiny):
    cfg, ref_idx, gidx = tiny["cfg"], tiny["ref_idx"], tiny["gidx"]
    for j in range(cfg["n_clusters"]):
        cm = ref_idx.core(j)
        for l in range(cfg["L"]):
            keys, ids = gidx.export_array(j, l)
            diff = (keys != cm.keys[l]) | (ids != cm.sorted_ids[l])
            assert not np.any(diff & ~cm.flags[l]), (j, l)


def test_rmi_window_invariant_and_root(tiny):
    """Every corpus key's first position lies in its leaf's window, evaluated
    with the GPU-built RMI parameters; the root model matches the oracle's."""
    cfg, ref_idx, gidx = tiny["cfg"], tiny["ref_idx"], tiny["gidx"]
    for j in range(cfg["n_clusters"]):
        cm = ref_idx.core(j)
        for l in range(cfg["L"]):
            g = gidx.export_rmi(j, l)
            ks = cm.keys[l]
            n_c = len(ks)
            assert g["x_min"] == int(ks[0]) and g["x_max"] == int(ks[-1])
            rmi = O.RMI(n_c, cfg["leaves"], g["a0"], g["b0"], g["a"], g["b"], g["e_lo"], g["e_hi"])
            o = cm.rmi[l]
            assert abs(g["b0"] - o.b0) <= 1e-9 * abs(o.b0) + 1e-12
            assert abs(g["a0"] - o.a0) <= 1e-9 * max(abs(o.a0), n_c) + 1e-12
            lb = np.searchsorted(ks, ks, side="left")
            for i in range(n_c):
                r = O.rescale(int(ks[i]), g["x_min"], g["x_max"], n_c)
                lf, p = rmi.predict(r)
                assert p + g["e_lo"][lf] <= lb[i] <= p + g["e_hi"][lf], (j, l, i)


def test_search_steps_match_oracle(tiny):
    cfg = tiny["cfg"]
    ids, sc, stats, tr = tiny["gidx"].search(tiny["Qd"], cfg["k"], cfg["c"], stats=True, trace=True)
    bad, exempt = F.check_trace(tr, tiny["ref"])
    assert not bad, bad[:10]
    assert len(exempt) <= 2
    assert stats["candidates"] == int(tr["ucount"].sum())
    assert stats["pairs"] == cfg["nq"] * cfg["c"]
    assert stats["empty_pairs"] == 0


def test_topk_matches_oracle(tiny):
    cfg, ref = tiny["cfg"], tiny["ref"]
    ids, sc = tiny["gidx"].search(tiny["Qd"], cfg["k"], cfg["c"])
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    bad = F.check_topk(ids, sc, ref.ids, ref.scores, tiny["X"], tiny["Q"])
    assert not bad, bad[:10]


def test_host_path_equals_device_path(tiny):
    import torch
    cfg = tiny["cfg"]
    ids, sc = tiny["gidx"].search(tiny["Qd"], cfg["k"], cfg["c"])
    Qh = torch.from_numpy(tiny["Q"]).pin_memory()
    hid, hsc = tiny["gidx"].search_host(Qh, cfg["k"], cfg["c"])
    assert torch.equal(hid, ids.cpu()) and torch.equal(hsc, sc.cpu())


@pytest.mark.parametrize("pinned", [True, False])
def test_host_path_in_chunks_equals_device_path(tiny, pinned):
    """9,000 queries reach the device in four chunks whose hash and route
    start as each lands; results go straight into pinned (mapped) result
    buffers, or are copied back into pageable ones: either way bit-equal to
    the search of the same queries already on the device."""
    import torch
    from paper_2205_00970_b300 import synth
    cfg = tiny["cfg"]
    Q = synth.queries(cfg["seed"] + 1, 9_000, cfg["d"], cfg["n_comp"], cfg["sigma"], cfg["zipf_s"])
    ids, sc = tiny["gidx"].search(torch.from_numpy(Q).cuda(), cfg["k"], cfg["c"])
    Qh = torch.from_numpy(Q)
    hid = torch.full((len(Q), cfg["k"]), 7, dtype=torch.int64)
    hsc = torch.zeros((len(Q), cfg["k"]), dtype=torch.float32)
    if pinned:
        Qh, hid, hsc = Qh.pin_memory(), hid.pin_memory(), hsc.pin_memory()
    hid, hsc = tiny["gidx"].search_host(Qh, cfg["k"], cfg["c"], hid, hsc)
    assert torch.equal(hid, ids.cpu()) and torch.equal(hsc, sc.cpu())


@pytest.mark.parametrize("pinned", [True, False])
def test_host_path_in_passes_equals_device_path(tiny, pinned):
    """With a probe batch of 2,500 the host path searches 9,000 queries in
    four passes (chunks of 2,500 and 1,500 queries whose copies land on a
    second stream); results and summed counters equal the device search."""
    import torch
    from paper_2205_00970_b300 import synth
    cfg = tiny["cfg"]
    g = tiny["gidx"]
    Q = synth.queries(cfg["seed"] + 2, 9_000, cfg["d"], cfg["n_comp"], cfg["sigma"], cfg["zipf_s"])
    ids, sc, st = g.search(torch.from_numpy(Q).cuda(), cfg["k"], cfg["c"], stats=True)
    Qh = torch.from_numpy(Q)
    hid = torch.full((len(Q), cfg["k"]), 7, dtype=torch.int64)
    hsc = torch.zeros((len(Q), cfg["k"]), dtype=torch.float32)
    if pinned:
        Qh, hid, hsc = Qh.pin_memory(), hid.pin_memory(), hsc.pin_memory()
    before = g.tuning()
    try:
        g.set_tuning(probe_batch=2_500)
        hid, hsc, hst = g.search_host(Qh, cfg["k"], cfg["c"], hid, hsc, stats=True)
    finally:
        g.set_tuning(**before)
    assert hst["passes"] == 4 and st["passes"] == 1
    assert torch.equal(hid, ids.cpu()) and torch.equal(hsc, sc.cpu())
    for key in ("candidates", "pairs", "qkey_boundary", "locate_fallback", "n_queries"):
        assert hst[key] == st[key], key


@pytest.mark.parametrize("nq", [0, 1, 7, 33, 257])
def test_ragged_batches_are_batch_invariant(tiny, nq):
    """A query's result does not depend on its batch-mates or batch size."""
    import torch
    cfg = tiny["cfg"]
    full_ids, full_sc = tiny["gidx"].search(tiny["Qd"], cfg["k"], cfg["c"])
    sub = tiny["Qd"][100:100 + nq].contiguous()
    ids, sc = tiny["gidx"].search(sub, cfg["k"], cfg["c"])
    assert ids.shape == (nq, cfg["k"])
    assert torch.equal(ids, full_ids[100:100 + nq]) and torch.equal(sc, full_sc[100:100 + nq])


def test_exhaustive_search_is_exact_knn(tiny):
    """All clusters probed with R >= every cluster size: exact brute force."""
    import torch
    cfg = dict(tiny["cfg"])
    X, Q, C, A, b = tiny["X"][:2000], tiny["Q"][:50], tiny["C"], tiny["A"], tiny["b"]
    asg, _ = O.assign(X, C)
    k = 1
    cfg["r0"] = int(np.bincount(asg).max())       # R >= every cluster size
    assert cfg["r0"] * k * cfg["L"] <= 4096
    g = F.gpu_index(cfg, X, C, A, b)
    ids, sc = g.search(torch.from_numpy(Q).cuda(), k, cfg["n_clusters"])
    tid, tsc = O.exact_knn(X, Q, k)
    bad = F.check_topk(ids.cpu().numpy(), sc.cpu().numpy(), tid, tsc, X, Q)
    assert not bad, bad[:5]


def test_k_beyond_candidates_pads(tiny):
    import torch
    cfg = dict(tiny["cfg"])
    cfg["r0"] = 1
    X, C, A, b = tiny["X"], tiny["C"], tiny["A"], tiny["b"]
    Q = tiny["Q"][:20]
    g = F.gpu_index(cfg, X, C, A, b)
    k = 600                               # R = 600 per array but clusters are smaller
    ids, sc = g.search(torch.from_numpy(Q).cuda(), k, 1)
    ref = O.search(O.build_index(X, C, A, b, cfg["L"], cfg["m"], cfg["W"], cfg["leaves"]), Q, k, 1, k)
    bad = F.check_topk(ids.cpu().numpy(), sc.cpu().numpy(), ref.ids, ref.scores, X, Q)
    assert not bad, bad[:5]
    assert np.any(ids.cpu().numpy() == -1)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_duplicates_empty_and_singleton_clusters(mode):
    """Duplicate corpus rows (equal keys), a centroid no point chooses (empty
    cluster) and a one-point cluster."""
    import torch
    rng = np.random.default_rng(5)
    d, n = 16, 600
    X = rng.standard_normal((n, d)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X[100:140] = X[3]                                   # 41 identical rows
    X[599] *= 10.0                                      # an outlier with its own centroid
    far = np.full((1, d), 50.0, np.float32)             # nobody's nearest centroid
    lone = X[599:600].copy()
    C = np.concatenate([X[rng.choice(599, 4, replace=False)], far, lone]).astype(np.float32)
    cfg = dict(L=3, m=8, W=0.7, leaves=8, r0=3, B=2, k=5, score_mode=mode)
    A = rng.standard_normal((cfg["L"] * cfg["m"], d)).astype(np.float32)
    b = (rng.random(cfg["L"] * cfg["m"]) * cfg["W"]).astype(np.float32)
    Q = np.concatenate([X[:40], rng.standard_normal((20, d)).astype(np.float32)])
    g = F.gpu_index(cfg, X, C, A, b)
    ref_idx = O.build_index(X, C, A, b, cfg["L"], cfg["m"], cfg["W"], cfg["leaves"], B=cfg["B"])
    sizes = np.diff(g.cluster_offsets())
    assert sizes[4] == 0 and sizes[5] == 1
    for c in (1, 3, 6):
        ids, sc, st, tr = g.search(torch.from_numpy(Q).cuda(), cfg["k"], c, stats=True, trace=True)
        ref = O.search(ref_idx, Q, cfg["k"], c, cfg["r0"] * cfg["k"])
        bad, _ = F.check_trace(tr, ref)
        assert not bad, bad[:5]
        bad = F.check_topk(ids.cpu().numpy(), sc.cpu().numpy(), ref.ids, ref.scores, X, Q)
        assert not bad, bad[:5]
        if c == 6:
            assert st["empty_pairs"] == len(Q)


@pytest.mark.parametrize("mode", [0, 3], ids=["tensor", "f16"])
def test_massive_ties_take_the_multi_level_select(mode):
    """A corpus of 3,000 copies of one vector (plus 1,000 others): a query's
    candidate scores all tie, so the two-pass histogram select cannot bound
    its collection and hands the query to the multi-level select.  Results
    still equal the SIMT path's bit for bit (ties by lower id)."""
    import torch
    rng = np.random.default_rng(11)
    d, n = 32, 4000
    X = rng.standard_normal((n, d)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X[:3000] = X[0]
    C = X[rng.choice(n, 4, replace=False)].astype(np.float32)
    C[0] = X[0]
    cfg = dict(L=1, m=8, W=0.7, leaves=8, r0=256, B=1, k=16)
    A = rng.standard_normal((cfg["L"] * cfg["m"], d)).astype(np.float32)
    b = (rng.random(cfg["L"] * cfg["m"]) * cfg["W"]).astype(np.float32)
    Q = np.concatenate([X[:8] + 1e-3 * rng.standard_normal((8, d)).astype(np.float32),
                        rng.standard_normal((8, d)).astype(np.float32)])
    Qd = torch.from_numpy(Q).cuda()
    out = {}
    for m in (mode, 1):
        g = F.gpu_index(dict(cfg, score_mode=m), X, C, A, b)
        ids, sc, st, tr = g.search(Qd, cfg["k"], 2, stats=True, trace=True)
        out[m] = (ids.cpu().numpy(), sc.cpu().numpy(), tr["ucount"].cpu().numpy().sum(axis=1))
        g.free()
    assert out[mode][2].max() > 2048          # some tied query exceeds the histogram collection
    assert np.array_equal(out[mode][0], out[1][0])
    assert np.array_equal(out[mode][1].view(np.uint32), out[1][1].view(np.uint32))


@pytest.mark.parametrize("mode", [0, 3], ids=["tensor", "f16"])
def test_near_tied_kth_scores_at_d768_equal_simt(mode):
    """d = 768: 1,500 rows within 1e-6 of one unit vector (and 300 within
    1e-6 of its negation) among 4,000, with queries near that vector, so the
    k-th best score has hundreds of neighbours inside the guard band and
    scores of opposite sign cancel in the accumulation.  The band holds them
    all (it outgrows the re-score list, so the second kernel re-scores the
    whole band) and the exact re-score orders them: ids and scores equal the
    SIMT path's bit for bit."""
    import torch
    rng = np.random.default_rng(31)
    d, n = 768, 4000
    base = rng.standard_normal(d)
    base /= np.linalg.norm(base)
    X = rng.standard_normal((n, d))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X[:1500] = base + 1e-6 * rng.standard_normal((1500, d))
    X[1500:1800] = -base + 1e-6 * rng.standard_normal((300, d))
    X = X.astype(np.float32)
    C = np.concatenate([base[None], X[rng.choice(np.arange(1800, n), 5, replace=False)]]).astype(np.float32)
    cfg = dict(L=2, m=8, W=0.7, leaves=8, r0=100, B=1, k=16)
    A = rng.standard_normal((cfg["L"] * cfg["m"], d)).astype(np.float32)
    b = (rng.random(cfg["L"] * cfg["m"]) * cfg["W"]).astype(np.float32)
    Q = np.concatenate([base + 1e-3 * rng.standard_normal((12, d)),
                        rng.standard_normal((4, d))]).astype(np.float32)
    Qd = torch.from_numpy(Q).cuda()
    out, overflow = {}, 0
    for m in (mode, 1):
        g = F.gpu_index(dict(cfg, score_mode=m), X, C, A, b)
        for c in (1, 3):
            ids, sc, st = g.search(Qd, cfg["k"], c, stats=True)
            out[m, c] = (ids.cpu().numpy(), sc.cpu().numpy())
            overflow += st["select_overflow"] if m == mode else 0
        g.free()
    assert mode == 0 or overflow > 0          # the FP16 band outgrows the list
    for c in (1, 3):
        assert np.array_equal(out[mode, c][0], out[1, c][0]), c
        assert np.array_equal(out[mode, c][1].view(np.uint32), out[1, c][1].view(np.uint32)), c


@pytest.mark.parametrize("mode", [0, 3], ids=["tensor", "f16"])
def test_wide_rows_beyond_1024_equal_simt(mode):
    """d = 1,104 (more than 32 float4 per lane): the re-score takes its
    generic row loop instead of an unrolled instance; ids and scores equal
    the SIMT path's bit for bit, with no band overflow (so the re-score, not
    the band kernel, writes every result)."""
    import torch
    rng = np.random.default_rng(41)
    d, n = 1104, 3000
    centers = rng.standard_normal((12, d))
    X = centers[rng.integers(0, 12, n)] + 0.5 * rng.standard_normal((n, d))
    X = (X / np.linalg.norm(X, axis=1, keepdims=True)).astype(np.float32)
    C = X[rng.choice(n, 6, replace=False)].copy()
    cfg = dict(L=2, m=8, W=0.7, leaves=8, r0=3, B=1, k=10)
    A = rng.standard_normal((cfg["L"] * cfg["m"], d)).astype(np.float32)
    b = (rng.random(cfg["L"] * cfg["m"]) * cfg["W"]).astype(np.float32)
    Q = (centers[rng.integers(0, 12, 40)] + 0.5 * rng.standard_normal((40, d))).astype(np.float32)
    Qd = torch.from_numpy(Q).cuda()
    out, overflow = {}, 0
    for m in (mode, 1):
        g = F.gpu_index(dict(cfg, score_mode=m), X, C, A, b)
        for c in (1, 3):
            ids, sc, st = g.search(Qd, cfg["k"], c, stats=True)
            out[m, c] = (ids.cpu().numpy(), sc.cpu().numpy())
            overflow += st["select_overflow"]
        g.free()
    assert overflow == 0
    for c in (1, 3):
        assert np.array_equal(out[mode, c][0], out[1, c][0]), c
        assert np.array_equal(out[mode, c][1].view(np.uint32), out[1, c][1].view(np.uint32)), c
    assert np.all(out[mode, 3][0] >= 0)


@pytest.mark.parametrize("mode", [0, 3], ids=["tensor", "f16"])
def test_route_with_tied_centroids_equals_simt(mode):
    """Centroids in groups of equal rows (exactly tied routing scores) and of
    rows 1e-7 apart (within the tensor-core error guard): the tensor path
    scores exactly only the entries whose approximate order is open, and its
    route equals the SIMT path's (exact scores, ties to the lower index) for
    every query and every c."""
    import torch
    rng = np.random.default_rng(21)
    d, n = 64, 3000
    X = rng.standard_normal((n, d)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    base = X[rng.choice(n, 12, replace=False)]
    C = np.concatenate([base, base[:6], base[:6] + 1e-7 * rng.standard_normal((6, d))]).astype(np.float32)
    cfg = dict(L=2, m=8, W=0.7, leaves=8, r0=3, B=1, k=10)
    A = rng.standard_normal((cfg["L"] * cfg["m"], d)).astype(np.float32)
    b = (rng.random(cfg["L"] * cfg["m"]) * cfg["W"]).astype(np.float32)
    Q = np.concatenate([X[:60], base + 1e-3 * rng.standard_normal((12, d)).astype(np.float32),
                        rng.standard_normal((20, d)).astype(np.float32)]).astype(np.float32)
    Qd = torch.from_numpy(Q).cuda()
    routes = {}
    for m in (mode, 1):
        g = F.gpu_index(dict(cfg, score_mode=m), X, C, A, b)
        for c in (1, 3, 8, 17, 24):
            _, _, _, tr = g.search(Qd, cfg["k"], c, stats=True, trace=True)
            routes[m, c] = tr["route"].cpu().numpy()
        g.free()
    for c in (1, 3, 8, 17, 24):
        assert np.array_equal(routes[mode, c], routes[1, c]), c


def test_invalid_search_arguments(tiny):
    import torch
    from paper_2205_00970_b300 import lider
    g, Qd = tiny["gidx"], tiny["Qd"][:4]
    for k, c, code in [(0, 1, -1), (10, 0, -1), (10, 17, -1), (2000, 1, -4), (1000, 1, -4)]:
        with pytest.raises(lider.LiderError) as e:
            g.search(Qd, k, c)
        assert e.value.code == code
    # queries not on a 16-byte boundary are refused before any launch
    import ctypes
    ids = torch.empty((3, 10), dtype=torch.int64, device="cuda")
    sc = torch.empty((3, 10), dtype=torch.float32, device="cuda")
    rc = lider.raw_call("lider_search", g.handle, Qd.data_ptr() + 4, 3, 10, 1, ids.data_ptr(), sc.data_ptr(),
                        None, None)
    assert rc == -1 and "16-byte" in lider.last_error()


@pytest.mark.parametrize("mode,min_agree", [(2, 0.995), (4, 0.98)], ids=["bf16", "fp8"])
def test_served_forms(mode, min_agree):
    """Served forms (BF16 or FP8-e4m3 scoring + FP32 re-rank of a shortlist of
    rerank * k): every returned id is a candidate of its query, scores are the
    exact FP32 inner products, results are sorted, batch-invariant, and agree
    with the plain top-k on almost every rank."""
    import torch
    cfg, X, Q, C, A, b = F.workload("tiny")
    cfg["score_mode"] = mode
    cfg["rerank"] = 4
    g = F.gpu_index(cfg, X, C, A, b)
    Qd = torch.from_numpy(Q).cuda()
    ids, sc, st, tr = g.search(Qd, cfg["k"], cfg["c"], stats=True, trace=True)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    ref = O.search(F.oracle_index(cfg, X, C, A, b), Q, cfg["k"], cfg["c"], cfg["R"])
    bad, _ = F.check_trace(tr, ref)
    assert not bad, bad[:5]
    ref_idx = F.oracle_index(cfg, X, C, A, b)
    agree = 0
    for i in range(len(Q)):
        nv = int(np.sum(ids[i] >= 0))
        assert nv == int(np.sum(ref.ids[i] >= 0))
        exact = X[ids[i, :nv]].astype(np.float64) @ Q[i].astype(np.float64)
        assert np.all(np.abs(sc[i, :nv] - exact) <= F.SCORE_RTOL * np.abs(exact) + F.SCORE_ATOL)
        assert np.all(np.diff(sc[i, :nv]) <= 0)
        agree += len(set(ids[i, :nv].tolist()) & set(ref.ids[i, :nv].tolist()))
    total = int(np.sum(ref.ids >= 0))
    assert agree / total > min_agree, agree / total
    sub_ids, sub_sc = g.search(Qd[37:291].contiguous(), cfg["k"], cfg["c"])
    assert np.array_equal(sub_ids.cpu().numpy(), ids[37:291])


@pytest.mark.parametrize("k", [1, 10, 37])
@pytest.mark.parametrize("mode", [0, 3], ids=["tensor", "f16"])
def test_tensor_path_equals_simt_path_exactly(mode, k):
    """The tensor-core paths (3xTF32 or FP16 scores, a guard band around the
    k-th approximate score, exact FP32 re-score) return exactly the SIMT
    path's results: the exact FP32 top-k of every query's candidate union,
    same ids, same scores bit for bit, ties by lower id."""
    import torch
    cfg, X, Q, C, A, b = F.workload("tiny")
    Qd = torch.from_numpy(Q).cuda()
    out = {}
    for m in (mode, 1):
        g = F.gpu_index(dict(cfg, score_mode=m), X, C, A, b)
        ids, sc, st = g.search(Qd, k, cfg["c"], stats=True)
        out[m] = (ids.cpu().numpy(), sc.cpu().numpy(), st)
        g.free()
    assert out[mode][2]["select_overflow"] == 0
    assert np.array_equal(out[mode][0], out[1][0])
    assert np.array_equal(out[mode][1].view(np.uint32), out[1][1].view(np.uint32))


def test_passes_equal_one_pass(tiny):
    """A batch searched in passes of probe_batch queries (one lider_search
    call) returns what one pass returns, trace arrays included, and the
    counters add up over the passes."""
    cfg = tiny["cfg"]
    g = tiny["gidx"]
    ids1, sc1, st1, tr1 = g.search(tiny["Qd"], cfg["k"], cfg["c"], stats=True, trace=True)
    before = g.tuning()
    try:
        g.set_tuning(probe_batch=300)
        ids4, sc4, st4, tr4 = g.search(tiny["Qd"], cfg["k"], cfg["c"], stats=True, trace=True)
    finally:
        g.set_tuning(**before)
    assert st1["passes"] == 1 and st4["passes"] == 4
    assert (ids1 == ids4).all() and (sc1 == sc4).all()
    for name in tr1:
        assert (tr1[name] == tr4[name]).all(), name
    for key in ("candidates", "pairs", "tc_tiles", "qkey_boundary", "locate_fallback"):
        if key != "tc_tiles":
            assert st1[key] == st4[key], key
