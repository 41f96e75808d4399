"""k-means inside lider_build (Sec. 3.2; Sec. 3.3.2 "LIDER is built as
follows"; Table 5 stage 1) against the FP64 oracle's Lloyd iterations.

Both sides start from the Forgy rows that SplitMix64 + Floyd's sampling draw
from the workload's seed and keep FP32 centroids (readings R24, R25).  The
oracle's centroids are the fixtures in tests/golden (written by
make_centroids.py, which calls only the oracle).  Independently of the
oracle's iterations, every exported assignment must be the FP64 argmax of
x.mu - |mu|^2/2 over the exported centroids (near-ties within 1e-9 relative
counted, not failed)."""
import numpy as np
import pytest

from oracle import lider_oracle as O
from paper_2205_00970_b300 import configs, synth

from tests.lider_fixtures import GOLDEN, workload

pytestmark = pytest.mark.gpu

# Centroid values are ~0.05-0.5; a single row moved between clusters shifts a
# centroid by ~1e-3, FP64 rounding-order differences shift none beyond 1 ulp.
CENTROID_ATOL = 1e-6


def _build(X, cfg, A=None, b=None, n=None, **kw):
    import torch
    from paper_2205_00970_b300 import lider
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    X = X if n is None else X[:n]
    return lider.Index(t(X), None, None if A is None else t(A), None if b is None else t(b),
                       L=cfg["L"], m=cfg["m"], W=cfg["W"], rmi_leaves=cfg["leaves"], r0=cfg["r0"], B=cfg["B"],
                       score_mode=kw.pop("score_mode", lider.SCORE_F16), n_clusters=cfg["n_clusters"],
                       kmeans_iters=kw.pop("kmeans_iters", cfg["kmeans_iters"]),
                       kmeans_sample=kw.pop("kmeans_sample", cfg["kmeans_sample"]), seed=cfg["seed"], **kw)


def _argmax_violations(X, C, asg, rows):
    """Rows whose assignment is not the FP64 argmax (ties to the lower index),
    and how many of those are near-ties within 1e-9 relative."""
    C64 = C.astype(np.float64)
    hn = 0.5 * np.sum(C64 * C64, axis=1)
    bad = near = 0
    for s in range(0, len(rows), 8192):
        r = rows[s:s + 8192]
        S = X[r].astype(np.float64) @ C64.T - hn
        best = np.argmax(S, axis=1)
        wrong = best != asg[r]
        if np.any(wrong):
            top = S[np.arange(len(r)), best]
            got = S[np.arange(len(r)), asg[r]]
            tie = (top - got) <= 1e-9 * np.maximum(1.0, np.abs(top))
            near += int(np.count_nonzero(wrong & tie))
            bad += int(np.count_nonzero(wrong & ~tie))
    return bad, near


@pytest.fixture(scope="module")
def tiny():
    return workload("tiny")


def test_tiny_kmeans_equals_oracle_and_assignment_is_argmax(tiny):
    cfg, X, Q, C_ref, A, b = tiny
    idx = _build(X, cfg, A, b)
    info = idx.build_info()
    assert info["clustered"] and not info["projections_drawn"]
    assert info["train_rows"] == min(cfg["kmeans_sample"], cfg["n"]) and info["kmeans_iters"] == cfg["kmeans_iters"]
    C = idx.centroids()
    np.testing.assert_allclose(C, C_ref, rtol=0, atol=CENTROID_ATOL)
    asg = idx.assignment()
    bad, near = _argmax_violations(X, C, asg, np.arange(cfg["n"]))
    assert bad == 0, (bad, near)
    # the partition is the assignment: cluster sizes agree
    np.testing.assert_array_equal(np.diff(idx.cluster_offsets()), np.bincount(asg, minlength=cfg["n_clusters"]))
    idx.free()


def test_tiny_zero_iterations_keeps_the_forgy_rows(tiny):
    """With no Lloyd iteration the centroids are the Forgy rows: the library's
    generator draws the same rows as the oracle's forgy_rows."""
    cfg, X, Q, C_ref, A, b = tiny
    idx = _build(X, cfg, A, b, kmeans_iters=0)
    rows = O.forgy_rows(cfg["seed"], min(cfg["kmeans_sample"], cfg["n"]), cfg["n_clusters"])
    np.testing.assert_array_equal(idx.centroids(), X[rows])
    idx.free()


def test_tiny_clustered_index_searches_like_the_fixture_index(tiny):
    """The index whose clustering ran on the device returns the same results as
    the one built from the oracle's centroids (the centroids agree)."""
    from tests.lider_fixtures import gpu_index
    import torch
    cfg, X, Q, C_ref, A, b = tiny
    cfg = dict(cfg, score_mode=3)
    a = _build(X, cfg, A, b)
    ref = gpu_index(cfg, X, C_ref, A, b)
    Qd = torch.from_numpy(Q).cuda()
    ia, sa = a.search(Qd, cfg["k"], cfg["c"])
    ir, sr = ref.search(Qd, cfg["k"], cfg["c"])
    assert torch.equal(ia, ir) and torch.equal(sa, sr)
    a.free()
    ref.free()


def test_seeded_projections_are_gaussian_and_reproducible(tiny):
    """Without A and b the build draws them from the seed: N(0,1) entries and
    offsets in [0, W); the same seed gives the same draws, and an index built
    from the exported draws searches identically."""
    import torch
    cfg, X, Q, C_ref, A, b = tiny
    cfg = dict(cfg, score_mode=3)
    i1 = _build(X, cfg)
    i2 = _build(X, cfg)
    assert i1.build_info()["projections_drawn"]
    A1, b1 = i1.projections()
    A2, b2 = i2.projections()
    np.testing.assert_array_equal(A1, A2)
    np.testing.assert_array_equal(b1, b2)
    v = A1.astype(np.float64).ravel()
    n = v.size
    assert abs(v.mean()) < 5 / np.sqrt(n)
    assert abs(v.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(np.abs(v) < 1.0) - 0.682689) < 5 * np.sqrt(0.2166 / n)
    assert np.all(b1 >= 0) and np.all(b1 < cfg["W"])
    i3 = _build(X, cfg, A1, b1)
    Qd = torch.from_numpy(Q).cuda()
    r1 = i1.search(Qd, cfg["k"], cfg["c"])
    r3 = i3.search(Qd, cfg["k"], cfg["c"])
    assert torch.equal(r1[0], r3[0]) and torch.equal(r1[1], r3[1])
    for i in (i1, i2, i3):
        i.free()


def test_mid_kmeans_equals_oracle():
    """Mid: 65,536 training rows, 256 clusters, 10 iterations; every centroid
    against the oracle's, and the assignment of 40,000 sampled rows of the
    1,000,000 against the FP64 argmax."""
    cfg = configs.get("mid")
    ns = min(cfg["kmeans_sample"], cfg["n"])
    X = synth.corpus(cfg["seed"], cfg["n"], cfg["d"], cfg["n_comp"], cfg["sigma"], cfg["zipf_s"])
    A, b = synth.projections(cfg["seed"], cfg["L"], cfg["m"], cfg["d"], cfg["W"])
    C_ref = np.load(f"{GOLDEN}/centroids_mid.npy")
    idx = _build(X, cfg, A, b)
    info = idx.build_info()
    assert info["train_rows"] == ns
    C = idx.centroids()
    np.testing.assert_allclose(C, C_ref, rtol=0, atol=CENTROID_ATOL)
    asg = idx.assignment()
    rows = np.sort(np.random.default_rng(1).choice(cfg["n"], 40_000, replace=False))
    bad, near = _argmax_violations(X, C, asg, rows)
    assert bad == 0, (bad, near)
    idx.free()


def test_batched_kmeans_equals_oracle():
    """Batched: the clustering learns from the first 131,072 rows of the
    8.8M Zipf corpus (1,024 clusters), so an index over those rows alone runs
    the same k-means; all 1,024 centroids against the oracle's, and the
    assignment of every training row against the FP64 argmax."""
    cfg = configs.get("batched")
    ns = min(cfg["kmeans_sample"], cfg["n"])
    X = synth.corpus(cfg["seed"], cfg["n"], cfg["d"], cfg["n_comp"], cfg["sigma"], cfg["zipf_s"], stop=ns)
    A, b = synth.projections(cfg["seed"], cfg["L"], cfg["m"], cfg["d"], cfg["W"])
    C_ref = np.load(f"{GOLDEN}/centroids_batched.npy")
    idx = _build(X, cfg, A, b, kmeans_sample=0)
    C = idx.centroids()
    np.testing.assert_allclose(C, C_ref, rtol=0, atol=CENTROID_ATOL)
    bad, near = _argmax_violations(X, C, idx.assignment(), np.arange(ns))
    assert bad == 0, (bad, near)
    assert idx.build_info()["empty_clusters"] == int(np.sum(np.diff(idx.cluster_offsets()) == 0))
    idx.free()
