"""The benchmark's measurement helpers on CPU: the FP64 brute-force ground
truth behind its recall figures equals the oracle's exact kNN (ties to the
lower id), and recall@10 counts set overlap."""
import numpy as np


def test_fp64_knn_equals_oracle_exact_knn():
    import bench
    from oracle import lider_oracle as O
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3000, 24)).astype(np.float32)
    X[17] = X[4]                                   # an exact tie across chunks
    Q = np.concatenate([rng.standard_normal((9, 24)), X[4:5]]).astype(np.float32)
    got = bench.fp64_knn(X, Q, 12, chunk=700, device="cpu")
    np.testing.assert_array_equal(got, O.exact_knn(X, Q, 12)[0])


def test_recall10_counts_overlap():
    import bench
    truth = np.arange(20).reshape(2, 10)
    found = truth.copy()
    found[0, :3] = [100, 101, 102]
    found[1] = found[1][::-1]
    assert bench.recall10(found, truth) == (7 / 10 + 10 / 10) / 2


def test_oracle_pool_search_equals_serial_search():
    """The CPU baseline's fork pool returns what one oracle search over the
    same queries returns, in query order."""
    import bench
    from oracle import lider_oracle as O
    rng = np.random.default_rng(6)
    X = rng.standard_normal((600, 16)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    Q = rng.standard_normal((11, 16)).astype(np.float32)
    A = rng.standard_normal((3 * 8, 16)).astype(np.float32)
    b = rng.random(3 * 8).astype(np.float32)
    C = X[:5]
    idx = O.build_index(X, C, A, b, 3, 8, 1.0, 4)
    cfg = {"k": 7, "c": 2, "R": 14}
    got, sec = bench.oracle_pool_search(idx, Q, cfg, cores=2, batch=3, budget_s=None)
    np.testing.assert_array_equal(got, O.search(idx, Q, 7, 2, 14).ids)
    assert sec > 0


def test_score_roofline_counts_the_methods_work():
    """frac = 2 x candidates x d / phase time / peak; the executed tiles and
    the unique bytes are reported beside it."""
    import bench
    hbm, bf16, _, _ = bench.measured_peaks()
    stats = {"candidates": 1_000_000, "tc_tiles": 100}
    route = np.array([[0, 1], [1, 2]], dtype=np.int32)
    cl_off = np.array([0, 100, 300, 364, 500])
    r = bench.score_roofline("f16", stats, route, cl_off, 768, 1e-3, {})
    assert r["bound"] == "tensor" and r["peak"] == bf16
    assert abs(r["achieved"] - 2 * 1e6 * 768 / 1e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / bf16) < 1e-12
    assert r["executed"]["flop_per_launch"] == 100 * 128 * 256 * 768 * 2
    # probed clusters 0, 1, 2 (364 rows), 4 gathered queries, bitmap words 4 + 7 + 7 + 2
    assert r["unique_bytes"]["bytes_per_launch"] == (364 * 768 * 2 + 4 * 768 * 2 + (4 + 7 + 7 + 2) * 4)


def test_launches_per_pass_follows_the_grouping_path():
    """A pass small enough for the one-block grouping launches three (SIMT:
    two) kernels fewer than one that takes the multi-kernel grouping."""
    import bench
    assert bench.launches_per_pass("f16", 10_000, 8, 256) == 17          # mid: 80,000 pairs
    assert bench.launches_per_pass("f16", 12_500, 16, 1_024) == 20       # batched pass: 200,000 pairs
    assert bench.launches_per_pass("simt", 10_000, 8, 256) == 8
    assert bench.launches_per_pass("bf16", 16_384, 8, 256) == 16         # exactly 131,072 pairs
    assert bench.launches_per_pass("tensor", 100, 8, 5_000) == 20        # too many clusters
