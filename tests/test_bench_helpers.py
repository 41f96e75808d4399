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
