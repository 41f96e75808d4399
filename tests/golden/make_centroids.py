"""Write the k-means centroids used as index input for the named workloads.

The centroids are an input of the index (the clustering of Sec. 3.2 is plain
k-means).  They are computed here by the FP64 oracle's Lloyd iterations
(``oracle.lider_oracle.kmeans``) on the first ``kmeans_sample`` corpus rows,
seeded by ``synth.init_rows``, and stored as FP32 so that the CUDA path and the
oracle build from the same clustering.

usage: python tests/golden/make_centroids.py tiny mid batched precision

(batched and precision share the generator, the seed and kmeans_sample, so
their sample rows and centroids are identical.)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lider_oracle as O  # noqa: E402
from paper_2205_00970_b300 import configs, synth  # noqa: E402


def centroids_for(name: str) -> np.ndarray:
    cfg = configs.get(name)
    ns = min(cfg["kmeans_sample"], cfg["n"])
    X = synth.corpus(cfg["seed"], cfg["n"], cfg["d"], cfg["n_comp"], cfg["sigma"],
                     cfg["zipf_s"], start=0, stop=ns)
    init = X[synth.init_rows(cfg["seed"], ns, cfg["n_clusters"])]
    return O.kmeans(X, init, cfg["kmeans_iters"]).astype(np.float32)


if __name__ == "__main__":
    for name in sys.argv[1:]:
        C = centroids_for(name)
        path = os.path.join(HERE, f"centroids_{name}.npy")
        np.save(path, C)
        print(name, C.shape, path)
