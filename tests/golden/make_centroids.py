"""Write the k-means centroids the oracle computes for the named workloads.

The clustering of Sec. 3.2 is plain k-means.  Here the FP64 oracle runs it
(``oracle.lider_oracle.kmeans``: Lloyd iterations, FP32-stored centroids) on
the first ``kmeans_sample`` corpus rows, from the Forgy rows that
``oracle.lider_oracle.forgy_rows`` draws from the workload's seed.  The CUDA
build runs the same clustering itself from the same seed; the tests compare its
centroids with these files, and the search parity tests give these centroids
to both sides as a shared input.

usage: python tests/golden/make_centroids.py tiny mid batched precision

(batched and precision share the generator, the seed and kmeans_sample, so
their sample rows and centroids are identical; they are computed once.)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lider_oracle as O  # noqa: E402
from paper_2205_00970_b300 import configs, synth  # noqa: E402


def clustering_key(cfg: dict) -> tuple:
    return tuple(cfg[k] for k in ("seed", "n", "d", "n_comp", "sigma", "zipf_s", "kmeans_sample",
                                  "n_clusters", "kmeans_iters"))


def centroids_for(name: str) -> np.ndarray:
    cfg = configs.get(name)
    ns = min(cfg["kmeans_sample"], cfg["n"])
    X = synth.corpus(cfg["seed"], cfg["n"], cfg["d"], cfg["n_comp"], cfg["sigma"],
                     cfg["zipf_s"], start=0, stop=ns)
    init = X[O.forgy_rows(cfg["seed"], ns, cfg["n_clusters"])]
    return O.kmeans(X, init, cfg["kmeans_iters"])


if __name__ == "__main__":
    done = {}
    for name in sys.argv[1:]:
        key = clustering_key(configs.get(name))
        if key not in done:
            done[key] = centroids_for(name)
        C = done[key]
        path = os.path.join(HERE, f"centroids_{name}.npy")
        np.save(path, C)
        print(name, C.shape, C.dtype, path, flush=True)
