"""Named synthetic workloads for LIDER batched search.

Each entry fixes the corpus/query generator recipe (see ``synth``) and the
index/search parameters in the paper's vocabulary (Table 1, Sec. 6):
``n_clusters`` = c (total k-means clusters), ``c`` = c_0 (clusters probed per
query), ``L`` = H (hashkey arrays per core model), ``m`` = M (hashes per
hashkey), ``r0`` with R = r0 * k (expansion range per array, Sec. 6.1),
``leaves`` = RMI width (number of second-stage linear models, Sec. 5.2),
``W`` = p-stable bucket width.
"""

CONFIGS = {
    # Plain method, tiny: every query fits the oracle in seconds.
    "tiny": dict(n=10_000, d=128, n_comp=64, sigma=0.3, zipf_s=None, nq=1_000,
                 n_clusters=16, c=4, L=4, m=8, W=1.0, leaves=16, k=10, r0=2,
                 B=1, kmeans_iters=10, kmeans_sample=10_000, seed=0),
    # Plain method, mid: 1M x 768, 256 clusters, c=8, L=8, m=16, k=100.
    "mid": dict(n=1_000_000, d=768, n_comp=1_024, sigma=0.3, zipf_s=None, nq=10_000,
                n_clusters=256, c=8, L=8, m=16, W=1.0, leaves=1_024, k=100, r0=3,
                B=1, kmeans_iters=10, kmeans_sample=65_536, seed=0),
    # Batched uneven: 8.8M x 768 with Zipf(1.1) component sizes (so uneven
    # clusters), 1,024 clusters, c=16, 50,000 queries, k=100.
    "batched": dict(n=8_800_000, d=768, n_comp=1_024, sigma=0.3, zipf_s=1.1, nq=50_000,
                    n_clusters=1_024, c=16, L=8, m=16, W=1.0, leaves=1_024, k=100, r0=3,
                    B=1, kmeans_iters=10, kmeans_sample=131_072, seed=0),
    # Precision: 21M x 768, same generator, 100,000 queries; the served forms
    # keep a shortlist of 4,000 (rerank 40 at k=100) re-ranked in FP32.
    "precision": dict(n=21_000_000, d=768, n_comp=1_024, sigma=0.3, zipf_s=1.1, nq=100_000,
                      n_clusters=1_024, c=16, L=8, m=16, W=1.0, leaves=1_024, k=100, r0=3,
                      B=1, kmeans_iters=10, kmeans_sample=131_072, seed=0, rerank=40),
}


def get(name: str) -> dict:
    cfg = dict(CONFIGS[name])
    cfg["name"] = name
    cfg["R"] = cfg["r0"] * cfg["k"]
    return cfg
