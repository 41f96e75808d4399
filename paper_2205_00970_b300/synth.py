"""Seeded synthetic inputs for LIDER search: corpus, queries, projections.

This module is the only code shared by the CUDA path's tests/bench and the
FP64 oracle. It holds none of the method's arithmetic: it draws Gaussian-mixture
embeddings (the stand-in for the paper's 768-d passage embeddings, Sec. 7.1,
which are L2-normalised so that cosine equals inner product) and the random
LSH projections the method would otherwise draw itself (Sec. 4.1: the hash
family is random; here the draws are inputs).

Every stream is counter-based (numpy Philox, 128-bit key = (seed, stream id),
256-bit counter) and row-addressable in chunks of ``CHUNK`` rows, so any row
range can be regenerated on any machine without materialising the whole
corpus, and generation can run on several threads.

Recipe (mixture):
  * component centers mu_c ~ N(0, I_d)                (FP64)
  * component of row i: uniform over n_comp, or Zipf(s) weights w_c ~ 1/c^s
  * x_i = mu_{comp(i)} + sigma * N(0, I_d), then x_i /= ||x_i||  (FP64)
  * rounded to FP32
Queries use the same centers with a different stream id.
Projections: a ~ N(0, I_d) per hash (FP32), offsets b ~ U[0, W) (FP32).
"""
from __future__ import annotations

import concurrent.futures as _cf
import os

import numpy as np

CHUNK = 4096

# stream ids (second word of the Philox key)
STREAM_CENTERS = 1
STREAM_CORPUS = 2
STREAM_QUERIES = 3
STREAM_PROJ = 4
STREAM_COMPONENT = 5


def _rng(seed: int, stream: int, chunk: int = 0) -> np.random.Generator:
    key = np.array([np.uint64(seed), np.uint64(stream)], dtype=np.uint64)
    counter = np.array([0, chunk, 0, 0], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key, counter=counter))


def mixture_centers(seed: int, n_comp: int, d: int) -> np.ndarray:
    """Component centers, FP64 (n_comp, d)."""
    return _rng(seed, STREAM_CENTERS).standard_normal((n_comp, d))


def _component_weights(n_comp: int, zipf_s: float | None) -> np.ndarray | None:
    if zipf_s is None:
        return None
    w = 1.0 / np.arange(1, n_comp + 1, dtype=np.float64) ** zipf_s
    return np.cumsum(w / w.sum())


def _chunk_rows(seed, stream, chunk, rows, centers, sigma, cdf):
    rng = _rng(seed, stream, chunk)
    n_comp, d = centers.shape
    if cdf is None:
        comp = rng.integers(0, n_comp, size=rows)
    else:
        comp = np.minimum(np.searchsorted(cdf, rng.random(rows), side="right"), n_comp - 1)
    noise = rng.standard_normal((rows, d), dtype=np.float32)
    x = centers[comp] + sigma * noise.astype(np.float64)
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x.astype(np.float32), comp


def mixture_rows(seed: int, stream: int, start: int, stop: int, d: int, n_comp: int,
                 sigma: float = 0.3, zipf_s: float | None = None,
                 threads: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    """Rows [start, stop) of a seeded mixture stream, FP32 (stop-start, d)."""
    centers = mixture_centers(seed, n_comp, d)
    cdf = _component_weights(n_comp, zipf_s)
    n = stop - start
    if out is None:
        out = np.empty((n, d), dtype=np.float32)
    c0, c1 = start // CHUNK, (stop + CHUNK - 1) // CHUNK

    def work(c):
        lo, hi = c * CHUNK, (c + 1) * CHUNK
        x, _ = _chunk_rows(seed, stream, c, CHUNK, centers, sigma, cdf)
        a, b = max(lo, start), min(hi, stop)
        out[a - start:b - start] = x[a - lo:b - lo]

    threads = threads or min(16, os.cpu_count() or 1)
    if c1 - c0 <= 1 or threads == 1:
        for c in range(c0, c1):
            work(c)
    else:
        with _cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, range(c0, c1)))
    return out


def corpus(seed: int, n: int, d: int, n_comp: int, sigma: float = 0.3,
           zipf_s: float | None = None, start: int = 0, stop: int | None = None,
           threads: int | None = None) -> np.ndarray:
    stop = n if stop is None else stop
    return mixture_rows(seed, STREAM_CORPUS, start, stop, d, n_comp, sigma, zipf_s, threads)


def queries(seed: int, nq: int, d: int, n_comp: int, sigma: float = 0.3,
            zipf_s: float | None = None, threads: int | None = None) -> np.ndarray:
    return mixture_rows(seed, STREAM_QUERIES, 0, nq, d, n_comp, sigma, zipf_s, threads)


def projections(seed: int, L: int, m: int, d: int, W: float):
    """LSH draws: A (L*m, d) FP32 with N(0,1) entries, b (L*m,) FP32 in [0, W).

    Row l*m + j of A (and entry l*m + j of b) is hash j of hashkey array l.
    """
    rng = _rng(seed, STREAM_PROJ)
    A = rng.standard_normal((L * m, d), dtype=np.float32)
    b = (rng.random(L * m) * W).astype(np.float32)
    b = np.minimum(b, np.nextafter(np.float32(W), np.float32(0)))
    return A, b
