"""By-cluster sharding of one LIDER index over several GPUs.

LIDER searches the clusters a query probes independently of one another and
merges their top-k lists (Sec. 3.3.2; Sec. 6.2 keeps a heap over the
per-cluster lists), so the clusters can live on different GPUs:

  * every rank holds the same centroids and LSH draws, and the corpus rows of
    the clusters it owns (owner_of_clusters balances rows across ranks);
  * a rank's index routes every query over all centroids, so a probed cluster
    that another rank owns is simply empty in it, and it returns the exact
    top-k of its own candidates;
  * one exchange step: an all-gather of every rank's nq x k ids and scores,
    then each query keeps its k best by (score descending, id ascending).

Because a cluster's core model depends only on that cluster's rows (kept in
ascending id order), the merged result equals what one index over the whole
corpus returns.  This module is host logic (NumPy and torch.distributed); the
search itself runs in the CUDA library through lider.Index.
"""
from __future__ import annotations

import numpy as np


def owner_of_clusters(sizes: np.ndarray, world: int) -> np.ndarray:
    """Rank owning each cluster: clusters by size descending (ties: lower
    index first) each go to the rank holding the fewest rows so far (ties:
    lower rank).  Returns an int array of len(sizes)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    owner = np.zeros(len(sizes), dtype=np.int64)
    load = np.zeros(world, dtype=np.int64)
    for j in sorted(range(len(sizes)), key=lambda j: (-sizes[j], j)):
        r = int(np.argmin(load))
        owner[j] = r
        load[r] += sizes[j]
    return owner


def rows_of_rank(assignment: np.ndarray, owner: np.ndarray, rank: int) -> np.ndarray:
    """Global row ids, ascending, of the clusters `rank` owns."""
    return np.nonzero(owner[np.asarray(assignment)] == rank)[0].astype(np.int64)


def merge_topk(ids_parts, scores_parts, k: int):
    """Per query, the k best of the concatenated lists by score descending,
    then id ascending; -1 ids (padding) are dropped, and missing places are
    padded with id -1 and score -inf.  Parts are (nq, k_i) arrays; the scores
    keep their type."""
    ids = np.concatenate([np.asarray(p, dtype=np.int64) for p in ids_parts], axis=1)
    sc = np.concatenate([np.asarray(p) for p in scores_parts], axis=1)
    nq = ids.shape[0]
    out_ids = np.full((nq, k), -1, dtype=np.int64)
    out_sc = np.full((nq, k), -np.inf, dtype=sc.dtype)
    for i in range(nq):
        keep = ids[i] >= 0
        ii, ss = ids[i][keep], sc[i][keep]
        order = np.lexsort((ii, -ss.astype(np.float64)))[:k]
        out_ids[i, :len(order)] = ii[order]
        out_sc[i, :len(order)] = ss[order]
    return out_ids, out_sc


def all_gather_merge(ids, scores, k: int, group=None):
    """The exchange step: every rank's (nq, k) ids and scores (torch tensors on
    the process group's device) are gathered and merged (merge_topk); every
    rank gets the same (ids, scores) as NumPy arrays."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    got_i = [ids.new_empty(ids.shape) for _ in range(world)]
    got_s = [scores.new_empty(scores.shape) for _ in range(world)]
    dist.all_gather(got_i, ids.contiguous(), group=group)
    dist.all_gather(got_s, scores.contiguous(), group=group)
    return merge_topk([t.cpu().numpy() for t in got_i], [t.cpu().numpy() for t in got_s], k)


class ShardedIndex:
    """This rank's part of a by-cluster sharded index: a lider.Index over the
    rows of the clusters the rank owns, built from the shared centroids and
    LSH draws.  search() returns global ids merged over all ranks."""

    def __init__(self, corpus_rows, global_ids: np.ndarray, centroids, A, b, **index_params):
        from . import lider
        self.global_ids = np.asarray(global_ids, dtype=np.int64)
        if len(self.global_ids) and np.any(np.diff(self.global_ids) <= 0):
            raise ValueError("global_ids must be strictly ascending (a cluster's rows keep their id order)")
        self.index = lider.Index(corpus_rows, centroids, A, b, **index_params) if len(self.global_ids) else None

    def local_search(self, Q, k: int, c: int):
        """This rank's top-k over its own clusters, as global ids: (ids, scores)
        torch tensors on the queries' device."""
        import torch
        if self.index is None:
            nq = Q.shape[0]
            return (torch.full((nq, k), -1, dtype=torch.int64, device=Q.device),
                    torch.full((nq, k), float("-inf"), dtype=torch.float32, device=Q.device))
        ids, sc = self.index.search(Q, k, c)
        gid = torch.from_numpy(self.global_ids).to(ids.device)
        mapped = torch.where(ids >= 0, gid[ids.clamp(min=0)], ids)
        return mapped, sc

    def search(self, Q, k: int, c: int, group=None):
        ids, sc = self.local_search(Q, k, c)
        return all_gather_merge(ids, sc, k, group)

    def free(self):
        if self.index is not None:
            self.index.free()
            self.index = None
