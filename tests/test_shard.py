"""By-cluster sharding (Sec. 3.3.2: probed clusters are searched
independently; Sec. 6.2: their top-k lists are merged): the host logic on
two gloo ranks on CPU, and on one GPU two shards searched in turn.

On CPU the per-rank search is the FP64 oracle's over the rank's rows (the
stand-in for the GPU search there); the merged result must equal the
oracle's search over the whole corpus."""
import os
import socket

import numpy as np
import pytest

from paper_2205_00970_b300 import shard


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_owner_of_clusters_balances_rows():
    sizes = np.array([50, 10, 10, 40, 0, 30, 20])
    owner = shard.owner_of_clusters(sizes, 3)
    load = np.bincount(owner, weights=sizes, minlength=3)
    assert load.sum() == sizes.sum() and load.max() - load.min() <= sizes.max()
    # largest first, to the least-loaded rank, ties to the lower rank
    assert owner[0] == 0 and owner[3] == 1 and owner[5] == 2
    assert np.all(shard.owner_of_clusters(sizes, 1) == 0)


def test_merge_topk_equals_sorting_the_union():
    rng = np.random.default_rng(3)
    parts_i, parts_s = [], []
    for r in range(3):
        ids = rng.choice(1000, (5, 6), replace=False) + 1000 * r
        sc = rng.integers(0, 4, (5, 6)).astype(np.float32)       # many exact ties
        ids[:, -1] = -1
        sc[:, -1] = -np.inf
        parts_i.append(ids)
        parts_s.append(sc)
    got_i, got_s = shard.merge_topk(parts_i, parts_s, 7)
    for q in range(5):
        pool = [(-float(s), int(i)) for p_i, p_s in zip(parts_i, parts_s) for i, s in zip(p_i[q], p_s[q]) if i >= 0]
        best = sorted(pool)[:7]
        assert got_i[q].tolist() == [i for _, i in best]
        assert got_s[q].tolist() == [-s for s, _ in best]
    # fewer than k candidates: padding
    gi, gs = shard.merge_topk([np.array([[3, -1]])], [np.array([[1.0, -np.inf]], np.float32)], 3)
    assert gi.tolist() == [[3, -1, -1]] and np.isneginf(gs[0, 1:]).all()


def _problem():
    from oracle import lider_oracle as O
    rng = np.random.default_rng(21)
    X = rng.standard_normal((900, 16)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    Q = rng.standard_normal((14, 16)).astype(np.float32)
    C = X[rng.choice(900, 6, replace=False)]
    A = rng.standard_normal((3 * 8, 16)).astype(np.float32)
    b = rng.random(3 * 8).astype(np.float32)
    full = O.build_index(X, C, A, b, 3, 8, 1.0, 4)
    return O, X, Q, C, A, b, full


def _rank(rank: int, world: int, port: int, out_dir: str):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        O, X, Q, C, A, b, full = _problem()
        owner = shard.owner_of_clusters(np.bincount(full.asg, minlength=len(C)), world)
        rows = shard.rows_of_rank(full.asg, owner, rank)
        part = O.build_index(X[rows], C, A, b, 3, 8, 1.0, 4)
        r = O.search(part, Q, 5, 3, 10)
        ids = np.where(r.ids >= 0, rows[np.maximum(r.ids, 0)], -1)
        got_i, got_s = shard.all_gather_merge(torch.from_numpy(ids), torch.from_numpy(r.scores), 5)
        np.save(os.path.join(out_dir, f"ids{rank}.npy"), got_i)
        np.save(os.path.join(out_dir, f"sc{rank}.npy"), got_s)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_merge_equals_one_index(tmp_path):
    import torch.multiprocessing as mp
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    O, X, Q, C, A, b, full = _problem()
    ref = O.search(full, Q, 5, 3, 10)
    for r in range(2):
        np.testing.assert_array_equal(np.load(tmp_path / f"ids{r}.npy"), ref.ids)
        np.testing.assert_array_equal(np.load(tmp_path / f"sc{r}.npy"), ref.scores)


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [3, 1])
def test_two_shards_on_one_gpu_equal_one_index(mode):
    """Tiny workload: the index over the whole corpus against two shards
    (each a lider.Index over the rows of its clusters, the shared centroids
    and draws) searched in turn and merged; equal bit for bit."""
    import torch
    from tests.lider_fixtures import workload
    from paper_2205_00970_b300 import lider
    cfg, X, Q, C, A, b = workload("tiny")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    kw = dict(L=cfg["L"], m=cfg["m"], W=cfg["W"], rmi_leaves=cfg["leaves"], r0=cfg["r0"], B=cfg["B"],
              score_mode=mode)
    full = lider.Index(t(X), t(C), t(A), t(b), **kw)
    Qd = t(Q)
    ref_i, ref_s = full.search(Qd, cfg["k"], cfg["c"])
    asg = full.assignment()
    owner = shard.owner_of_clusters(np.bincount(asg, minlength=len(C)), 2)
    parts_i, parts_s = [], []
    for r in range(2):
        rows = shard.rows_of_rank(asg, owner, r)
        sh = shard.ShardedIndex(t(X[rows]), rows, t(C), t(A), t(b), **kw)
        i, s = sh.local_search(Qd, cfg["k"], cfg["c"])
        parts_i.append(i.cpu().numpy())
        parts_s.append(s.cpu().numpy())
        sh.free()
    got_i, got_s = shard.merge_topk(parts_i, parts_s, cfg["k"])
    np.testing.assert_array_equal(got_i, ref_i.cpu().numpy())
    np.testing.assert_array_equal(got_s, ref_s.cpu().numpy())
    full.free()
