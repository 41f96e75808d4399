"""Continuous-batching server: the scheduler's host logic against a fake
executor (C++, no CUDA), the C ABI's argument checks, and (GPU) each
request's results under a mixed Poisson load equal to the same request
searched alone."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_scheduler_core_with_fake_executor(tmp_path):
    exe = tmp_path / "server_core_check"
    src = os.path.join(ROOT, "tests", "server_core_check.cpp")
    subprocess.run(["g++", "-std=c++17", "-O1", "-pthread", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2205_00970_b300", "csrc"), src, "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "all checks passed" in r.stdout


def test_server_abi_validates_without_gpu():
    from paper_2205_00970_b300 import lider
    p = lider.ServerParams(4, 3, 1024, 100, 1 << 30, 100.0)
    out = ctypes.c_void_p()
    assert lider.raw_call("lider_server_create", None, ctypes.byref(p), ctypes.byref(out)) == -1
    assert "NULL" in lider.last_error()
    assert lider.raw_call("lider_server_create", None, ctypes.byref(p), None) == -1
    t = ctypes.c_int64()
    assert lider.raw_call("lider_server_submit", None, None, 0, 10, None, None, ctypes.byref(t)) == -1
    assert lider.raw_call("lider_server_wait", None, 0, 0.0) == -1
    lider.raw_call("lider_server_destroy", None)          # NULL accepted


def _poisson(Q, srv, rate, seconds, ks, max_req, seed):
    from paper_2205_00970_b300.serving import poisson_schedule, run_load
    sch = poisson_schedule(rate, seconds, ks=ks, max_req=max_req, n_queries=Q.shape[0], seed=seed)
    return run_load(srv, Q, sch)


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
def test_served_mix_equals_alone(mode):
    """Each request's ids and scores, served in a Poisson mix of requests of
    several sizes and two k on overlapping streams, are bit-identical to the
    same request searched alone with lider_search."""
    import torch
    from paper_2205_00970_b300.serving import Server
    from tests.lider_fixtures import gpu_index, workload

    cfg, X, Q, C, A, b = workload("tiny")
    cfg = dict(cfg, score_mode=mode, rerank=2 if mode in (2, 4) else 0)
    ix = gpu_index(cfg, X, C, A, b)
    srv = Server(ix, cfg["c"], slots=3, max_batch=512, max_k=20, mem_budget=256 << 20, max_wait_us=300)
    sent = _poisson(Q, srv, 300000, 0.5, (10, 20), 128, 7)
    results = [(off, size, k, t.result(timeout=60)) for off, size, k, t in sent]
    st = srv.stats()
    lat = srv.latencies_ms()
    srv.close()
    assert st["requests"] == len(sent) and st["failed"] == 0
    assert st["batches"] < len(sent)
    assert len(lat) == len(sent) and np.all(lat > 0)
    assert 0 < st["max_inflight_bytes"] <= 256 << 20
    for off, size, k, (ids, sc) in results:
        ai, asc = ix.search(torch.from_numpy(Q[off:off + size]).cuda(), k, cfg["c"])
        assert np.array_equal(ids, ai.cpu().numpy()), (off, size, k)
        assert np.array_equal(sc, asc.cpu().numpy()), (off, size, k)
    ix.free()


@pytest.mark.gpu
def test_pinned_and_pageable_requests_in_one_batch():
    """Requests alternating between pinned queries (copied to the device
    directly) and pageable ones (gathered into the slot's staging) share
    batches; each result equals the same request searched alone."""
    import torch
    from paper_2205_00970_b300.serving import Server, poisson_schedule
    from tests.lider_fixtures import gpu_index, workload

    cfg, X, Q, C, A, b = workload("tiny")
    cfg = dict(cfg, score_mode=3)
    ix = gpu_index(cfg, X, C, A, b)
    Qp = torch.from_numpy(Q).pin_memory().numpy()
    srv = Server(ix, cfg["c"], slots=2, max_batch=512, max_k=20, mem_budget=256 << 20, max_wait_us=2000)
    _, size, ks, off = poisson_schedule(300000, 0.2, ks=(10, 20), max_req=64, n_queries=Q.shape[0], seed=3)
    sent = []
    for i in range(len(size)):
        src = Qp if i % 2 else Q
        o, n, k = int(off[i]), int(size[i]), int(ks[i])
        sent.append((o, n, k, srv.submit(src[o:o + n], k)))
    results = [(o, n, k, t.result(timeout=60)) for o, n, k, t in sent]
    st = srv.stats()
    srv.close()
    assert st["failed"] == 0 and st["batches"] < len(sent)
    for o, n, k, (ids, sc) in results:
        ai, asc = ix.search(torch.from_numpy(Q[o:o + n]).cuda(), k, cfg["c"])
        assert np.array_equal(ids, ai.cpu().numpy()), (o, n, k)
        assert np.array_equal(sc, asc.cpu().numpy()), (o, n, k)
    ix.free()


@pytest.mark.gpu
def test_server_refusals_and_drain():
    from paper_2205_00970_b300 import lider
    from paper_2205_00970_b300.serving import Server
    from tests.lider_fixtures import gpu_index, workload

    cfg, X, Q, C, A, b = workload("tiny")
    ix = gpu_index(cfg, X, C, A, b)
    with pytest.raises(lider.LiderError):                  # c out of range
        Server(ix, cfg["n_clusters"] + 1)
    srv = Server(ix, cfg["c"], slots=2, max_batch=64, max_k=10, mem_budget=1 << 30)
    with pytest.raises(lider.LiderError) as e:
        srv.submit(Q[:65], 10)
    assert e.value.code == -4
    with pytest.raises(lider.LiderError):
        srv.submit(Q[:8], 11)
    empty = srv.submit(Q[:0], 10)
    assert empty.result(timeout=1)[0].shape == (0, 10)
    tickets = [srv.submit(Q[i:i + 7], 10) for i in range(0, 700, 7)]
    srv.close()                                            # drains every request
    for i, t in zip(range(0, 700, 7), tickets):
        ids, _ = t.result(timeout=0)
        assert ids.shape == (7, 10) and np.all(ids[:, 0] >= 0)
    ix.free()


@pytest.mark.gpu
def test_concurrent_host_searches_equal_device_search():
    """Two host threads, each calling lider_search_host on a stream of its
    own (how the bench keeps two batches in flight end to end), get the ids
    and scores lider_search returns on device buffers, bit for bit; the
    batches are large enough for the chunked copy-in, and both threads' searches
    share the index's second stream."""
    import threading

    import torch
    from paper_2205_00970_b300 import lider, synth

    d, k, c = 128, 20, 4
    X = synth.corpus(3, 120_000, d, 64, 0.3, None)
    Q = synth.queries(3, 12_000, d, 64, 0.3, None)
    A, b = synth.projections(3, 4, 16, d, 1.0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ix = lider.Index(t(X), None, t(A), t(b), L=4, m=16, W=1.0, rmi_leaves=64, r0=2, score_mode=lider.SCORE_F16,
                     n_clusters=32, kmeans_iters=4, kmeans_sample=16_384, seed=3)
    ref_ids, ref_sc = ix.search(t(Q), k, c)
    ref_ids, ref_sc = ref_ids.cpu().numpy(), ref_sc.cpu().numpy()
    Qh = torch.from_numpy(Q).pin_memory()
    slices = [(0, 12_000), (1_000, 9_000), (5_000, 12_000), (0, 4_096)]
    out, errors = {}, []

    def work(tid):
        try:
            s = torch.cuda.Stream()
            for j, (lo, hi) in enumerate(slices):
                ids = torch.empty((hi - lo, k), dtype=torch.int64).pin_memory()
                sc = torch.empty((hi - lo, k), dtype=torch.float32).pin_memory()
                ix.search_host(Qh[lo:hi], k, c, ids, sc, stream=s)
                out[(tid, j)] = (ids.numpy().copy(), sc.numpy().copy())
        except Exception as e:  # surfaced in the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    assert len(out) == 2 * len(slices)
    for (tid, j), (ids, sc) in out.items():
        lo, hi = slices[j]
        assert np.array_equal(ids, ref_ids[lo:hi]), (tid, j)
        assert np.array_equal(sc, ref_sc[lo:hi]), (tid, j)
    ix.free()
