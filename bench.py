#!/usr/bin/env python
"""LIDER batched query search throughput on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lider|reference]

One step = one lider_search of the whole query batch of the workload (all
steps of the method: hash, route, group, locate/expand, gather/score/top-k,
merge) with the index and queries resident in HBM.  Prints one JSON line.

  value     queries/s over all ranks (device-resident inputs, CUDA events)
  e2e       the same through lider_search_host: queries copied from pinned
            host memory and results copied back inside the timed region
  roofline  the tensor-core score kernel (tc_score_kernel): executed tensor
            FLOPs per launch (tiles x 128 x 256 x K x 2, x3 for 3xTF32) / its
            event-timed duration vs the measured dense peak of its type
            (--score simt: the FP32 CUDA-core peak)
  cpu_baseline  the FP64 oracle on a bounded query sample on host cores

--impl reference times the FP64 oracle itself (there is no released
implementation of the paper) on the same workload and prints its line.
Under torchrun (N > 1) every rank searches its own replica (replicas only:
the method has no cross-GPU exchange at one-GPU scale); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2205_00970_b300 import configs, synth  # noqa: E402

METRIC = "queries/s at fixed recall@10 vs FP64 oracle (plain vs served BF16); p50/p99 ms"
# our kernels per pass of lider_search on device buffers with the
# multi-kernel grouping (phase list in search.cu; confirmed by the ncu launch
# list; the tensor modes launch the front kernel twice, routing and hash
# tiles); a pass of at most GROUP_ONE_BLOCK_PAIRS pairs over at most
# GROUP_ONE_BLOCK_CLUSTERS clusters groups them in one launch instead of
# GROUP_SAVED + 1
LAUNCHES_PER_SEARCH = {"tensor": 20, "simt": 10, "bf16": 19, "f16": 20, "fp8": 19}
GROUP_SAVED = {"tensor": 3, "simt": 2, "bf16": 3, "f16": 3, "fp8": 3}
GROUP_ONE_BLOCK_PAIRS, GROUP_ONE_BLOCK_CLUSTERS = 131_072, 4_096


def launches_per_pass(score: str, nq_pass: int, c: int, n_clusters: int) -> int:
    n = LAUNCHES_PER_SEARCH[score]
    if nq_pass * c <= GROUP_ONE_BLOCK_PAIRS and n_clusters <= GROUP_ONE_BLOCK_CLUSTERS:
        n -= GROUP_SAVED[score]
    return n
MODES = {"tensor": 0, "simt": 1, "bf16": 2, "f16": 3, "fp8": 4}
DTYPES = {"tensor": "f32", "simt": "f32", "bf16": "bf16", "f16": "f16", "fp8": "fp8-e4m3"}
FP8_PER_BF16 = 4.5 / 2.25     # nominal dense FP8 / BF16 tensor rate (B300)
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one warm tc_score_kernel<KindF16>
# launch on the full mid workload, per tile (None: no capture of the current kernel)
F16_TC_DRAM_BYTES_PER_TILE = (1739497472 + 1207282432) / 20234
F16_TC_DRAM_NOTE = "ncu DRAM bytes of one full-size mid launch (20,234 tiles), per tile, times this launch's tiles"


def workload_desc(cfg) -> dict:
    return {
        "workload": (f"{cfg['name']}: corpus {cfg['n']:,} x {cfg['d']} FP32 ({cfg['n_comp']:,}-component "
                     f"Gaussian mixture{', Zipf(%s) component sizes' % cfg['zipf_s'] if cfg['zipf_s'] else ''}, "
                     f"sigma {cfg['sigma']}, L2-normalised), {cfg['nq']:,} queries; "
                     f"{cfg['n_clusters']} k-means clusters, c={cfg['c']}; L={cfg['L']}, m={cfg['m']}, "
                     f"W={cfg['W']}; RMI {cfg['leaves']} leaves; k={cfg['k']}, R=r0*k={cfg['R']}; seed {cfg['seed']}"),
        "nq_per_step": cfg["nq"],
        "l2": f"inputs larger than L2 (corpus {cfg['n'] * cfg['d'] * 4 / 1e9:.2f} GB resident)",
    }


def load_inputs(cfg):
    """Corpus, queries and the LSH draws of the workload (seeded, synthetic).
    The clustering is not an input: lider_build runs k-means itself."""
    X = synth.corpus(cfg["seed"], cfg["n"], cfg["d"], cfg["n_comp"], cfg["sigma"], cfg["zipf_s"])
    Q = synth.queries(cfg["seed"], cfg["nq"], cfg["d"], cfg["n_comp"], cfg["sigma"], cfg["zipf_s"])
    A, b = synth.projections(cfg["seed"], cfg["L"], cfg["m"], cfg["d"], cfg["W"])
    return X, Q, A, b


def build_gpu_index(cfg, Xd, A, b, centroids=None, **kw):
    """lider_build with k-means on the device (the workload's n_clusters,
    kmeans_iters, kmeans_sample and seed), or lider_build_centroids when the
    centroids of an earlier build are given.  Returns the index."""
    import torch

    from paper_2205_00970_b300 import lider
    dev = Xd.device
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    opts = dict(L=cfg["L"], m=cfg["m"], W=cfg["W"], rmi_leaves=cfg["leaves"], r0=cfg["r0"], B=cfg["B"])
    opts.update(kw)
    if centroids is not None:
        return lider.Index(Xd, t(centroids), t(A), t(b), **opts)
    return lider.Index(Xd, None, t(A), t(b), n_clusters=cfg["n_clusters"], kmeans_iters=cfg["kmeans_iters"],
                       kmeans_sample=cfg["kmeans_sample"], seed=cfg["seed"], **opts)


TF32_PER_BF16 = 1.1 / 2.25     # nominal dense TF32 / BF16 tensor rate (B300)


def measured_peaks():
    """(HBM GB/s, BF16 TFLOP/s burst, BF16 TFLOP/s sustained, source)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    return 6400.0, 1800.0, 1400.0, "fallback"


def fp32_simt_peak_tflops(sm_mhz: float, sms: int = 148) -> float:
    """FP32 FMA issue peak of the CUDA cores: 128 lanes x 2 flop per SM per clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, keep_dir: str | None = None):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.keep_dir = keep_dir        # where the raw samples stay (default: a temporary file)

    def start(self):
        if self.keep_dir:
            os.makedirs(self.keep_dir, exist_ok=True)
            self.path = os.path.join(self.keep_dir, f"clocks_gpu{self.gpu}.csv")
        else:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix=f"clocks_gpu{self.gpu}_", suffix=".csv")
            os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            if not self.keep_dir and self.path:
                try:
                    os.unlink(self.path)
                except OSError:
                    pass
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names[1:], f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not self.keep_dir:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- oracle ---

class blas_threads:
    """Limit the OpenBLAS bundled with numpy to `n` threads inside the block
    (so the timed oracle uses one core); a no-op if no OpenBLAS is loaded."""

    def __init__(self, n: int):
        import ctypes
        self.n, self.prev, self.set, self.get = n, None, None, None
        for line in open("/proc/self/maps"):
            path = line.split()[-1]
            if "openblas" in path.lower() and ".so" in path:
                lib = ctypes.CDLL(path)
                for prefix in ("scipy_openblas", "openblas"):
                    for suffix in ("64_", ""):
                        s = getattr(lib, f"{prefix}_set_num_threads{suffix}", None)
                        g = getattr(lib, f"{prefix}_get_num_threads{suffix}", None)
                        if s is not None and g is not None:
                            self.set, self.get = s, g
                            break
                    if self.set:
                        break
            if self.set:
                break

    @property
    def active(self) -> bool:
        return self.set is not None

    def __enter__(self):
        if self.set:
            self.prev = int(self.get())
            self.set(self.n)
        return self

    def __exit__(self, *a):
        if self.set and self.prev:
            self.set(self.prev)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_POOL_INDEX = None     # the oracle index the forked pool workers search


def _pool_init():
    global _POOL_LIMIT
    _POOL_LIMIT = blas_threads(1)       # one BLAS thread per worker: the pool owns the cores
    _POOL_LIMIT.__enter__()


def _pool_search(job):
    from oracle import lider_oracle as O
    Q, k, c, R = job
    r = O.search(_POOL_INDEX, Q, k, c, R)
    return r.ids


def oracle_build(cfg, X, A, b):
    """The oracle's own index: its k-means from the same seed (Forgy rows,
    Lloyd iterations), the partition and hashes, and every cluster's sorted
    arrays (the search builds them on first use otherwise).  Returns
    (index, seconds of k-means, seconds of the rest)."""
    from oracle import lider_oracle as O
    t = time.perf_counter()
    ns = min(cfg["kmeans_sample"], cfg["n"])
    C = O.kmeans(X[:ns], X[:ns][O.forgy_rows(cfg["seed"], ns, cfg["n_clusters"])], cfg["kmeans_iters"])
    t_km = time.perf_counter() - t
    t = time.perf_counter()
    idx = O.build_index(X, C, A, b, cfg["L"], cfg["m"], cfg["W"], cfg["leaves"], B=cfg["B"])
    for j in range(cfg["n_clusters"]):
        idx.core(j, fit=False)
    return idx, t_km, time.perf_counter() - t


def oracle_pool_search(idx, Q, cfg, cores: int, batch: int, budget_s: float | None, min_queries: int = 0):
    """Search queries Q[0], Q[1], ... with the oracle on `cores` forked
    workers (batches of `batch` queries, in order) until all are done or,
    with a budget, at least min_queries are done and budget_s has passed.
    Returns (ids of the queries done, seconds)."""
    import multiprocessing as mp
    global _POOL_INDEX
    _POOL_INDEX = idx
    jobs = [(Q[i:i + batch], cfg["k"], cfg["c"], cfg["R"]) for i in range(0, len(Q), batch)]
    out = []
    with mp.get_context("fork").Pool(cores, initializer=_pool_init) as pool:
        t = time.perf_counter()
        for ids in pool.imap(_pool_search, jobs, chunksize=1):
            out.append(ids)
            done = sum(len(o) for o in out)
            if budget_s is not None and done >= min_queries and time.perf_counter() - t >= budget_s:
                break
        elapsed = time.perf_counter() - t
        pool.terminate()
    return np.concatenate(out) if out else np.zeros((0, cfg["k"]), np.int64), elapsed


class OracleBaseline:
    """The FP64 oracle timed on every host core, in a child process forked
    before this process starts CUDA (so its worker pool forks from a process
    without a CUDA context).  The child waits until the GPU measurement is
    over, then builds the oracle's own index (k-means from the same seed) and
    searches a bounded sample of the queries: at least `min_queries` and at
    least `budget_s` seconds of search, on a fork pool of one worker per core
    (BLAS one thread each); its ids come back to this process.  Nothing in
    the child touches the GPU."""

    def __init__(self, cfg, X, Q, A, b, budget_s: float, min_queries: int):
        import multiprocessing as mp
        self.conn, child = mp.Pipe()
        self.pid = os.fork()
        if self.pid == 0:                                   # child: no CUDA here
            code = 0
            try:
                msg = child.recv()
                if msg is not None:
                    child.send(self._run(cfg, X, Q, A, b, budget_s, min_queries, msg))
            except Exception as e:  # noqa: BLE001 - reported in the line
                try:
                    child.send({"error": f"{type(e).__name__}: {e}"[:300]})
                except Exception:  # noqa: BLE001
                    code = 1
            os._exit(code)
        child.close()

    @staticmethod
    def _run(cfg, X, Q, A, b, budget_s, min_queries, _go):
        cores = host_cores()
        idx, t_km, t_build = oracle_build(cfg, X, A, b)
        ref_ids, search_s = oracle_pool_search(idx, Q, cfg, cores, 4, budget_s, min_queries)
        return {"ids": ref_ids, "search_s": search_s, "cores": cores, "t_km": t_km, "t_build": t_build}

    def result(self, gpu_ids, X, Q) -> dict:
        """Start the oracle, wait for it, and report its throughput with
        recall@10 of both sides on its sample against FP64 brute force (on the
        device, for at most the first 2,000 sampled queries)."""
        self.conn.send(True)
        r = self.conn.recv()
        os.waitpid(self.pid, 0)
        if "error" in r:
            return r
        ref_ids, search_s, cores = r["ids"], r["search_s"], r["cores"]
        done = len(ref_ids)
        nt = min(done, 2000)
        truth = fp64_knn(X, Q[:nt], 10)
        extrapolated = done < len(Q)
        return {
            "value": done / search_s, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": (f"first {done:,} of {len(Q):,} queries of the same workload, FP64 oracle search "
                       f"(Python/numpy) on {cores} worker processes (one BLAS thread each), {search_s:.1f} s"
                       f"{'; queries/s extrapolated from the sample' if extrapolated else ''}; the oracle's own "
                       f"k-means ({r['t_km']:.1f} s) and index build ({r['t_build']:.1f} s) not timed"),
            "oracle_build_s": {"kmeans": r["t_km"], "index": r["t_build"]},
            "recall_sample": f"first {nt:,} queries against FP64 brute force",
            "recall_at_10_gpu": recall10(gpu_ids[:nt], truth),
            "recall_at_10_oracle": recall10(ref_ids[:nt], truth),
            "gpu_eq_oracle_top10": float(np.mean([np.array_equal(gpu_ids[i, :10], ref_ids[i, :10])
                                                  for i in range(done)])),
        }

    def cancel(self):
        try:
            self.conn.send(None)
            os.waitpid(self.pid, 0)
        except Exception:  # noqa: BLE001
            pass


def run_reference(args, cfg):
    """--impl reference: the FP64 oracle timed on every host core (rank 0
    only): its own k-means and index build (not timed), then per step one
    batch of --ref-queries-per-step queries per core, searched by a fork pool
    of one worker per core."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    X, Q, A, b = load_inputs(cfg)
    idx, t_km, t_build = oracle_build(cfg, X, A, b)
    cores = host_cores()
    per_step = args.ref_queries_per_step * cores
    times = []
    for s in range(args.warmup + args.steps):
        q0 = (s * per_step) % len(Q)
        Qs = Q[q0:q0 + per_step]
        _, sec = oracle_pool_search(idx, Qs, cfg, cores, args.ref_queries_per_step, None)
        if s >= args.warmup:
            times.append(sec)
    total = sum(times)
    value = per_step * len(times) / total
    sample = (f"{per_step} queries per step of the {cfg['nq']:,}-query batch ({args.ref_queries_per_step} per "
              f"worker), FP64 oracle (Python/numpy) on {cores} worker processes (one BLAS thread each); its "
              f"k-means ({t_km:.1f} s) and index build ({t_build:.1f} s) not timed")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_desc(cfg),
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ lider ---

def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks of the job (its time is its slowest
    rank's); x itself when there is one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(nq_per_rank: int, steps: int, world: int, job_ms: float) -> float:
    """Queries/s of the whole job: every rank searches its own replica of the
    index over nq_per_rank queries per step (replicas: weak scaling)."""
    return world * nq_per_rank * steps / (job_ms / 1e3)


def score_roofline(score: str, stats: dict, route: np.ndarray, cl_off: np.ndarray, d: int, score_s: float,
                   clk: dict) -> dict:
    """Roofline of the score phase (tc_units_kernel + tc_score_kernel, or the
    SIMT score_group_kernel) on the method's own work:
      achieved  useful FLOPs, 2 x (unique candidates) x d, per second;
      peak      the measured dense tensor peak of the contraction's type
                (TF32 and FP8 from the BF16 figure by the nominal ratios);
      executed  the FLOPs of the dense tiles actually run (padding included);
      unique_bytes  what the phase must read at least once: the rows of the
                probed clusters and the gathered queries in the operand type,
                plus one candidate bitmap word per 32 cluster positions per
                (query, cluster) pair; against the measured copy bandwidth."""
    cand = stats["candidates"]
    useful = 2.0 * cand * d
    hbm, bf16, _, peak_kind = measured_peaks()
    src = "of measured (MEASURED_PEAKS.json)" if peak_kind == "measured" else "of fallback"
    sizes = np.diff(cl_off)
    probed = np.unique(route[route >= 0])
    pair_sizes = sizes[route.ravel()]
    operand = {"tensor": 8, "f16": 2, "bf16": 2, "fp8": 1, "simt": 4}[score]
    ub = float(sizes[probed].sum() * d * operand + route.size * d * operand + np.sum(-(-pair_sizes // 32)) * 4)
    if score == "simt":
        peak = fp32_simt_peak_tflops(clk.get("sm_max_mhz") or 2032.0)
        r = {"bound": "alu", "kernel": "score_group_kernel", "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
        executed = None
    else:
        if score == "tensor":
            kpad, mult, peak = -(-d // 32) * 32, 3, bf16 * TF32_PER_BF16
            psrc = f"bf16 burst {bf16} x {TF32_PER_BF16:.3f} (nominal TF32/BF16), {src}"
        elif score == "fp8":
            kpad, mult, peak = -(-d // 128) * 128, 1, bf16 * FP8_PER_BF16
            psrc = f"bf16 burst {bf16} x {FP8_PER_BF16:.1f} (nominal FP8/BF16), {src}"
        else:
            kpad, mult, peak = -(-d // 64) * 64, 1, bf16
            psrc = f"bf16 burst {bf16}" + (" (FP16 has the same dense rate)" if score == "f16" else "") + f", {src}"
        executed = stats["tc_tiles"] * 128 * 256 * kpad * 2.0 * mult
        r = {"bound": "tensor", "kernel": "tc_score_kernel", "peak_source": psrc}
    achieved = useful / score_s / 1e12
    # DRAM bytes per launch: the full-size capture's bytes per tile times this
    # launch's tiles (the FP16 mode's kernel at the time of the capture)
    traffic = F16_TC_DRAM_BYTES_PER_TILE * stats["tc_tiles"] if (score == "f16" and F16_TC_DRAM_BYTES_PER_TILE) else None
    r.update({
        "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
        "work": "useful: 2 x unique candidates x d per launch", "useful_flop_per_launch": useful,
        "phase_ms": score_s * 1e3,
        "unique_bytes": {"bytes_per_launch": ub, "achieved_gbs": ub / score_s / 1e9, "peak_gbs": hbm,
                         "frac": ub / score_s / 1e9 / hbm},
    })
    if executed is not None:
        r["executed"] = {"flop_per_launch": executed, "tiles_per_launch": stats["tc_tiles"],
                         "tflops": executed / score_s / 1e12, "frac": executed / score_s / 1e12 / peak,
                         "useful_share": useful / executed}
    if traffic is not None:
        r["traffic_gbs"] = {"achieved": traffic / score_s / 1e9, "peak": hbm, "frac": traffic / score_s / 1e9 / hbm,
                            "note": F16_TC_DRAM_NOTE}
    return r


def run_lider(args, cfg):
    import torch
    import torch.distributed as dist

    from paper_2205_00970_b300 import lider

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    X, Q, A, b = load_inputs(cfg)
    # the CPU baseline's process forks now, before this process starts CUDA
    oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        oracle = OracleBaseline(cfg, X, Q, A, b, args.cpu_budget, args.cpu_min_queries)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    Xd = t(X)
    mode = MODES[args.score]
    idx = build_gpu_index(cfg, Xd, A, b, score_mode=mode, rerank=args.rerank)
    build = idx.build_info()
    C = idx.centroids()          # reused by the served comparison's index
    del Xd
    Qd = t(Q)
    k, c, nq = cfg["k"], cfg["c"], cfg["nq"]
    ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
    sc = torch.empty((nq, k), dtype=torch.float32, device=dev)
    # a step searches the whole batch in one lider_search call (the library
    # splits a batch into passes when one pass cannot hold it), or in calls
    # of --sub-batch queries
    sub = call_size(idx, nq, k, c, args.sub_batch or nq)
    chunks = [(lo, min(nq, lo + sub)) for lo in range(0, nq, sub)]

    def search_all(stream=None):
        for lo, hi in chunks:
            idx.search(Qd[lo:hi], k, c, out=(ids[lo:hi], sc[lo:hi]), stream=stream)

    tuning = None
    if not args.no_autotune:
        # launch shapes picked by timing searches of the first call's queries (outside the timed region)
        lo, hi = chunks[0]
        tune, tune_ms = idx.autotune(Qd[lo:hi], k, c, reps=3)
        tuning = dict(tune, ms_per_search=tune_ms, queries_per_call=hi - lo)
    stats = None
    route = np.zeros((nq, c), dtype=np.int32)
    for lo, hi in chunks:
        _, _, st, tr = idx.search(Qd[lo:hi], k, c, stats=True, trace=True, out=(ids[lo:hi], sc[lo:hi]))
        route[lo:hi] = tr["route"].cpu().numpy()
        stats = st if stats is None else {key: stats[key] + st[key] for key in stats}
    gpu_ids = ids.cpu().numpy()

    for _ in range(args.warmup):
        search_all()
    nph = lider.NUM_PHASES + 1
    # the timed steps run the plain lider_search calls; events mark only the
    # steps' boundaries (phase events inside a search cost it time)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    # with one pass per call, the score phase of every timed call is timed too
    # (two events in the search, at its start and end: the roofline's kernel)
    one_pass = stats.get("passes", len(chunks)) <= len(chunks)
    iS, iE = lider.PHASES.index("score"), lider.PHASES.index("select")
    sev = [[[torch.cuda.Event(enable_timing=True) if i in (iS, iE) else None for i in range(nph)] for _ in chunks]
           for _ in range(args.steps)] if one_pass else None
    for e in evs + [e for st in (sev or []) for row in st for e in row if e is not None]:
        e.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local, args.clocks_dir)
    clocks.start()
    time.sleep(0.3)
    evs[0].record()
    for s in range(args.steps):
        if one_pass:
            for ci, (lo, hi) in enumerate(chunks):
                idx.search_phased(Qd[lo:hi], k, c, sev[s][ci], out=(ids[lo:hi], sc[lo:hi]))
        else:
            search_all()
        evs[s + 1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    total_ms = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[s].elapsed_time(evs[s + 1]) for s in range(args.steps)]
    passes = stats.get("passes", len(chunks))
    # the phases: an untimed run of the same search, one call per pass, with
    # the library recording events at its phase boundaries
    per_call = max(1, passes // len(chunks))
    pb = -(-min(hi - lo for lo, hi in chunks) // per_call) if passes > len(chunks) else None
    calls = [(a, min(hi, a + pb)) for lo, hi in chunks for a in range(lo, hi, pb)] if pb else list(chunks)
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(nph)] for _ in calls]
    for row in pev:
        for e in row:
            e.record()              # creates the event, so the library gets a handle to record
    for pi, (lo, hi) in enumerate(calls):
        idx.search_phased(Qd[lo:hi], k, c, pev[pi], out=(ids[lo:hi], sc[lo:hi]))
    torch.cuda.synchronize()
    phase_ms = {name: float(sum(ev[i].elapsed_time(ev[i + 1]) for ev in pev)) for i, name in enumerate(lider.PHASES)}
    phase_of = (f"an untimed run of the same search, {len(calls)} call(s) of "
                f"{max(hi - lo for lo, hi in calls):,} queries with phase events")
    if one_pass:
        score_ms = float(np.mean([sum(sev[s][ci][iS].elapsed_time(sev[s][ci][iE]) for ci in range(len(chunks)))
                                  for s in range(args.steps)]))
        score_of = "the timed steps (events at the score phase's start and end)"
    else:
        score_ms = phase_ms["score"]
        score_of = phase_of
    total_ms = max_over_ranks(total_ms, dev)
    value = job_throughput(nq, args.steps, world, total_ms)

    # the same search captured once into a CUDA graph and replayed
    graph = None
    try:
        gs = torch.cuda.Stream()
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=gs):
            search_all(stream=gs)
        for _ in range(args.warmup):
            cg.replay()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        g0.record()
        for _ in range(args.steps):
            cg.replay()
        g1.record()
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / args.steps
        graph = {"value": world * nq / (gms / 1e3), "unit": "queries/s", "ms_per_step": gms,
                 "of": "lider_search captured once with torch.cuda.graph and replayed"}
        del cg
    except Exception as e:  # noqa: BLE001 - reported, not fatal
        graph = {"error": str(e)[:200]}

    # end to end: pinned host queries in, host results out, every step
    Qh = torch.from_numpy(Q).pin_memory()
    ids_h = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    sc_h = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    def search_host_all():
        for lo, hi in chunks:
            idx.search_host(Qh[lo:hi], k, c, ids_h[lo:hi], sc_h[lo:hi])

    for _ in range(max(1, args.warmup // 2)):
        search_host_all()
    if world > 1:
        dist.barrier()
    te = time.perf_counter()
    for _ in range(args.steps):
        search_host_all()
    e2e_s = max_over_ranks(time.perf_counter() - te, dev)
    e2e_value = job_throughput(nq, args.steps, world, e2e_s * 1e3)
    # the same steps with two batches in flight, as a serving client keeps
    # them: two host threads, each calling lider_search_host on a stream and
    # result arrays of its own, take the steps in turn; every step still
    # copies its queries in and its results out inside the timed region
    from concurrent.futures import ThreadPoolExecutor
    p_streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    p_outs = [(ids_h, sc_h), (torch.empty_like(ids_h).pin_memory(), torch.empty_like(sc_h).pin_memory())]

    def host_steps(t, n_steps):
        for _ in range(n_steps):
            for lo, hi in chunks:
                idx.search_host(Qh[lo:hi], k, c, p_outs[t][0][lo:hi], p_outs[t][1][lo:hi], stream=p_streams[t])

    with ThreadPoolExecutor(2) as ex:
        list(ex.map(host_steps, [0, 1], [1, 1]))
        if world > 1:
            dist.barrier()
        tp = time.perf_counter()
        for f in [ex.submit(host_steps, t, (args.steps + 1 - t) // 2) for t in range(2)]:
            f.result()
        e2e2_s = max_over_ranks(time.perf_counter() - tp, dev)
    e2e2_value = job_throughput(nq, args.steps, world, e2e2_s * 1e3)
    pipe_ok = (np.array_equal(p_outs[1][0].numpy(), p_outs[0][0].numpy())
               and np.array_equal(p_outs[1][1].numpy(), p_outs[0][1].numpy()))
    link = host_link_rates(Qh, int(nq * k * (8 + 4)), dev)

    roofline = score_roofline(args.score, stats, route, idx.cluster_offsets(), cfg["d"], score_ms / 1e3,
                              clk)
    served = None
    if world == 1 and args.score in ("f16", "tensor", "simt") and not args.no_served:
        served = served_compare(args, cfg, X, C, A, b, Qd, chunks, gpu_ids, dev)
    build_line = {"kmeans_ms": build["kmeans_ms"], "build_ms": build["build_ms"],
                  "clustering": (f"k-means on the device: {build['n_clusters']} clusters, {build['kmeans_iters']} "
                                 f"Lloyd iterations on the first {build['train_rows']:,} rows, Forgy rows from "
                                 f"seed {build['seed']}"),
                  "empty_clusters": build["empty_clusters"], "timed": False}

    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.score], "data": "synthetic",
        "config": dict(workload_desc(cfg), parallelism=f"replicas x{world}"),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "of": f"one batch of {nq:,} queries"},
        "phase_ms": phase_ms,
        "phase_ms_of": phase_of,
        "passes_per_step": passes,
        "search_stats": stats,
        "roofline": dict(roofline, phase_timed_in=score_of),
        "e2e": {"value": e2e2_value, "unit": "queries/s", "h2d_bytes_per_step": int(Q.nbytes),
                "d2h_bytes_per_step": int(nq * k * (8 + 4)), "ms_per_step": e2e2_s * 1e3 / args.steps,
                "of": ("two batches in flight: two host threads, each calling lider_search_host on its own "
                       "stream and pinned result arrays, take the steps in turn (each step copies its "
                       "queries in and its results out inside the timed region)"),
                "results_equal_across_threads": bool(pipe_ok),
                "one_at_a_time": {"value": e2e_value, "ms_per_step": e2e_s * 1e3 / args.steps,
                                  "of": "one lider_search_host call at a time"},
                "host_link": link},
        "gpu_launches": sum(launches_per_pass(args.score, hi - lo, c, cfg["n_clusters"])
                            for lo, hi in calls) * args.steps,
        "graph_replay": graph,
        "tuning": tuning,
        "score_mode": args.score,
        "results": ("exact FP32 top-k of each query's candidate union (approximate tensor scores select with a "
                    "proven guard band, every listed id is re-scored in FP32; equal bit for bit across "
                    "f16/tensor/simt)") if args.score not in ("bf16", "fp8") else
                   f"served shortlist: {DTYPES[args.score]} scores, FP32 re-rank of the best {args.rerank} * k",
        "clocks": clk,
    }
    line["build"] = build_line
    if served is not None:
        line["served_bf16"] = served
    if oracle is not None:
        line["cpu_baseline"] = oracle.result(gpu_ids, X, Q)
    if rank == 0:
        print(json.dumps(line), flush=True)
    idx.free()
    if world > 1:
        dist.destroy_process_group()
    return 0


def served_compare(args, cfg, X, C, A, b, Qd, chunks, plain_ids, dev) -> dict:
    """The metric's other side: the served BF16 form (BF16 corpus copy scored
    on the tensor cores, FP32 re-rank of a shortlist of --served-rerank * k)
    on the same queries, timed the same way; recall@10 against FP64 brute
    force on the first --recall-nq queries for it and for the plain (exact)
    search, and against the plain search's top-10 on every query.  Errors are
    reported in the line, not raised."""
    import torch

    from paper_2205_00970_b300 import lider
    try:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        Xd = t(X)
        sidx = lider.Index(Xd, t(C), t(A), t(b), L=cfg["L"], m=cfg["m"], W=cfg["W"], rmi_leaves=cfg["leaves"],
                           r0=cfg["r0"], B=cfg["B"], score_mode=lider.SCORE_BF16, rerank=args.served_rerank)
        del Xd
        k, c, nq = cfg["k"], cfg["c"], Qd.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
        sc = torch.empty((nq, k), dtype=torch.float32, device=dev)

        def once():
            for lo, hi in chunks:
                sidx.search(Qd[lo:hi], k, c, out=(ids[lo:hi], sc[lo:hi]))

        if not args.no_autotune:
            lo, hi = chunks[0]
            sidx.autotune(Qd[lo:hi], k, c, reps=3)
        for _ in range(args.warmup):
            once()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            once()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        got = ids.cpu().numpy()
        sidx.free()
        del sidx
        torch.cuda.empty_cache()
        nr = min(args.recall_nq, nq)
        truth = fp64_knn(X, Qd[:nr].cpu().numpy(), 10)
        return {"value": nq / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms,
                "shortlist": f"{args.served_rerank} * k",
                "recall_at_10": recall10(got[:nr], truth), "recall_at_10_plain": recall10(plain_ids[:nr], truth),
                "recall_sample": f"first {nr:,} queries against FP64 brute force",
                "recall_at_10_vs_plain": recall10(got, plain_ids),
                "tuning": "autotuned" if not args.no_autotune else "default launch shapes"}
    except Exception as e:                               # the main line must still print
        return {"error": f"{type(e).__name__}: {e}"[:300]}


def run_serve(args, cfg):
    """Serving mode: Poisson arrivals of requests (log-uniform sizes of 1 to
    --serve-max-req queries, k of 10 or the workload's k) at an offered rate,
    served by the native continuous-batching server; reports the rate served
    and per-request latency percentiles (submission to results in the
    caller's host buffers)."""
    import torch

    from paper_2205_00970_b300 import lider
    from paper_2205_00970_b300.serving import Server, poisson_schedule, run_load

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    X, Q, A, b = load_inputs(cfg)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    Xd = t(X)
    mode = MODES[args.score]
    idx = build_gpu_index(cfg, Xd, A, b, score_mode=mode, rerank=args.rerank)
    del Xd
    ks = (10, cfg["k"])
    srv = Server(idx, cfg["c"], slots=args.serve_slots, max_batch=args.serve_max_batch, max_k=max(ks),
                 mem_budget=args.serve_mem_gb << 30, max_wait_us=args.serve_wait_us)
    nq = Q.shape[0]
    warm = poisson_schedule(args.serve, 0.5, ks=ks, max_req=args.serve_max_req, n_queries=nq, seed=1)
    # the requests' queries live in pinned host memory, so the server copies
    # them to the device directly
    Q = torch.from_numpy(Q).pin_memory().numpy()
    for *_, tk in run_load(srv, Q, warm):
        tk.result()
    srv.latencies_ms(clear=True)
    s0 = srv.stats()
    sch = poisson_schedule(args.serve, args.serve_seconds, ks=ks, max_req=args.serve_max_req, n_queries=nq, seed=2)
    clocks = ClockSampler(0, args.clocks_dir)
    clocks.start()
    t0 = time.perf_counter()
    sent = run_load(srv, Q, sch)
    t_sub = time.perf_counter() - t0
    for *_, tk in sent:
        tk.result()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    s1 = srv.stats()
    lat = srv.latencies_ms()
    srv.close()
    served = s1["queries"] - s0["queries"]
    batches = s1["batches"] - s0["batches"]
    pct = lambda p: float(np.percentile(lat, p)) if lat.size else None
    line = {
        "metric": "served queries/s under Poisson load", "value": served / wall, "unit": "queries/s",
        "offered_qps": args.serve, "offered_qps_actual": float(sch[1].sum() / args.serve_seconds),
        "n_gpus": 1, "requests": len(sent), "higher_is_better": True,
        "latency_ms": {"p50": pct(50), "p90": pct(90), "p99": pct(99), "max": pct(100),
                       "of": "one request, submission to results in host memory"},
        "batches": batches, "mean_batch_queries": served / max(1, batches),
        "max_inflight_batches": s1["max_inflight_batches"],
        "max_inflight_scratch_bytes": s1["max_inflight_bytes"],
        "host_s": {"submit_loop": t_sub, "launch": s1["launch_s"] - s0["launch_s"],
                   "finish": s1["finish_s"] - s0["finish_s"], "wall": wall},
        "dtype": DTYPES[args.score], "data": "synthetic", "score_mode": args.score,
        "config": dict(workload_desc(cfg), request_queries=f"log-uniform 1..{args.serve_max_req}",
                       k=list(ks), slots=args.serve_slots, max_batch=args.serve_max_batch,
                       max_wait_us=args.serve_wait_us),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    idx.free()
    return 0


def call_size(idx, nq, k, c, want):
    """Largest queries-per-call up to `want` that the search's per-call caps
    accept (halving from `want`)."""
    from paper_2205_00970_b300 import lider
    sub = max(1, min(nq, want))
    while sub > 1:
        try:
            idx.search_bytes(sub, k, c)
            return sub
        except lider.LiderError:
            sub //= 2
    return sub


def fp64_knn(X, Q, k: int, chunk: int = 262_144, device: str = "cuda:0") -> np.ndarray:
    """Ground truth for recall: the k largest FP64 inner products of each
    query over the whole corpus (ties to the lower id), computed with plain
    FP64 matrix products (on the GPU by default), chunk by chunk."""
    import torch
    dev = torch.device(device)
    q = torch.from_numpy(np.ascontiguousarray(Q)).to(dev, torch.float64)
    best_s = torch.full((len(Q), 0), 0.0, dtype=torch.float64, device=dev)
    best_i = torch.zeros((len(Q), 0), dtype=torch.int64, device=dev)
    for lo in range(0, X.shape[0], chunk):
        x = torch.from_numpy(np.ascontiguousarray(X[lo:lo + chunk])).to(dev, torch.float64)
        s = q @ x.T
        ids = torch.arange(lo, lo + x.shape[0], device=dev).expand(len(Q), -1)
        cs, ci = torch.cat([best_s, s], 1), torch.cat([best_i, ids], 1)
        # order by score descending, then id ascending (stable sort on id first)
        o1 = torch.argsort(ci, dim=1, stable=True)
        cs, ci = cs.gather(1, o1), ci.gather(1, o1)
        o2 = torch.argsort(-cs, dim=1, stable=True)[:, :k]
        best_s, best_i = cs.gather(1, o2), ci.gather(1, o2)
    return best_i.cpu().numpy()


def host_link_rates(Qh, d2h_bytes: int, dev) -> dict:
    """Plain pinned copies of one step's bytes (the queries in, a buffer of
    the results' size out), timed with CUDA events: the host link's rate, and
    the step's transfer time at that rate if nothing overlapped."""
    import torch
    src = Qh if Qh.is_pinned() else Qh.pin_memory()
    dbuf = torch.empty(src.shape, dtype=src.dtype, device=dev)
    hout = torch.empty(d2h_bytes, dtype=torch.uint8).pin_memory()
    dout = torch.empty(d2h_bytes, dtype=torch.uint8, device=dev)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(2):
        dbuf.copy_(src, non_blocking=True)
        hout.copy_(dout, non_blocking=True)
    torch.cuda.synchronize()
    e[0].record()
    dbuf.copy_(src, non_blocking=True)
    e[1].record()
    hout.copy_(dout, non_blocking=True)
    e[2].record()
    torch.cuda.synchronize()
    h2d_ms, d2h_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    return {"h2d_gbs": src.numel() * src.element_size() / h2d_ms / 1e6, "d2h_gbs": d2h_bytes / d2h_ms / 1e6,
            "copy_ms_per_step": h2d_ms + d2h_ms}


def recall10(found: np.ndarray, truth: np.ndarray) -> float:
    return float(np.mean([len(set(f[:10].tolist()) & set(t[:10].tolist())) / 10 for f, t in zip(found, truth)]))


def run_variants(args, cfg):
    """Fidelity variants of the paper on the workload, each built as its own
    index in the FP16 exact mode and searched over every query: the plain
    method (p-stable hashkeys, exact routing scan, re-scaled keys), hyperplane
    hashkeys (Sec. 4.1, one bit per hash, B = 3), the Layer-1 centroids
    retriever (Sec. 3.2), and RMIs on raw keys (the Sec. 7.4 ablation).
    Reports queries/s, recall@10 against FP64 brute force on a query sample
    and against the plain method on all queries, and the RMI diagnostics of
    Sec. 7.4 (OOR, LE = more than k from the lower bound, and both)."""
    import torch

    from paper_2205_00970_b300 import lider

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    X, Q, A, b = load_inputs(cfg)
    k, c, nq = cfg["k"], cfg["c"], cfg["nq"]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    Qd, Xd = t(Q), t(X)
    first = build_gpu_index(cfg, Xd, A, b, score_mode=lider.SCORE_F16)   # k-means once; the variants share it
    Cd = t(first.centroids())
    first.free()
    variants = {
        "plain": {},
        "hyperplane": dict(hash_kind=lider.HASH_HYPERPLANE, m=args.hyper_m),
        "core_route": dict(route_kind=lider.ROUTE_CORE),
        "raw_keys": dict(raw_keys=True),
    }
    ns = min(args.precision_sample * 16, nq)
    truth = fp64_knn(X, Q[:ns], 10)
    out = {}
    for name, v in variants.items():
        m = v.get("m", cfg["m"])
        if m != cfg["m"]:
            from paper_2205_00970_b300 import synth
            A2, b2 = synth.projections(cfg["seed"], cfg["L"], m, cfg["d"], cfg["W"])
        else:
            A2, b2 = A, b
        idx = lider.Index(Xd, Cd, t(A2), t(b2), L=cfg["L"], m=m, W=cfg["W"], rmi_leaves=cfg["leaves"],
                          r0=cfg["r0"], score_mode=lider.SCORE_F16, hash_kind=v.get("hash_kind", 0),
                          route_kind=v.get("route_kind", 0), raw_keys=v.get("raw_keys", False),
                          B=3 if v.get("hash_kind", 0) == lider.HASH_HYPERPLANE else cfg["B"])
        ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
        sc = torch.empty((nq, k), dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            idx.search(Qd, k, c, out=(ids, sc))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            idx.search(Qd, k, c, out=(ids, sc))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        _, _, st = idx.search(Qd, k, c, stats=True)
        out[name] = {"ids": ids.cpu().numpy(), "ms": ms, "stats": st, "m": m}
        idx.free()
        del idx, ids, sc
        torch.cuda.empty_cache()
    plain = out["plain"]["ids"]
    report = {}
    for name, r in out.items():
        st = r["stats"]
        triples = st["pairs"] * cfg["L"] - st["empty_pairs"] * cfg["L"]
        report[name] = {
            "queries_per_s": nq / (r["ms"] / 1e3), "ms_per_batch": r["ms"], "m": r["m"],
            "recall_at_10_vs_fp64_knn": recall10(r["ids"][:ns], truth),
            "recall_at_10_vs_plain": recall10(r["ids"], plain),
            "candidates_per_query": st["candidates"] / nq,
            "rmi": {"triples": triples, "oor": st["rmi_oor"], "le": st["rmi_le"], "oor_and_le": st["rmi_oor_le"],
                    "le_threshold": k, "locate_fallback": st["locate_fallback"]},
        }
    line = {
        "metric": "fidelity variants: queries/s, recall@10, RMI OOR/LE", "n_gpus": 1, "steps": args.steps,
        "data": "synthetic", "config": workload_desc(cfg), "score_mode": "f16",
        "sample": f"recall vs FP64 brute force on the first {ns} queries; vs plain on all {nq}",
        "variants": report,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args, cfg):
    """Recall@10 against FP64 brute force and queries/s over the operating
    parameters of the search: bucket width W and expansion factor r0 (index
    parameters; one index per pair, all from the first build's clustering) and
    clusters probed c.  The FP16 exact mode searches --sweep-nq queries per
    setting; recall is measured on the first --sweep-recall-nq of them.
    Reports every point and the fastest one with recall@10 >= 0.9 (or that
    none reaches it)."""
    import torch

    from paper_2205_00970_b300 import lider

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    X, Q, A, b = load_inputs(cfg)
    nq = min(args.sweep_nq, cfg["nq"])
    Qd = torch.from_numpy(np.ascontiguousarray(Q[:nq])).to(dev)
    k = cfg["k"]
    truth = fp64_knn(X, Q[:args.sweep_recall_nq], 10)
    Xd = torch.from_numpy(X).to(dev)
    C = None
    points = []
    bound = {}
    for W in args.sweep_W:
        for r0 in args.sweep_r0:
            if cfg["L"] * r0 * k > lider.MAX_LR:
                continue
            c_cfg = dict(cfg, W=W, r0=r0)
            if W != cfg["W"]:
                A2, b2 = synth.projections(cfg["seed"], cfg["L"], cfg["m"], cfg["d"], W)
            else:
                A2, b2 = A, b
            idx = build_gpu_index(c_cfg, Xd, A2, b2, centroids=C, score_mode=lider.SCORE_F16)
            if C is None:
                C = idx.centroids()
                # what any window size could reach: the share of the true top-10
                # that lies in the c probed clusters (the route does not depend
                # on W or r0), and the probed clusters' mean size
                asg = idx.assignment()
                sizes = np.bincount(asg, minlength=cfg["n_clusters"])
                for c in args.sweep_c:
                    if c > min(lider.MAX_C, cfg["n_clusters"]):
                        continue
                    _, _, _, tr = idx.search(Qd[:args.sweep_recall_nq].contiguous(), k, c, stats=True, trace=True)
                    route = tr["route"].cpu().numpy()
                    held = [np.isin(asg[truth[i][:10]], route[i]).mean() for i in range(len(route))]
                    bound[c] = {"true_top10_in_probed_clusters": float(np.mean(held)),
                                "mean_probed_cluster_rows": float(sizes[route].mean())}
            for c in args.sweep_c:
                if c > min(lider.MAX_C, cfg["n_clusters"]):
                    continue
                ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
                sc = torch.empty((nq, k), dtype=torch.float32, device=dev)
                idx.search(Qd, k, c, out=(ids, sc))                   # warm-up
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(args.steps):
                    idx.search(Qd, k, c, out=(ids, sc))
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                got = ids[:args.sweep_recall_nq].cpu().numpy()
                points.append({"W": W, "r0": r0, "c": c, "queries_per_s": nq / (ms / 1e3), "ms_per_batch": ms,
                               "recall_at_10": recall10(got, truth)})
                print(json.dumps({"sweep_point": points[-1]}), flush=True)
            idx.free()
            del idx
            torch.cuda.empty_cache()
    ok = [p for p in points if p["recall_at_10"] >= 0.9]
    best = max(ok, key=lambda p: p["queries_per_s"]) if ok else None
    line = {"metric": "queries/s and recall@10 vs FP64 brute force over W, r0, c", "n_gpus": 1, "steps": args.steps,
            "data": "synthetic", "config": workload_desc(cfg), "score_mode": "f16",
            "sample": (f"{nq:,} queries per setting; recall on the first {args.sweep_recall_nq} against FP64 brute "
                       f"force over all {cfg['n']:,} rows"),
            "points": points, "operating_point_recall_0_9": best,
            "probe_bound": {str(c): v for c, v in bound.items()},
            "window_positions_per_pair": {str(r0): cfg["L"] * r0 * k for r0 in args.sweep_r0},
            "note": None if best else "no setting in the sweep reaches recall@10 0.9"}
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args, cfg):
    """Precision mode: the workload's corpus indexed once per dtype (the exact
    FP16-guarded mode, the served BF16 and FP8-e4m3 forms with a shortlist of
    rerank * k re-ranked in FP32), every query searched; reports per dtype the
    queries/s, recall@10 against the exact mode, and, on a query sample
    against FP64 brute force (fp64_knn), recall@10 and the largest relative
    error of the returned scores."""
    import torch

    from paper_2205_00970_b300 import lider

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    X, Q, A, b = load_inputs(cfg)
    k, c, nq = cfg["k"], cfg["c"], cfg["nq"]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    Qd = t(Q)
    out = {}
    C = None                          # k-means runs in the first build; the others reuse its centroids
    runs = [("f16", 0)] + [(f"{name}@{rr}", rr) for rr in (args.precision_reranks or [args.rerank])
                            for name in ("bf16", "fp8")]
    for name, rr in runs:
        Xd = t(X)
        idx = build_gpu_index(cfg, Xd, A, b, centroids=C, score_mode=MODES[name.split("@")[0]], rerank=max(rr, 1))
        if C is None:
            C = idx.centroids()
        del Xd
        torch.cuda.empty_cache()
        sub = call_size(idx, nq, k, c, args.sub_batch or nq)
        chunks = [(lo, min(nq, lo + sub)) for lo in range(0, nq, sub)]
        ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
        sc = torch.empty((nq, k), dtype=torch.float32, device=dev)
        for lo, hi in chunks:                                   # warm-up
            idx.search(Qd[lo:hi], k, c, out=(ids[lo:hi], sc[lo:hi]))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            for lo, hi in chunks:
                idx.search(Qd[lo:hi], k, c, out=(ids[lo:hi], sc[lo:hi]))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[name] = {"ids": ids.cpu().numpy(), "scores": sc.cpu().numpy(), "ms": ms, "sub": sub}
        idx.free()
        del idx, ids, sc
        torch.cuda.empty_cache()
    plain = out["f16"]["ids"][:, :10]
    ns = min(args.precision_sample, nq)
    truth = fp64_knn(X, Q[:ns], 10)
    q64 = Q[:ns].astype(np.float64)
    report = {}
    for name, r in out.items():
        top = r["ids"][:, :10]
        agree = np.mean([len(set(top[i].tolist()) & set(plain[i].tolist())) / 10 for i in range(nq)])
        err, n_scores = 0.0, 0
        for i in range(ns):
            sel = r["ids"][i][r["ids"][i] >= 0]
            if not len(sel):
                continue
            ex = X[sel].astype(np.float64) @ q64[i]
            got = r["scores"][i][:len(sel)].astype(np.float64)
            rel = np.abs(got - ex) / np.maximum(np.abs(ex), 1e-30)
            err = max(err, float(np.max(rel)) if np.all(np.isfinite(rel)) else float("inf"))
            n_scores += len(sel)
        base, rr = (name.split("@") + ["0"])[:2]
        report[name] = {
            "queries_per_s": nq / (r["ms"] / 1e3), "ms_per_batch": r["ms"], "queries_per_call": r["sub"],
            "storage": {"f16": "FP16 (power-of-two scaled), guarded, exact", "bf16": "BF16",
                        "fp8": "FP8 e4m3, one scale per row (max|x|/448)"}[base],
            "shortlist": "guard band (exact)" if base == "f16" else f"{rr} * k",
            "recall_at_10_vs_plain": float(agree),
            "recall_at_10_vs_fp64_knn": recall10(r["ids"][:ns], truth),
            "max_rel_score_error_vs_fp64": err,
            "scores_checked": n_scores,
        }
    line = {
        "metric": "recall@10 and score error per dtype; queries/s", "n_gpus": 1, "steps": args.steps,
        "data": "synthetic", "config": workload_desc(cfg),
        "sample": f"first {ns} queries against FP64 brute force over the whole corpus", "dtypes": report,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["lider", "reference"], default="lider")
    ap.add_argument("--workload", default="mid")
    ap.add_argument("--score", choices=list(MODES), default="f16",
                    help="f16 (default), tensor (3xTF32) and simt give the same exact top-k; bf16 is the served "
                         "shortlist form")
    ap.add_argument("--served-rerank", type=int, default=1,
                    help="the main line's served BF16 comparison: shortlist = served_rerank * k")
    ap.add_argument("--recall-nq", type=int, default=1024,
                    help="queries whose recall@10 against FP64 brute force the served comparison measures")
    ap.add_argument("--rerank", type=int, default=None,
                    help="served BF16/FP8 forms: shortlist = rerank * k (default 1; precision workload: 40)")
    ap.add_argument("--serve", type=float, default=None,
                    help="serving mode: offered load in queries/s (Poisson arrivals)")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-max-req", type=int, default=256)
    ap.add_argument("--serve-max-batch", type=int, default=8192)
    ap.add_argument("--serve-slots", type=int, default=3)
    ap.add_argument("--serve-mem-gb", type=int, default=16)
    ap.add_argument("--serve-wait-us", type=float, default=200.0)
    ap.add_argument("--precision", action="store_true",
                    help="per-dtype recall and score error (f16 exact, bf16 and fp8 served forms)")
    ap.add_argument("--precision-sample", type=int, default=16)
    ap.add_argument("--precision-reranks", type=int, nargs="+", default=None,
                    help="--precision: shortlist factors of the served forms (default: --rerank)")
    ap.add_argument("--sweep", action="store_true",
                    help="recall@10 and queries/s over --sweep-W, --sweep-r0 and --sweep-c (FP16 exact mode)")
    ap.add_argument("--sweep-W", type=float, nargs="+", default=[1.0, 2.0])
    ap.add_argument("--sweep-r0", type=int, nargs="+", default=[1, 3, 5])
    ap.add_argument("--sweep-c", type=int, nargs="+", default=[8, 16, 32])
    ap.add_argument("--sweep-nq", type=int, default=10_000)
    ap.add_argument("--sweep-recall-nq", type=int, default=256)
    ap.add_argument("--variants", action="store_true",
                    help="fidelity variants: hyperplane hashkeys, Layer-1 centroids retriever, raw-key RMIs")
    ap.add_argument("--hyper-m", type=int, default=32, help="--variants: bits per hyperplane hashkey")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--clocks-dir", default=None,
                    help="keep the raw nvidia-smi clock samples of the timed region in this directory")
    ap.add_argument("--no-served", action="store_true",
                    help="skip the served BF16 comparison run on the same queries")
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="CPU baseline: seconds of oracle search at least (after --cpu-min-queries)")
    ap.add_argument("--cpu-min-queries", type=int, default=1000,
                    help="CPU baseline: queries the oracle searches at least")
    ap.add_argument("--ref-queries-per-step", type=int, default=8)
    ap.add_argument("--n", type=int, default=None, help="profiling size: first n corpus rows")
    ap.add_argument("--nq", type=int, default=None, help="profiling size: first nq queries")
    ap.add_argument("--sub-batch", type=int, default=None,
                    help="queries per lider_search call (default: the whole batch in one call)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    cfg = configs.get(args.workload)
    if args.n:
        cfg["n"] = min(cfg["n"], args.n)
    if args.nq:
        cfg["nq"] = min(cfg["nq"], args.nq)
    if args.rerank is None:
        args.rerank = cfg.get("rerank", 1)
    if args.impl == "reference":
        return run_reference(args, cfg)
    if args.serve:
        return run_serve(args, cfg)
    if args.sweep:
        return run_sweep(args, cfg)
    if args.precision:
        return run_precision(args, cfg)
    if args.variants:
        return run_variants(args, cfg)
    return run_lider(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
