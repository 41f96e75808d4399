"""Python binding of liblider.so (the C ABI in include/lider.h).

Argument marshalling only: every step of build and search runs in the CUDA
library.  Device buffers are torch CUDA tensors; the stream is torch's current
stream unless one is given.  There is no CPU fallback: if the library cannot
be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblider.so")

LIDER_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ELIMIT", -5: "ETIMEDOUT"}
ETIMEDOUT = -5
MAX_L, MAX_C, MAX_K, MAX_LR, MAX_D = 32, 32, 1024, 4096, 4096
NOALLOC_SCRATCH_BYTES = 64 << 20


class LiderError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


SCORE_TENSOR, SCORE_SIMT, SCORE_BF16, SCORE_F16, SCORE_FP8 = 0, 1, 2, 3, 4
HASH_PSTABLE, HASH_HYPERPLANE = 0, 1
ROUTE_EXACT, ROUTE_CORE = 0, 1


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("m", ctypes.c_int32), ("rmi_leaves", ctypes.c_int32),
                ("r0", ctypes.c_int32), ("B", ctypes.c_int32), ("hash_kind", ctypes.c_int32),
                ("W", ctypes.c_double), ("score_mode", ctypes.c_int32), ("rerank", ctypes.c_int32),
                ("route_kind", ctypes.c_int32), ("raw_keys", ctypes.c_int32)]


class ClusterParams(ctypes.Structure):
    _fields_ = [("n_clusters", ctypes.c_int32), ("kmeans_iters", ctypes.c_int32),
                ("kmeans_sample", ctypes.c_int64), ("seed", ctypes.c_uint64)]


class BuildInfo(ctypes.Structure):
    _fields_ = [("clustered", ctypes.c_int32), ("projections_drawn", ctypes.c_int32),
                ("cluster", ClusterParams), ("train_rows", ctypes.c_int64), ("empty_clusters", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("kmeans_ms", ctypes.c_double), ("build_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        c = self.cluster
        return {"clustered": bool(self.clustered), "projections_drawn": bool(self.projections_drawn),
                "n_clusters": int(c.n_clusters), "kmeans_iters": int(c.kmeans_iters),
                "kmeans_sample": int(c.kmeans_sample), "seed": int(c.seed), "train_rows": int(self.train_rows),
                "empty_clusters": int(self.empty_clusters), "kmeans_ms": float(self.kmeans_ms),
                "build_ms": float(self.build_ms)}


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("n_queries", "pairs", "candidates", "qkey_boundary", "qkey_clamped",
                 "locate_fallback", "empty_pairs", "tc_tiles", "route_fallback", "select_overflow",
                 "rmi_oor", "rmi_le", "rmi_oor_le", "passes")]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class Trace(ctypes.Structure):
    _fields_ = [("route", ctypes.c_void_p), ("qkeys", ctypes.c_void_p), ("pstar", ctypes.c_void_p),
                ("wstart", ctypes.c_void_p), ("wlen", ctypes.c_void_p), ("ucount", ctypes.c_void_p),
                ("events", ctypes.POINTER(ctypes.c_void_p))]

class Tuning(ctypes.Structure):
    _fields_ = [("select_threads", ctypes.c_int32), ("rescore_threads", ctypes.c_int32),
                ("mark_threads", ctypes.c_int32), ("tile_order", ctypes.c_int32), ("probe_batch", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class ServerParams(ctypes.Structure):
    _fields_ = [("c", ctypes.c_int32), ("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("max_k", ctypes.c_int32), ("mem_budget", ctypes.c_int64), ("max_wait_us", ctypes.c_double)]


class ServerCounters(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int64), ("queries", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("refused", ctypes.c_int64), ("failed", ctypes.c_int64), ("max_inflight_batches", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("max_inflight_bytes", ctypes.c_int64), ("launch_s", ctypes.c_double),
                ("finish_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


NUM_PHASES = 8
PHASES = ("hash", "route", "group", "locate", "gather", "score", "select", "merge")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2205_00970_b300.build_lib`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    sig = {
        "lider_build": ([P, I64, I32, ctypes.POINTER(ClusterParams), P, P, ctypes.POINTER(Params), P,
                         ctypes.POINTER(P)], ctypes.c_int),
        "lider_build_centroids": ([P, I64, I32, P, I32, P, P, ctypes.POINTER(Params), P, ctypes.POINTER(P)],
                                  ctypes.c_int),
        "lider_get_build_info": ([P, ctypes.POINTER(BuildInfo)], ctypes.c_int),
        "lider_export_centroids": ([P, P], ctypes.c_int),
        "lider_export_assignment": ([P, P], ctypes.c_int),
        "lider_export_projections": ([P, P, P], ctypes.c_int),
        "lider_search": ([P, P, I64, I32, I32, P, P, ctypes.POINTER(Stats), P], ctypes.c_int),
        "lider_search_trace": ([P, P, I64, I32, I32, P, P, ctypes.POINTER(Trace), ctypes.POINTER(Stats), P],
                               ctypes.c_int),
        "lider_search_host": ([P, P, I64, I32, I32, P, P, ctypes.POINTER(Stats), P], ctypes.c_int),
        "lider_search_noalloc": ([P, P, I64, I32, I32, P, P, ctypes.POINTER(Stats), P], ctypes.c_int),
        "lider_search_scratch_bytes": ([P, I64, I32, I32, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "lider_get_tuning": ([P, ctypes.POINTER(Tuning)], ctypes.c_int),
        "lider_set_tuning": ([P, ctypes.POINTER(Tuning)], ctypes.c_int),
        "lider_autotune": ([P, P, I64, I32, I32, I32, ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_double), P],
                           ctypes.c_int),
        "lider_index_info": ([P, ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I32),
                              ctypes.POINTER(Params)], ctypes.c_int),
        "lider_cluster_offsets": ([P, P], ctypes.c_int),
        "lider_export_array": ([P, I32, I32, P, P], ctypes.c_int),
        "lider_export_rmi": ([P, I32, I32, P, P, P, P], ctypes.c_int),
        "lider_debug_tc_tile": ([P, I32, P, I32, I32, I32, P, P], ctypes.c_int),
        "lider_debug_tc_wait_expiry": ([P, I32, P, I32, I32, I32, P, ctypes.c_double, P], ctypes.c_int),
        "lider_server_create": ([P, ctypes.POINTER(ServerParams), ctypes.POINTER(P)], ctypes.c_int),
        "lider_server_submit": ([P, P, I64, I32, P, P, ctypes.POINTER(I64)], ctypes.c_int),
        "lider_server_wait": ([P, I64, ctypes.c_double], ctypes.c_int),
        "lider_server_stats": ([P, ctypes.POINTER(ServerCounters)], ctypes.c_int),
        "lider_server_latencies": ([P, P, I64, I32, ctypes.POINTER(I64)], ctypes.c_int),
        "lider_server_destroy": ([P], None),
        "lider_free": ([P], None),
        "lider_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def exported_symbols() -> list[str]:
    return [n for n in ("lider_build", "lider_build_centroids", "lider_get_build_info", "lider_export_centroids",
                        "lider_export_assignment", "lider_export_projections", "lider_search", "lider_search_trace", "lider_search_host",
                        "lider_search_noalloc", "lider_search_scratch_bytes", "lider_debug_tc_tile",
                        "lider_debug_tc_wait_expiry",
                        "lider_get_tuning", "lider_set_tuning", "lider_autotune",
                        "lider_index_info", "lider_cluster_offsets", "lider_export_array",
                        "lider_export_rmi", "lider_server_create", "lider_server_submit", "lider_server_wait",
                        "lider_server_stats", "lider_server_latencies", "lider_server_destroy",
                        "lider_free", "lider_last_error") if hasattr(_lib, n)]


def _check(rc: int):
    if rc != LIDER_OK:
        raise LiderError(rc, (_lib.lider_last_error() or b"").decode())


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return t.contiguous()


class Index:
    """A LIDER index resident on the current CUDA device (owns its memory)."""

    def __init__(self, corpus: torch.Tensor, centroids: torch.Tensor | None = None, A: torch.Tensor | None = None,
                 b: torch.Tensor | None = None, *, L: int, m: int, W: float, rmi_leaves: int, r0: int = 2,
                 B: int | None = None, score_mode: int = SCORE_TENSOR, rerank: int = 0,
                 hash_kind: int = HASH_PSTABLE, route_kind: int = ROUTE_EXACT, raw_keys: bool = False,
                 n_clusters: int | None = None, kmeans_iters: int = 10, kmeans_sample: int = 0, seed: int = 0,
                 stream=None):
        """Build the index from an FP32 CUDA corpus (n, d).

        With centroids (n_clusters, d) the index partitions by them
        (lider_build_centroids; A and b required).  Without, lider_build runs
        k-means on the device: n_clusters clusters, kmeans_iters Lloyd
        iterations on the first kmeans_sample rows (0: all) from the Forgy rows
        drawn from `seed`; A (L*m, d) and b (L*m) may then be None, and are
        drawn from `seed`.

        L, m, W, rmi_leaves, r0, B: the core models' parameters (hashkey arrays,
        hashes per key, p-stable bucket width, RMI leaves, expansion factor
        R = r0 * k, elements read by dist_e; B defaults to 1 for p-stable
        hashes and 3 for hyperplane bits).  score_mode: SCORE_F16, SCORE_TENSOR
        or SCORE_SIMT (exact FP32 top-k, equal across the three), SCORE_BF16 or
        SCORE_FP8 (served forms, FP32 re-rank of rerank * k).  hash_kind:
        HASH_PSTABLE or HASH_HYPERPLANE.  route_kind: ROUTE_EXACT (scan every
        centroid) or ROUTE_CORE (the Layer-1 centroids retriever).  raw_keys:
        the RMIs learn raw key values instead of re-scaled ones."""
        if B is None:
            B = 3 if hash_kind == HASH_HYPERPLANE else 1
        corpus = _dev(corpus, torch.float32, "corpus")
        if (A is None) != (b is None):
            raise ValueError("give both A and b, or neither")
        A = None if A is None else _dev(A, torch.float32, "A")
        b = None if b is None else _dev(b, torch.float32, "b")
        n, d = corpus.shape
        p = Params(L, m, rmi_leaves, r0, B, hash_kind, float(W), score_mode, rerank, route_kind, int(raw_keys))
        h = ctypes.c_void_p()
        if centroids is not None:
            centroids = _dev(centroids, torch.float32, "centroids")
            if A is None:
                raise ValueError("a build from given centroids needs A and b")
            _check(_lib.lider_build_centroids(corpus.data_ptr(), n, d, centroids.data_ptr(), centroids.shape[0],
                                              A.data_ptr(), b.data_ptr(), ctypes.byref(p), _stream_ptr(stream),
                                              ctypes.byref(h)))
            n_clusters = int(centroids.shape[0])
        else:
            if n_clusters is None:
                raise ValueError("n_clusters is required when k-means runs in the build")
            cp = ClusterParams(int(n_clusters), int(kmeans_iters), int(kmeans_sample), int(seed))
            _check(_lib.lider_build(corpus.data_ptr(), n, d, ctypes.byref(cp),
                                    None if A is None else A.data_ptr(), None if b is None else b.data_ptr(),
                                    ctypes.byref(p), _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        self.n, self.d, self.n_clusters = int(n), int(d), int(n_clusters)
        self.L, self.m, self.W, self.rmi_leaves, self.r0, self.B = L, m, W, rmi_leaves, r0, B
        self.score_mode = score_mode
        self.rerank = rerank
        self.hash_kind, self.route_kind, self.raw_keys = hash_kind, route_kind, bool(raw_keys)

    def build_info(self) -> dict:
        bi = BuildInfo()
        _check(_lib.lider_get_build_info(self._h, ctypes.byref(bi)))
        return bi.as_dict()

    def centroids(self) -> np.ndarray:
        out = np.zeros((self.n_clusters, self.d), dtype=np.float32)
        _check(_lib.lider_export_centroids(self._h, out.ctypes.data))
        return out

    def assignment(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int32)
        _check(_lib.lider_export_assignment(self._h, out.ctypes.data))
        return out

    def projections(self):
        A = np.zeros((self.L * self.m, self.d), dtype=np.float32)
        b = np.zeros(self.L * self.m, dtype=np.float32)
        _check(_lib.lider_export_projections(self._h, A.ctypes.data, b.ctypes.data))
        return A, b

    @property
    def handle(self) -> int:
        return self._h.value

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lider_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def search(self, Q: torch.Tensor, k: int, c: int, stats: bool = False, trace: bool = False,
               stream=None, out: tuple | None = None):
        """ids (nq, k) int64 and scores (nq, k) float32 on the device.

        With stats=True also returns the counters (the call synchronises);
        with trace=True also returns the per-step outputs as tensors."""
        Q = _dev(Q, torch.float32, "queries")
        nq = Q.shape[0]
        if out is None:
            ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
            sc = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
        else:
            ids, sc = out
        st = Stats()
        sp = ctypes.byref(st) if stats else None
        if trace:
            tr_t = {
                "route": torch.empty((nq, c), dtype=torch.int32, device=Q.device),
                "qkeys": torch.empty((nq, self.L), dtype=torch.int64, device=Q.device),
                "pstar": torch.empty((nq, c, self.L), dtype=torch.int32, device=Q.device),
                "wstart": torch.empty((nq, c, self.L), dtype=torch.int32, device=Q.device),
                "wlen": torch.empty((nq, c, self.L), dtype=torch.int32, device=Q.device),
                "ucount": torch.empty((nq, c), dtype=torch.int32, device=Q.device),
            }
            tr = Trace(*(tr_t[n].data_ptr() for n in ("route", "qkeys", "pstar", "wstart", "wlen", "ucount")), None)
            _check(_lib.lider_search_trace(self._h, Q.data_ptr(), nq, k, c, ids.data_ptr(), sc.data_ptr(),
                                           ctypes.byref(tr), sp, _stream_ptr(stream)))
        else:
            _check(_lib.lider_search(self._h, Q.data_ptr(), nq, k, c, ids.data_ptr(), sc.data_ptr(), sp,
                                     _stream_ptr(stream)))
        res = [ids, sc]
        if stats:
            res.append(st.as_dict())
        if trace:
            res.append(tr_t)
        return tuple(res)

    def search_phased(self, Q: torch.Tensor, k: int, c: int, events, stream=None, out=None):
        """lider_search that records NUM_PHASES + 1 torch.cuda.Events (already
        created, e.g. recorded once) at the phase boundaries on the stream;
        a None entry skips that boundary."""
        Q = _dev(Q, torch.float32, "queries")
        nq = Q.shape[0]
        ids, sc = out if out is not None else (
            torch.empty((nq, k), dtype=torch.int64, device=Q.device),
            torch.empty((nq, k), dtype=torch.float32, device=Q.device))
        handles = [e.cuda_event if e is not None else 0 for e in events]
        if len(handles) != NUM_PHASES + 1 or not all(h for h, e in zip(handles, events) if e is not None):
            raise ValueError(f"search_phased needs {NUM_PHASES + 1} created events or None (record each once first)")
        arr = (ctypes.c_void_p * (NUM_PHASES + 1))(*handles)
        tr = Trace(None, None, None, None, None, None, ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)))
        _check(_lib.lider_search_trace(self._h, Q.data_ptr(), nq, k, c, ids.data_ptr(), sc.data_ptr(),
                                       ctypes.byref(tr), None, _stream_ptr(stream)))
        return ids, sc

    def search_host(self, Q: torch.Tensor, k: int, c: int, ids: torch.Tensor | None = None,
                    scores: torch.Tensor | None = None, stats: bool = False, stream=None):
        """End-to-end search on host tensors (pinned for asynchronous copies)."""
        if Q.is_cuda or Q.dtype != torch.float32 or not Q.is_contiguous():
            raise TypeError("queries must be a contiguous float32 CPU tensor")
        nq = Q.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int64) if ids is None else ids
        scores = torch.empty((nq, k), dtype=torch.float32) if scores is None else scores
        st = Stats()
        _check(_lib.lider_search_host(self._h, Q.data_ptr(), nq, k, c, ids.data_ptr(), scores.data_ptr(),
                                      ctypes.byref(st) if stats else None, _stream_ptr(stream)))
        return (ids, scores, st.as_dict()) if stats else (ids, scores)

    def tuning(self) -> dict:
        t = Tuning()
        _check(_lib.lider_get_tuning(self._h, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, **fields):
        cur = self.tuning()
        cur.update(fields)
        _check(_lib.lider_set_tuning(self._h, ctypes.byref(Tuning(**cur))))

    def autotune(self, Q: torch.Tensor, k: int, c: int, reps: int = 5, stream=None):
        """Pick the kernels' launch shapes by timing searches of Q; returns
        (tuning dict, median ms of one search with it)."""
        Q = _dev(Q, torch.float32, "queries")
        t = Tuning()
        ms = ctypes.c_double()
        _check(_lib.lider_autotune(self._h, Q.data_ptr(), Q.shape[0], k, c, reps, ctypes.byref(t), ctypes.byref(ms),
                                   _stream_ptr(stream)))
        return t.as_dict(), ms.value

    def search_bytes(self, nq: int, k: int, c: int) -> int:
        """Device scratch one search of nq queries takes from the index's pool."""
        b = ctypes.c_size_t()
        _check(_lib.lider_search_scratch_bytes(self._h, nq, k, c, ctypes.byref(b)))
        return int(b.value)

    def cluster_offsets(self) -> np.ndarray:
        off = np.zeros(self.n_clusters + 1, dtype=np.int64)
        _check(_lib.lider_cluster_offsets(self._h, off.ctypes.data))
        return off

    def export_array(self, cluster: int, array: int):
        off = self.cluster_offsets()
        n_c = int(off[cluster + 1] - off[cluster])
        keys = np.zeros(n_c, dtype=np.uint64)
        ids = np.zeros(n_c, dtype=np.int64)
        _check(_lib.lider_export_array(self._h, cluster, array, keys.ctypes.data, ids.ctypes.data))
        return keys, ids

    def export_rmi(self, cluster: int, array: int) -> dict:
        mm = np.zeros(2, dtype=np.uint64)
        root = np.zeros(2, dtype=np.float64)
        leaf = np.zeros(2 * self.rmi_leaves, dtype=np.float64)
        err = np.zeros(2 * self.rmi_leaves, dtype=np.int32)
        _check(_lib.lider_export_rmi(self._h, cluster, array, mm.ctypes.data, root.ctypes.data,
                                     leaf.ctypes.data, err.ctypes.data))
        return {"x_min": int(mm[0]), "x_max": int(mm[1]), "a0": float(root[0]), "b0": float(root[1]),
                "a": leaf[0::2].copy(), "b": leaf[1::2].copy(), "e_lo": err[0::2].astype(np.int64),
                "e_hi": err[1::2].astype(np.int64)}


def tc_tile(A: torch.Tensor, B: torch.Tensor, kind: int = 0, stream=None) -> torch.Tensor:
    """A . B^T through the tensor-core engine (self-test entry); kind 0:
    three TF32 products, kind 1: BF16 operands, kind 2: FP16 operands,
    kind 3: FP8 e4m3 operands (d % 16 == 0)."""
    A = _dev(A, torch.float32, "A")
    B = _dev(B, torch.float32, "B")
    out = torch.empty((A.shape[0], B.shape[0]), dtype=torch.float32, device=A.device)
    _check(_lib.lider_debug_tc_tile(A.data_ptr(), A.shape[0], B.data_ptr(), B.shape[0], A.shape[1], kind,
                                    out.data_ptr(), _stream_ptr(stream)))
    return out


def tc_wait_expiry(A: torch.Tensor, B: torch.Tensor, kind: int = 1, limit_ms: float = 5.0, stream=None) -> int:
    """Run the engine's one-tile self-test with a stage left unloaded and every
    wait limited to limit_ms; returns the C return code (the wait must run out:
    LIDER_ECUDA, message in last_error())."""
    A = _dev(A, torch.float32, "A")
    B = _dev(B, torch.float32, "B")
    out = torch.empty((A.shape[0], B.shape[0]), dtype=torch.float32, device=A.device)
    return _lib.lider_debug_tc_wait_expiry(A.data_ptr(), A.shape[0], B.data_ptr(), B.shape[0], A.shape[1], kind,
                                           out.data_ptr(), float(limit_ms), _stream_ptr(stream))


def raw_call(name: str, *args):
    """Call a C ABI function by name and return its code (tests of argument
    validation use this to pass deliberately invalid arguments)."""
    return getattr(_lib, name)(*args)


def last_error() -> str:
    return (_lib.lider_last_error() or b"").decode()
