"""The C-ABI library loads and exports every declared entry point; argument
validation answers without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lider.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lider_[a-z_]+)\s*\(", text)))


def test_header_declares_core_abi():
    syms = declared_symbols()
    for s in ("lider_build", "lider_search", "lider_free", "lider_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_2205_00970_b300 import build_lib
    lib = ctypes.CDLL(build_lib.build())
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_loads_and_validates_without_gpu():
    from paper_2205_00970_b300 import lider
    assert set(declared_symbols()) <= set(lider.exported_symbols())
    # NULL out pointer / NULL index are rejected before any CUDA call
    rc = lider.raw_call("lider_build_centroids", None, 10, 8, None, 2, None, None, None, None, None)
    assert rc == -1 and "out is NULL" in lider.last_error()
    rc = lider.raw_call("lider_search", None, None, 0, 10, 1, None, None, None, None)
    assert rc == -1 and "index is NULL" in lider.last_error()
    rc = lider.raw_call("lider_index_info", None, None, None, None, None)
    assert rc == -1
    lider.raw_call("lider_free", None)   # NULL is accepted
    # invalid build arguments are rejected before the device is touched
    out = ctypes.c_void_p()
    p = lider.Params(4, 8, 16, 2, 1, 0, 1.0, 0, 0)
    dummy = ctypes.c_void_p(16)
    for n, d, ncl, pp, msg in [
        (0, 8, 2, p, "n must be"),
        (10, 6, 2, p, "multiple of 4"),
        (10, 8, 0, p, "n_clusters"),
        (10, 8, 2, lider.Params(4, 8, 16, 2, 1, 0, -1.0, 0, 0), "W must be"),
        (10, 8, 2, lider.Params(4, 8, 16, 2, 8, 0, 1.0, 0, 0), "<= 56"),
        (10, 8, 2, lider.Params(4, 8, 16, 2, 1, 7, 1.0, 0, 0), "hash_kind"),
        (10, 8, 2, lider.Params(0, 8, 16, 2, 1, 0, 1.0, 0, 0), ">= 1"),
        (10, 8, 2, lider.Params(4, 8, 16, 2, 1, 0, 1.0, 7, 0), "score_mode"),
        (10, 12, 2, lider.Params(4, 8, 16, 2, 1, 0, 1.0, 2, 0), "d % 8"),
        (10, 8, 2, lider.Params(4, 8, 16, 2, 1, 0, 1.0, 2, 65), "rerank"),
        (10, 8, 2, lider.Params(4, 8, 16, 2, 1, 0, 1.0, 4, 0), "d % 16"),
        (10, 8, 2, lider.Params(4, 8, 16, 2, 1, 0, 1.0, 0, 0, 2, 0), "route_kind"),
        (10, 8, 2, lider.Params(4, 8, 16, 2, 1, 0, 1.0, 0, 0, 0, 2), "raw_keys"),
        (10, 8, 2, lider.Params(4, 65, 16, 2, 1, 1, 1.0, 1, 0), "m must be <= 64"),
    ]:
        rc = lider.raw_call("lider_build_centroids", dummy, n, d, dummy, ncl, dummy, dummy, ctypes.byref(pp), None,
                            ctypes.byref(out))
        assert rc == -1 and msg in lider.last_error(), (msg, lider.last_error())
    rc = lider.raw_call("lider_build_centroids", dummy, 10, 8, dummy, 2, dummy, dummy,
                        ctypes.byref(lider.Params(33, 8, 16, 2, 1, 0, 1.0, 1, 0)), None, ctypes.byref(out))
    assert rc == -4
    rc = lider.raw_call("lider_build_centroids", dummy, 10, 8, dummy, 2, dummy, dummy,
                        ctypes.byref(lider.Params(17, 8, 16, 2, 1, 0, 1.0, 0, 0)), None, ctypes.byref(out))
    assert rc == -4 and "L <= 16" in lider.last_error()
    rc = lider.raw_call("lider_build_centroids", dummy, 10, 8, dummy, 20000, dummy, dummy,
                        ctypes.byref(lider.Params(4, 8, 16, 2, 1, 0, 1.0, 0, 0, 1, 0)), None, ctypes.byref(out))
    assert rc == -4 and "8192" in lider.last_error()
    # hyperplane bits: B is limited by one bit per element, not floor(64/m)
    rc = lider.raw_call("lider_build_centroids", dummy, 10, 8, dummy, 2, dummy, dummy,
                        ctypes.byref(lider.Params(4, 8, 16, 2, 57, 1, 1.0, 0, 0)), None, ctypes.byref(out))
    assert rc == -1 and "<= 56" in lider.last_error()


def test_kmeans_build_validates_without_gpu():
    """lider_build (k-means inside) rejects inconsistent clustering arguments
    before any device work."""
    from paper_2205_00970_b300 import lider
    out = ctypes.c_void_p()
    p = lider.Params(4, 8, 16, 2, 1, 0, 1.0, 0, 0)
    dummy = ctypes.c_void_p(16)
    rc = lider.raw_call("lider_build", dummy, 10, 8, None, None, None, ctypes.byref(p), None, ctypes.byref(out))
    assert rc == -1 and "cluster is NULL" in lider.last_error()
    for cp, A, b, msg in [
        (lider.ClusterParams(20, 5, 0, 0), None, None, "n_clusters exceeds"),
        (lider.ClusterParams(4, 5, 3, 0), None, None, "n_clusters exceeds"),
        (lider.ClusterParams(0, 5, 0, 0), None, None, "n_clusters must be"),
        (lider.ClusterParams(2, -1, 0, 0), None, None, "kmeans_iters"),
        (lider.ClusterParams(2, 5, -4, 0), None, None, "kmeans_sample"),
        (lider.ClusterParams(2, 5, 0, 0), dummy, None, "both A and b"),
    ]:
        rc = lider.raw_call("lider_build", dummy, 10, 8, ctypes.byref(cp), A, b, ctypes.byref(p), None,
                            ctypes.byref(out))
        assert rc == -1 and msg in lider.last_error() and not out.value, (msg, lider.last_error())


def test_tuning_abi_validates_without_gpu():
    import ctypes
    from paper_2205_00970_b300 import lider
    t = lider.Tuning(256, 256, 128, 1)
    assert lider.raw_call("lider_set_tuning", None, ctypes.byref(t)) == -1
    assert lider.raw_call("lider_get_tuning", None, ctypes.byref(t)) == -1
    assert lider.raw_call("lider_autotune", None, None, 1, 10, 1, 1, None, None, None) == -1


def test_header_is_plain_c_and_links(tmp_path):
    """A C99 client (tests/c_abi_check.c) compiles against include/lider.h
    alone with -pedantic, links liblider.so and gets argument errors back
    without touching a GPU."""
    import subprocess
    pkg = os.path.join(ROOT, "paper_2205_00970_b300")
    exe = tmp_path / "c_abi_check"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi_check.c"), "-L", pkg, "-llider",
                        f"-Wl,-rpath,{pkg}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "c abi checks passed" in r.stdout, r.stdout + r.stderr
