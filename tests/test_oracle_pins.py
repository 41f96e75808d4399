"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test ties one oracle function to something other than itself: the
paper's worked example, a closed form, a lemma checked by brute force, a
textbook routine, or a hand-computed special case.
"""
import bisect
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import lider_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bits_to_key(s: str) -> int:
    return int(s, 2)


# --- Sec. 4.2 worked example -------------------------------------------------

def test_dist_e_worked_example():
    rows = []
    with open(os.path.join(GOLDEN, "dist_e_worked_example.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    assert len(rows) == 4
    for ka, kb, B, KL, KD, C in rows:
        got = O.dist_e(bits_to_key(ka), bits_to_key(kb), m=6, beta=1, B=int(B))
        assert got == (int(KL), int(KD))
        assert O.dist_e_value(bits_to_key(ka), bits_to_key(kb), 6, 1, int(B)) == \
            int(KL) + int(KD) / int(C)


def test_dist_e_identical_and_padding():
    # identical keys: KL = 0, KD = 0
    assert O.dist_e(0b1011, 0b1011, m=4, beta=1, B=3) == (0, 0)
    # difference in the last element: the B-element window runs past the end
    # and is padded with zeros: Decimal(1,0,0) - Decimal(0,0,0) = 4
    assert O.dist_e(0b0001, 0b0000, m=4, beta=1, B=3) == (1, 4)
    # multi-bit elements (beta = 4): elements (3, 9) vs (3, 2): KL = 1, KD = 7
    assert O.dist_e(0x39, 0x32, m=2, beta=4, B=1) == (1, 7)


# --- Sec. 4.1 hash functions ------------------------------------------------

def test_pstable_hash_hand_values():
    X = np.array([[1.0, 0.0], [0.0, 1.0]], dtype=np.float32)
    A = np.array([[0.75, 0.0], [0.0, -1.25]], dtype=np.float32)
    b = np.array([0.5, 0.25], dtype=np.float32)
    t = O.projections_t(X, A, b, W=0.5)
    # (0.75*1 + 0.5)/0.5 = 2.5 ; (0 + 0.25)/0.5 = 0.5 ; (0 + 0.5)/0.5 = 1.0 ;
    # (-1.25 + 0.25)/0.5 = -2.0
    np.testing.assert_array_equal(t, [[2.5, 0.5], [1.0, -2.0]])
    h, flag = O.hash_values(t)
    np.testing.assert_array_equal(h, [[2, 0], [1, -2]])
    np.testing.assert_array_equal(flag, [[False, False], [True, True]])
    h2, f2 = O.hash_values(np.array([[2.0000004, 2.00001, -0.9999996]]))
    np.testing.assert_array_equal(h2, [[2, 2, -1]])
    np.testing.assert_array_equal(f2, [[True, False, True]])


def _pstable_collision_closed_form(u: float, W: float) -> float:
    """Datar-Immorlica-Indyk-Mirrokni (SoCG 2004), Gaussian (2-stable) case:
    p(u) = 1 - 2*Phi(-W/u) - 2/(sqrt(2 pi) W/u) * (1 - exp(-W^2 / (2 u^2)))."""
    r = W / u
    return 1 - 2 * stats.norm.cdf(-r) - 2 / (math.sqrt(2 * math.pi) * r) * (1 - math.exp(-r * r / 2))


def test_pstable_closed_form_matches_integral():
    # p(u) = int_0^W (1/u) f(t/u) (1 - t/W) dt, f the density of |N(0,1)|
    for u, W in [(0.3, 1.0), (1.0, 1.0), (0.7, 2.5)]:
        f = lambda t: (1 / u) * 2 * stats.norm.pdf(t / u) * (1 - t / W)
        val, _ = integrate.quad(f, 0, W)
        assert abs(val - _pstable_collision_closed_form(u, W)) < 1e-10


def _two_points(d, dist, rng):
    p1 = rng.standard_normal(d)
    v = rng.standard_normal(d)
    v /= np.linalg.norm(v)
    return p1, p1 + dist * v


def test_pstable_collision_probability_and_lemma1():
    """Single-hash collision frequency equals the 2-stable closed form, and the
    common-prefix law of Lemma 1 (Sec. 4.1, eq. dist-and-p_theta) holds with
    p the collision probability: P[KL <= m - l] = p^l."""
    rng = np.random.default_rng(1)
    d, m, N, W = 8, 6, 20000, 1.7
    p1, p2 = _two_points(d, 1.1, rng)
    X = np.stack([p1, p2]).astype(np.float32)
    u = float(np.linalg.norm(X[0].astype(np.float64) - X[1].astype(np.float64)))
    p = _pstable_collision_closed_form(u, W)
    A = rng.standard_normal((N * m, d)).astype(np.float32)
    b = (rng.random(N * m) * W).astype(np.float32)
    t = O.projections_t(X, A, b, W)             # (2, N*m)
    h, _ = O.hash_values(t)
    eq = (h[0] == h[1]).reshape(N, m)
    f1 = eq[:, 0].mean()
    assert abs(f1 - p) < 5 * math.sqrt(p * (1 - p) / N)
    keys, clamped = O.pack_keys(h.reshape(2, N * m), L=N, m=m)
    assert clamped == 0
    beta = O.element_bits(m)
    KL = np.array([O.dist_e(int(keys[0, i]), int(keys[1, i]), m, beta, 1)[0] for i in range(N)])
    for l in range(m + 1):
        freq = np.mean(KL <= m - l)
        pl = p ** l
        assert abs(freq - pl) < 5 * math.sqrt(max(pl * (1 - pl), 1e-12) / N) + 1e-12, (l, freq, pl)


def test_hyperplane_collision_and_lemma1():
    """Hyperplane LSH: P[h(p1) = h(p2)] = 1 - theta/pi (eq. lsh-prob-equal) and
    Lemma 1 with that p."""
    rng = np.random.default_rng(2)
    d, m, N = 8, 6, 20000
    p1, p2 = _two_points(d, 0.9, rng)
    X = np.stack([p1, p2]).astype(np.float32)
    x64 = X.astype(np.float64)
    theta = math.acos(float(x64[0] @ x64[1]) / float(np.linalg.norm(x64[0]) * np.linalg.norm(x64[1])))
    p = 1 - theta / math.pi
    A = rng.standard_normal((N * m, d)).astype(np.float32)
    keys, kf, _ = O.hash_keys(X, A, np.zeros(N * m, np.float32), L=N, m=m, W=1.0,
                              hash_kind=O.HASH_HYPERPLANE)
    KL = np.array([O.dist_e(int(keys[0, i]), int(keys[1, i]), m, 1, 3)[0] for i in range(N)])
    for l in range(m + 1):
        freq = np.mean(KL <= m - l)
        pl = p ** l
        assert abs(freq - pl) < 5 * math.sqrt(max(pl * (1 - pl), 1e-12) / N) + 1e-12, (l, freq, pl)


def test_pack_order_is_lexicographic_tuple_order():
    rng = np.random.default_rng(3)
    for m in (4, 8, 16, 5):
        beta = O.element_bits(m)
        h = rng.integers(-(1 << beta), 1 << beta, size=(300, m))   # includes clamping
        keys, clamped = O.pack_keys(h, L=1, m=m)
        assert clamped > 0
        v = np.clip(h + (1 << (beta - 1)), 0, (1 << beta) - 1)
        tuples = [tuple(int(x) for x in row) for row in v]
        by_tuple = sorted(range(300), key=lambda i: (tuples[i], i))
        by_key = sorted(range(300), key=lambda i: (int(keys[i, 0]), i))
        assert by_tuple == by_key
        # elements read back
        for i in range(0, 300, 37):
            assert O.key_elements(int(keys[i, 0]), m, beta) == list(tuples[i])


# --- Lemmas 2-3: dist_e is monotone away from the query along a sorted array -----

@pytest.mark.parametrize("m,beta,B", [(6, 1, 3), (6, 1, 1), (4, 4, 1), (4, 4, 2), (3, 8, 2)])
def test_lemmas_2_3_monotone(m, beta, B):
    rng = np.random.default_rng(4 + m + B)
    nbits = m * beta
    for trial in range(6):
        # small alphabets to get shared prefixes and duplicates
        elems = rng.integers(0, min(4, 1 << beta), size=(40, m))
        keys = sorted(sum(int(e) << (beta * (m - 1 - j)) for j, e in enumerate(row)) for row in elems)
        for K in keys[::3] + [int(rng.integers(0, 1 << min(nbits, 62)))]:
            p = bisect.bisect_left(keys, K)
            left = [O.dist_e(keys[i], K, m, beta, B) for i in range(p - 1, -1, -1)]
            right = [O.dist_e(keys[i], K, m, beta, B) for i in range(p, len(keys))]
            assert left == sorted(left)
            assert right == sorted(right)
            vals = [O.dist_e_value(keys[i], K, m, beta, B) for i in range(p - 1, -1, -1)]
            assert vals == sorted(vals)


# --- Sec. 5.1 re-scaling -----------------------------------------------------

def test_rescale_endpoints_and_monotone():
    rng = np.random.default_rng(5)
    keys = np.sort(rng.integers(0, 2**63, size=500, dtype=np.int64).astype(np.uint64) * np.uint64(2))
    n = len(keys)
    r = [O.rescale(int(x), int(keys[0]), int(keys[-1]), n) for x in keys]
    assert r[0] == 0.0 and r[-1] == float(n - 1)
    assert all(a <= b for a, b in zip(r, r[1:]))
    assert O.rescale(5, 5, 5, 10) == 0.0
    # a query key below x_min re-scales below 0 (reading R5)
    assert O.rescale(0, 10, 20, 11) == -10.0


# --- Sec. 5.2 RMI ---------------------------------------------------------------

def test_ols_three_points_closed_form():
    a, s = O.ols(np.array([0.0, 1.0, 2.0]), np.array([0.0, 1.0, 3.0]))
    assert abs(s - 1.5) < 1e-15 and abs(a + 1.0 / 6.0) < 1e-15
    a, s = O.ols(np.array([2.0, 2.0]), np.array([4.0, 5.0]))
    assert s == 0.0 and a == 4.5


def test_rmi_exact_linear_data_has_zero_error():
    n = 2**10 + 1
    keys = np.arange(n, dtype=np.uint64) + np.uint64(1000)
    r = np.array([O.rescale(int(x), int(keys[0]), int(keys[-1]), n) for x in keys])
    np.testing.assert_array_equal(r, np.arange(n, dtype=np.float64))
    lb = np.arange(n)
    for F in (1, 8):
        rmi = O.fit_rmi(r, lb, F)
        assert rmi.b0 == 1.0 and rmi.a0 == 0.0
        assert np.all(rmi.e_lo == 0) and np.all(rmi.e_hi == 0)
        assert [rmi.predict(float(i))[1] for i in range(n)] == list(range(n))


def test_rmi_window_invariant_with_duplicates():
    rng = np.random.default_rng(6)
    for trial in range(5):
        n = int(rng.integers(50, 400))
        keys = np.sort(rng.integers(0, 1 << 40, size=n, dtype=np.int64)).astype(np.uint64)
        keys[10:20] = keys[10]  # a run of duplicates
        keys = np.sort(keys)
        r = np.array([O.rescale(int(x), int(keys[0]), int(keys[-1]), n) for x in keys])
        lb = np.searchsorted(keys, keys, side="left")
        for F in (1, 4, 64, 1024):
            rmi = O.fit_rmi(r, lb, F)
            for i in range(n):
                lf, p = rmi.predict(float(r[i]))
                assert 0 <= p <= n - 1
                assert p + rmi.e_lo[lf] <= lb[i] <= p + rmi.e_hi[lf]


def test_rmi_prediction_clamped():
    n = 100
    keys = np.arange(n, dtype=np.uint64) * np.uint64(3)
    r = np.array([O.rescale(int(x), 0, int(keys[-1]), n) for x in keys])
    rmi = O.fit_rmi(r, np.arange(n), 4)
    assert rmi.predict(-1e12)[1] == 0
    assert rmi.predict(1e12)[1] == n - 1


# --- locate and expand ------------------------------------------------------------

def test_lower_bound_matches_bisect():
    rng = np.random.default_rng(7)
    keys = np.sort(rng.integers(0, 50, size=200)).astype(np.uint64)
    for x in list(range(-3, 55)):
        if x < 0:
            continue
        assert O.lower_bound(keys, x) == bisect.bisect_left([int(k) for k in keys], x)
    assert O.lower_bound(np.zeros(0, np.uint64), 5) == 0


def _brute_window(keys, p, qk, R, m, beta, B):
    """Among all windows of length T = min(R, n) that contain position p as a
    boundary, the one with the lexicographically smallest sorted list of
    distances; ties -> leftmost."""
    n = len(keys)
    T = min(R, n)
    best = None
    for s in range(max(0, p - T), min(p, n - T) + 1):
        ds = sorted(O.dist_e(int(keys[i]), qk, m, beta, B) for i in range(s, s + T))
        if best is None or ds < best[0]:
            best = (ds, s)
    return best[1], best[1] + T


def test_expand_equals_brute_force_window():
    rng = np.random.default_rng(8)
    m, beta = 4, 4
    for trial in range(60):
        n = int(rng.integers(1, 30))
        elems = rng.integers(0, 3, size=(n, m))
        keys = np.array(sorted(sum(int(e) << (beta * (m - 1 - j)) for j, e in enumerate(row))
                               for row in elems), dtype=np.uint64)
        qe = rng.integers(0, 3, size=m)
        qk = sum(int(e) << (beta * (m - 1 - j)) for j, e in enumerate(qe))
        p = O.lower_bound(keys, qk)
        for R in (1, 2, 5, 17, 40):
            for B in (1, 2):
                got = O.expand(keys, p, qk, R, m, beta, B)
                assert got == _brute_window(keys, p, qk, R, m, beta, B), (trial, R, B)


def test_expand_exhausted_cluster_returns_all():
    keys = np.array([1, 5, 9], dtype=np.uint64)
    assert O.expand(keys, 1, 4, 10, 4, 4, 1) == (0, 3)
    assert O.expand(np.zeros(0, np.uint64), 0, 4, 10, 4, 4, 1) == (0, 0)


# --- clustering ---------------------------------------------------------------------

def test_route_and_assign_equal_l2_nearest():
    rng = np.random.default_rng(9)
    C = rng.standard_normal((20, 12)).astype(np.float32)
    Q = rng.standard_normal((50, 12)).astype(np.float32)
    rt, near, _ = O.route(Q, C, 5)
    D = ((Q.astype(np.float64)[:, None, :] - C.astype(np.float64)[None]) ** 2).sum(-1)
    for i in range(50):
        order = sorted(range(20), key=lambda j: (D[i, j], j))[:5]
        assert list(rt[i]) == order
    asg, _ = O.assign(Q, C)
    np.testing.assert_array_equal(asg, D.argmin(axis=1))


def test_kmeans_recovers_separated_blob_means():
    rng = np.random.default_rng(10)
    centers = rng.standard_normal((4, 6)) * 10
    lab = np.repeat(np.arange(4), 50)
    X = (centers[lab] + rng.standard_normal((200, 6))).astype(np.float32)
    init = X[[0, 50, 100, 150]]
    C = O.kmeans(X, init, iters=5)
    assert C.dtype == np.float32
    for j in range(4):
        exact = [math.fsum(float(v) for v in X[lab == j][:, i]) / 50 for i in range(6)]
        np.testing.assert_array_equal(C[j], np.float32(exact))


def _exact_lloyd_step(X, C):
    """One Lloyd update written out by hand: nearest centroid by squared L2
    distance (ties to the lower index), exact member sums (math.fsum), mean
    rounded to FP32; an empty cluster keeps its centroid."""
    Xd = X.astype(np.float64)
    out = C.copy()
    lab = []
    for x in Xd:
        dist = [math.fsum((x - c.astype(np.float64)) ** 2) for c in C]
        lab.append(min(range(len(C)), key=lambda j: (dist[j], j)))
    lab = np.array(lab)
    for j in range(len(C)):
        rows = Xd[lab == j]
        if len(rows):
            out[j] = np.float32([math.fsum(rows[:, i]) / len(rows) for i in range(X.shape[1])])
    return out


def test_kmeans_steps_equal_hand_lloyd_updates():
    """Overlapping clusters, three iterations, an initial centroid far away
    (its cluster empties and keeps its place): each iteration equals a
    hand-written Lloyd step."""
    rng = np.random.default_rng(12)
    X = rng.standard_normal((120, 5)).astype(np.float32)
    init = np.concatenate([X[:3], np.full((1, 5), 50.0, np.float32)])
    C = init.copy()
    for it in range(1, 4):
        C = _exact_lloyd_step(X, C)
        np.testing.assert_array_equal(O.kmeans(X, init, iters=it), C)
    np.testing.assert_array_equal(C[3], init[3])


def test_splitmix64_published_sequence():
    """The generator's first outputs from state 0, as published with the
    reference implementation of SplitMix64 (Steele, Lea and Flood, 2014)."""
    assert [O.splitmix64(0, i) for i in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                       0x06C45D188009454F]


def test_forgy_rows_distinct_sorted_and_uniform():
    assert O.forgy_rows(3, 7, 7).tolist() == list(range(7))
    for seed in range(20):
        r = O.forgy_rows(seed, 50, 10)
        assert len(set(r.tolist())) == 10 and np.all(np.diff(r) > 0) and r[0] >= 0 and r[-1] < 50
    # every row is chosen with probability count/n: 4,000 draws of 5 of 20 rows
    counts = np.zeros(20)
    for seed in range(4000):
        counts[O.forgy_rows(seed, 20, 5)] += 1
    p = 5 / 20
    mean, sd = 4000 * p, math.sqrt(4000 * p * (1 - p))
    assert np.all(np.abs(counts - mean) < 5 * sd)


# --- whole search --------------------------------------------------------------------

def _small_problem(seed=11, n=400, d=16, nclu=5):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    Q = rng.standard_normal((12, d)).astype(np.float32)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    C = X[rng.choice(n, nclu, replace=False)]
    L, m = 3, 8
    A = rng.standard_normal((L * m, d)).astype(np.float32)
    b = (rng.random(L * m)).astype(np.float32)
    return X, Q, C, A, b, L, m


def test_search_reduces_to_exact_knn():
    """All clusters probed and R >= cluster size: the search is exhaustive, so
    it must return the brute-force top-k."""
    X, Q, C, A, b, L, m = _small_problem()
    idx = O.build_index(X, C, A, b, L, m, W=1.0, F=4)
    k = 10
    res = O.search(idx, Q, k=k, c=C.shape[0], R=X.shape[0])
    ids, sc = O.exact_knn(X, Q, k)
    np.testing.assert_array_equal(res.ids, ids)
    np.testing.assert_allclose(res.scores, sc, rtol=1e-14, atol=0)  # FP64 summation order only


def test_search_pads_when_candidates_run_out():
    X, Q, C, A, b, L, m = _small_problem(n=30, nclu=3)
    idx = O.build_index(X, C, A, b, L, m, W=1.0, F=2)
    res = O.search(idx, Q, k=40, c=1, R=2)
    for i in range(Q.shape[0]):
        got = res.ids[i]
        nvalid = int(np.sum(got >= 0))
        assert nvalid <= 2 * L
        assert np.all(got[nvalid:] == -1) and np.all(np.isneginf(res.scores[i, nvalid:]))
        assert len(set(got[:nvalid])) == nvalid


def test_exact_knn_matches_full_sort():
    rng = np.random.default_rng(12)
    X = rng.standard_normal((300, 8)).astype(np.float32)
    X[7] = X[3]  # an exact tie
    Q = np.concatenate([rng.standard_normal((5, 8)), X[3:4]]).astype(np.float32)
    ids, sc = O.exact_knn(X, Q, 7)
    S = Q.astype(np.float64) @ X.astype(np.float64).T
    for i in range(Q.shape[0]):
        full = sorted(range(300), key=lambda j: (-S[i, j], j))[:7]
        assert list(ids[i]) == full


def test_core_model_sorted_arrays_and_window_invariant():
    X, Q, C, A, b, L, m = _small_problem(n=600)
    idx = O.build_index(X, C, A, b, L, m, W=0.5, F=8)
    total = 0
    for j in range(C.shape[0]):
        cm = idx.core(j)
        total += len(cm.ids)
        for l in range(L):
            ks, ids = cm.keys[l], cm.sorted_ids[l]
            pairs = list(zip((int(k) for k in ks), (int(i) for i in ids)))
            assert pairs == sorted(pairs)
            assert sorted(int(i) for i in ids) == sorted(int(i) for i in cm.ids)
            n_c = len(ks)
            lb = np.searchsorted(ks, ks, side="left")
            rmi = cm.rmi[l]
            for i in range(n_c):
                r = O.rescale(int(ks[i]), cm.x_min[l], cm.x_max[l], n_c)
                lf, p = rmi.predict(r)
                assert p + rmi.e_lo[lf] <= lb[i] <= p + rmi.e_hi[lf]
    assert total == X.shape[0]
