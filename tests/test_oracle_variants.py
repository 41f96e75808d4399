"""Pins of the oracle's fidelity variants: the Layer-1 centroids retriever
(Sec. 3.2), hyperplane hashkeys (Sec. 4.1) and the RMI diagnostics of
Sec. 7.4 (with and without key re-scaling).

Each test ties the oracle to something other than itself: a special case
that reduces to the exact routing scan, a brute-force union of windows, a
hand-packed key, or a least-squares line from numpy.polyfit.
"""
import numpy as np

from oracle import lider_oracle as O


def _problem(seed=21, n=500, d=16, nclu=24, nq=15, L=3, m=8):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    Q = rng.standard_normal((nq, d)).astype(np.float32)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    C = X[rng.choice(n, nclu, replace=False)] * 0.9
    A = rng.standard_normal((L * m, d)).astype(np.float32)
    b = rng.random(L * m).astype(np.float32)
    return X, Q, C, A, b, L, m


# --- Layer-1 centroids retriever ---------------------------------------------

def test_route_core_with_covering_windows_is_the_exact_scan():
    """When each window spans every centroid (Rc >= n_clusters), the
    centroids retriever scores all of them: its route is the exact scan's."""
    for hk in (O.HASH_PSTABLE, O.HASH_HYPERPLANE):
        X, Q, C, A, b, L, m = _problem()
        idx = O.build_index(X, C, A, b, L, m, W=1.0, F=4, hash_kind=hk)
        qk, qf, _ = O.hash_keys(Q, A, b, L, m, 1.0, hk)
        for c in (1, 3, 7):
            got, _ = O.route_core(idx, Q, qk, qf, c, Rc=C.shape[0])
            ref, _, _ = O.route(Q, C, c)
            np.testing.assert_array_equal(got, ref)


def test_route_core_equals_brute_force_union():
    """Small Rc: the route is the c best (FP64 score, ties to the lower index)
    of the union of the L windows, each window being the R picks nearest the
    query key by dist_e found by brute force over the sorted centroid keys."""
    X, Q, C, A, b, L, m = _problem(seed=5)
    idx = O.build_index(X, C, A, b, L, m, W=0.7, F=4)
    qk, qf, _ = O.hash_keys(Q, A, b, L, m, 0.7)
    ck, _, _ = O.hash_keys(C, A, b, L, m, 0.7)
    beta = O.element_bits(m)
    c, Rc = 3, 4
    got, _ = O.route_core(idx, Q, qk, qf, c, Rc)
    ids = np.arange(C.shape[0])
    for i in range(Q.shape[0]):
        cand = set()
        for l in range(L):
            order = sorted(ids, key=lambda j: (int(ck[j, l]), j))
            keys = [int(ck[j, l]) for j in order]
            p = sum(1 for x in keys if x < int(qk[i, l]))            # lower bound
            # greedy merge of the two runs, ties to the left
            left, right, picks = p - 1, p, []
            while len(picks) < Rc and (left >= 0 or right < len(keys)):
                dl = O.dist_e(keys[left], int(qk[i, l]), m, beta, 1) if left >= 0 else None
                dr = O.dist_e(keys[right], int(qk[i, l]), m, beta, 1) if right < len(keys) else None
                if dr is None or (dl is not None and dl <= dr):
                    picks.append(order[left]); left -= 1
                else:
                    picks.append(order[right]); right += 1
            cand.update(int(j) for j in picks)
        sc = {j: float(sum(float(Q[i, t]) * float(C[j, t]) for t in range(C.shape[1]))
                       - 0.5 * sum(float(C[j, t]) ** 2 for t in range(C.shape[1]))) for j in cand}
        best = sorted(cand, key=lambda j: (-sc[j], j))[:c]
        assert list(got[i]) == best, (i, list(got[i]), best)


def test_search_with_core_route_probes_the_core_route():
    X, Q, C, A, b, L, m = _problem(seed=9)
    idx = O.build_index(X, C, A, b, L, m, W=1.0, F=4)
    res = O.search(idx, Q, k=5, c=2, R=10, route_kind=O.ROUTE_CORE)
    qk, qf, _ = O.hash_keys(Q, A, b, L, m, 1.0)
    rt, _ = O.route_core(idx, Q, qk, qf, 2, Rc=(10 // 5) * 2)
    np.testing.assert_array_equal(res.route, rt)
    for i in range(Q.shape[0]):            # every result lies in a probed cluster
        got = res.ids[i][res.ids[i] >= 0]
        assert set(idx.asg[got].tolist()) <= set(rt[i].tolist())


# --- hyperplane hashkeys -------------------------------------------------------

def test_hyperplane_keys_by_hand():
    """h = [a.x >= 0] (zero counts as positive), one bit per hash, h_1 most
    significant; b and W play no part."""
    A = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [1.0, 1.0]], dtype=np.float32)
    X = np.array([[2.0, -1.0], [0.0, 0.0], [-1.0, 3.0]], dtype=np.float32)
    keys, flags, clamped = O.hash_keys(X, A, np.full(4, 0.5, np.float32), L=1, m=4, W=3.0,
                                       hash_kind=O.HASH_HYPERPLANE)
    assert [int(k) for k in keys[:, 0]] == [0b1001, 0b1111, 0b0111]
    assert clamped == 0
    assert list(flags[:, 0]) == [False, True, False]       # x = 0 sits on every hyperplane


# --- RMI diagnostics (Sec. 7.4) ---------------------------------------------------

def _one_cluster_index(keys: np.ndarray, F: int, raw: bool) -> O.Index:
    n = len(keys)
    z = np.zeros((n, 1), np.float32)
    return O.Index(X=z, C=np.zeros((1, 1), np.float32), A=np.zeros((1, 1), np.float32),
                   b=np.zeros(1, np.float32), L=1, m=16, W=1.0, F=F, B=1, hash_kind=O.HASH_PSTABLE,
                   asg=np.zeros(n, np.int64), asg_near_ties=0, keys=keys.reshape(n, 1),
                   kflags=np.zeros((n, 1), bool), clamped=0, raw_keys=raw)


def test_rmi_diagnostics_uniform_keys():
    """Evenly spaced keys: the RMI is exact, so no prediction is a large
    error; the out-of-range ones are the two end keys and two queries outside
    [x_min, x_max] (clamped to the ends), with and without re-scaling."""
    n = 2**8 + 1
    keys = np.arange(n, dtype=np.uint64) + np.uint64(1000)
    q = np.concatenate([keys, np.array([5, 10**6], np.uint64)]).reshape(-1, 1)
    for raw in (False, True):
        idx = _one_cluster_index(keys, F=4, raw=raw)
        route = np.zeros((len(q), 1), np.int64)
        assert O.rmi_diagnostics(idx, q, route, k=1) == (4, 0, 0)


def test_rmi_diagnostics_match_polyfit_line():
    """Two clumps of keys and a single leaf: the RMI is one least-squares line
    of position on (re-scaled or raw) key, here taken from numpy.polyfit; OOR,
    LE and their overlap follow from its clamped floor predictions."""
    rng = np.random.default_rng(3)
    keys = np.sort(np.concatenate([rng.integers(0, 400, 120), rng.integers(10**6, 10**6 + 400, 80)])).astype(np.uint64)
    qs = np.sort(rng.integers(0, 10**6 + 900, 300)).astype(np.uint64)
    n, k = len(keys), 10
    for raw in (False, True):
        idx = _one_cluster_index(keys, F=1, raw=raw)
        x0, x1 = float(keys[0]), float(keys[-1])
        to_r = (lambda x: float(x)) if raw else (lambda x: (float(x) - x0) / (x1 - x0) * (n - 1))
        slope, icpt = np.polyfit(np.array([to_r(x) for x in keys]), np.arange(n, dtype=np.float64), 1)
        # queries whose line value is too close to an integer to call against polyfit are left out
        kept = np.array([x for x in qs if abs(icpt + slope * to_r(x) - round(icpt + slope * to_r(x))) > 1e-6],
                        np.uint64)
        exp = [0, 0, 0]
        for x in kept:
            ph = min(max(int(np.floor(icpt + slope * to_r(x))), 0), n - 1)
            p = int(np.searchsorted(keys, x, side="left"))
            oor, le = ph in (0, n - 1), abs(ph - p) > k
            exp[0] += oor; exp[1] += le; exp[2] += oor and le
        got = O.rmi_diagnostics(idx, kept.reshape(-1, 1), np.zeros((len(kept), 1), np.int64), k)
        assert got == tuple(exp), (raw, got, exp)
        assert got[1] > 100                                # the clumps defeat a single line


# --- L = 1, c = 1: one SK-LSH core model ------------------------------------------

def test_single_array_single_cluster_is_one_core_model():
    """With one hashkey array and one probed cluster the search is a single
    SK-LSH core model: a query's candidates are exactly the ids of its one
    expansion window (no union to take), and its top-k is the best of them by
    FP64 score, ties to the lower id."""
    X, Q, C, A, b, _, m = _problem(seed=13, n=800, nclu=4, L=1)
    idx = O.build_index(X, C, A[:m], b[:m], 1, m, W=0.8, F=8)
    k, R = 7, 25
    res = O.search(idx, Q, k=k, c=1, R=R)
    for i in range(Q.shape[0]):
        j = int(res.route[i, 0])
        cm = idx.core(j, fit=False)
        s, ln = int(res.wstart[i, 0, 0]), int(res.wlen[i, 0, 0])
        window = [int(x) for x in cm.sorted_ids[0][s:s + ln]]
        assert ln == min(R, len(cm.ids)) and res.ucount[i, 0] == len(set(window)) == ln
        sc = {x: float(np.dot(X[x].astype(np.float64), Q[i].astype(np.float64))) for x in window}
        best = sorted(window, key=lambda x: (-sc[x], x))[:k]
        assert list(res.ids[i][:len(best)]) == best
