"""FP64 CPU oracle for LIDER batched query search (arXiv 2205.00970).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. It shares no code with
the CUDA path (``paper_2205_00970_b300``) apart from the seeded input
generators in ``paper_2205_00970_b300.synth``, which hold none of the method's
arithmetic.

Every step follows the paper in its own order and notation, in FP64 (the paper
fixes no precision):

  build (Sec. 3.3.2, Sec. 3.3.1)
    partition      -- each point goes to its nearest k-means centroid
    hash           -- ESK-LSH compound hash G = (h_1..h_m), L(=H) repetitions
                      (Sec. 4.1; p-stable floor((a.x+b)/W) or hyperplane bits)
    pack / sort    -- hashkeys in SK-LSH linear (lexicographic) order (Sec. 4.2)
    re-scale       -- min-max normalisation into [0, n_c-1] (Sec. 5.1, eq. x_norm)
    RMI            -- two layers of linear regression (Sec. 5.2)
  search (Sec. 3.3.1, Sec. 3.3.2, Sec. 6.2)
    route          -- the c_0 nearest centroids
    locate         -- exact lower bound of the query key (plain binary search;
                      the RMI is checked through its error-window invariant)
    expand         -- bi-directional expansion by dist_e (Sec. 4.2, eqs. KD_e,
                      dist_e), R = r_0 * k steps per array, arrays independent
                      (Sec. 4.3)
    verify         -- exact inner-product scores of the union of candidates
    top-k          -- score descending, id ascending

Readings where the paper is silent (numbered as in the design notes):
R2 packing width beta = floor(64/m) bits, offset 2^(beta-1), clamp; R3 the
projections are shared by all clusters; R4 routing by x.mu - |mu|^2/2;
R5 query keys outside [x_min, x_max] re-scale outside [0, n_c-1];
R6 search starts at the exact lower bound; R8 expansion ties go left;
R9 B=1 for p-stable, B=3 for hyperplane; R10 least squares, floor, clamp,
empty leaf copies the root; R11 equal keys ordered by id; R24 k-means starts
from Forgy rows drawn by SplitMix64; R25 k-means stores FP32 centroids.

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BOUNDARY_EPS = 1e-6  # |t - round(t)| below this (in units of W) flags a hash

HASH_PSTABLE = 0
HASH_HYPERPLANE = 1

ROUTE_EXACT = 0   # scan every centroid (Sec. 3.3.2 routing, reading R4)
ROUTE_CORE = 1    # Layer-1 centroids retriever: a core model over the centroids


# ----------------------------------------------------------------------------
# Sec. 4.1 -- LSH functions.  t = (a.x + b) / W; h = floor(t)  (p-stable), or
# h = [a.x >= 0] (hyperplane random projection, eq. lsh-prob-equal).
# ----------------------------------------------------------------------------

def projections_t(X: np.ndarray, A: np.ndarray, b: np.ndarray, W: float,
                  chunk: int = 65536) -> np.ndarray:
    """t[i, j] = (sum_k A[j,k] X[i,k] + b[j]) / W in FP64, shape (n, L*m)."""
    A64 = A.astype(np.float64)
    b64 = b.astype(np.float64)
    out = np.empty((X.shape[0], A.shape[0]), dtype=np.float64)
    for s in range(0, X.shape[0], chunk):
        x64 = X[s:s + chunk].astype(np.float64)
        out[s:s + chunk] = (x64 @ A64.T + b64) / W
    return out


def hash_values(t: np.ndarray, hash_kind: int = HASH_PSTABLE):
    """Hash values h and boundary flags from the projections.

    p-stable: h = floor(t); flagged if t lies within BOUNDARY_EPS of an integer.
    hyperplane: t is taken as a.x (call with b = 0, W = 1); h = 1 if t >= 0;
    flagged if |t| < BOUNDARY_EPS.
    """
    if hash_kind == HASH_PSTABLE:
        h = np.floor(t).astype(np.int64)
        flag = np.abs(t - np.rint(t)) < BOUNDARY_EPS
    else:
        h = (t >= 0).astype(np.int64)
        flag = np.abs(t) < BOUNDARY_EPS
    return h, flag


def element_bits(m: int, hash_kind: int = HASH_PSTABLE) -> int:
    """Bits per hashkey element (reading R2): floor(64/m) for p-stable, 1 for bits."""
    return 1 if hash_kind == HASH_HYPERPLANE else 64 // m


def pack_keys(h: np.ndarray, L: int, m: int, hash_kind: int = HASH_PSTABLE):
    """Pack the m hash values of each array into one sortable integer key.

    Element j (j = 0 is h_1, the most significant, Sec. 4.2) is stored as
    v_j = clamp(h_j + 2^(beta-1), 0, 2^beta - 1) (p-stable) or v_j = h_j (bits),
    and key = sum_j v_j * 2^(beta*(m-1-j)).  Numeric order of keys equals the
    lexicographic order of (v_1..v_m), the SK-LSH linear order.
    Returns keys as a list of L object-free uint64 arrays (n,) and the number
    of clamped values.
    """
    beta = element_bits(m, hash_kind)
    off = 0 if hash_kind == HASH_HYPERPLANE else 1 << (beta - 1)
    vmax = (1 << beta) - 1
    v = h + off
    clamped = int(np.count_nonzero((v < 0) | (v > vmax)))
    v = np.clip(v, 0, vmax).astype(np.uint64)
    n = h.shape[0]
    keys = np.zeros((n, L), dtype=np.uint64)
    for l in range(L):
        for j in range(m):
            keys[:, l] |= v[:, l * m + j] << np.uint64(beta * (m - 1 - j))
    return keys, clamped


def key_flags(hflag: np.ndarray, L: int, m: int) -> np.ndarray:
    """(n, L): True if any of the m hashes of that array is boundary-flagged."""
    return hflag.reshape(hflag.shape[0], L, m).any(axis=2)


# ----------------------------------------------------------------------------
# Sec. 4.2 -- hashkey distance.  dist(K1,K2) = KL + KD/C with KL the non-prefix
# length and KD the first differing element's distance; ESK-LSH's extension
# dist_e uses KD_e = |Decimal(K1[l+1:l+B]) - Decimal(K2[l+1:l+B])| and C = 2^B.
# Compared as the integer pair (KL, KD_e), which orders exactly like dist_e
# because KD_e < C.
# ----------------------------------------------------------------------------

def key_elements(key: int, m: int, beta: int) -> list[int]:
    mask = (1 << beta) - 1
    return [(int(key) >> (beta * (m - 1 - j))) & mask for j in range(m)]


def dist_e(k1: int, k2: int, m: int, beta: int, B: int) -> tuple[int, int]:
    """(KL, KD_e) between two packed hashkeys.

    The B elements after the common prefix are read as one number in radix
    2^beta (for bit elements, beta = 1, this is the paper's Decimal of a binary
    string); positions past the last element count as zeros.
    """
    e1 = key_elements(k1, m, beta)
    e2 = key_elements(k2, m, beta)
    lcp = 0
    while lcp < m and e1[lcp] == e2[lcp]:
        lcp += 1
    KL = m - lcp

    def decimal(e):
        val = 0
        for i in range(lcp, lcp + B):
            val = val * (1 << beta) + (e[i] if i < m else 0)
        return val

    return KL, abs(decimal(e1) - decimal(e2))


def dist_e_value(k1: int, k2: int, m: int, beta: int, B: int) -> float:
    """dist_e as the real number KL + KD_e / C with C = 2^(beta*B)."""
    KL, KD = dist_e(k1, k2, m, beta, B)
    return KL + KD / float(1 << (beta * B))


# ----------------------------------------------------------------------------
# Sec. 5.1 -- key re-scaling: x_norm = (x - x_min)/(x_max - x_min) * (b - a) + a
# with a = 0, b = n_c - 1.  The integer difference is exact; its conversion to
# FP64 rounds to nearest.  Reading R5: a query key below x_min gives r < 0.
# ----------------------------------------------------------------------------

def rescale(x: int, x_min: int, x_max: int, n_c: int, raw: bool = False) -> float:
    """raw: no re-scaling; the key value itself rounded to FP64 (the
    configuration Sec. 7.4 compares against)."""
    if raw:
        return float(int(x))
    if x_max == x_min:
        return 0.0
    return float(int(x) - int(x_min)) / float(int(x_max) - int(x_min)) * float(n_c - 1)


# ----------------------------------------------------------------------------
# Sec. 5.2 -- simplified two-stage RMI of linear models.  The root predicts a
# position; it selects leaf floor(pred * F / n_c) (clamped), whose linear model
# gives the final prediction, floored and clamped to [0, n_c - 1] (Sec. 7.4:
# big predictions truncate to L_array - 1, negative ones to 0).
# ----------------------------------------------------------------------------

def ols(r: np.ndarray, y: np.ndarray) -> tuple[float, float]:
    """Least squares y ~ intercept + slope * r.  Zero variance -> slope 0."""
    rbar = float(np.mean(r))
    ybar = float(np.mean(y))
    if float(np.min(r)) == float(np.max(r)):
        return ybar, 0.0
    dr = r - rbar
    slope = float(np.sum(dr * (y - ybar))) / float(np.sum(dr * dr))
    return ybar - slope * rbar, slope


@dataclass
class RMI:
    n_c: int
    F: int
    a0: float
    b0: float
    a: np.ndarray          # (F,) leaf intercepts
    b: np.ndarray          # (F,) leaf slopes
    e_lo: np.ndarray       # (F,) int64, min(lb - pred) over the leaf's keys
    e_hi: np.ndarray       # (F,) int64, max(lb - pred)

    def leaf(self, r: float) -> int:
        g = math.floor((self.a0 + self.b0 * r) * float(self.F) / float(self.n_c))
        return min(max(g, 0), self.F - 1)

    def predict(self, r: float) -> tuple[int, int]:
        """(leaf, clamped floor prediction)."""
        lf = self.leaf(r)
        p = math.floor(self.a[lf] + self.b[lf] * r)
        return lf, min(max(p, 0), self.n_c - 1)


def fit_rmi(r: np.ndarray, lb: np.ndarray, F: int) -> RMI:
    """Fit the RMI on (r_i, i) pairs of one sorted array; record error windows.

    Labels are positions i (Sec. 3.3.1: a key's location is that of its hashkey
    in the sorted array).  The error window of a leaf is [min, max] of
    lb_i - pred_i over its keys, lb_i being the first position holding key_i
    (duplicates stay local, Sec. 5.1).
    """
    n_c = len(r)
    y = np.arange(n_c, dtype=np.float64)
    a0, b0 = ols(r, y)
    model = RMI(n_c, F, a0, b0, np.full(F, a0), np.full(F, b0),
                np.zeros(F, np.int64), np.zeros(F, np.int64))
    leaf = np.array([model.leaf(float(x)) for x in r], dtype=np.int64)
    for f in range(F):
        sel = np.nonzero(leaf == f)[0]
        if len(sel) == 0:
            continue  # empty leaf keeps the root model (reading R10)
        model.a[f], model.b[f] = ols(r[sel], y[sel])
    for f in range(F):
        sel = np.nonzero(leaf == f)[0]
        if len(sel) == 0:
            continue
        err = [int(lb[i]) - model.predict(float(r[i]))[1] for i in sel]
        model.e_lo[f] = min(err)
        model.e_hi[f] = max(err)
    return model


# ----------------------------------------------------------------------------
# Sorted arrays, lower bound, expansion
# ----------------------------------------------------------------------------

def lower_bound(keys: np.ndarray, x: int) -> int:
    """First position whose key is >= x (plain binary search)."""
    lo, hi = 0, len(keys)
    while lo < hi:
        mid = (lo + hi) // 2
        if int(keys[mid]) < x:
            lo = mid + 1
        else:
            hi = mid
    return lo


def expand(keys: np.ndarray, p: int, qkey: int, R: int, m: int, beta: int, B: int):
    """Bi-directional expansion (Sec. 4, Sec. 4.3): from the query's position p,
    repeatedly take whichever neighbour (left cursor p-1, right cursor p) has
    the smaller dist_e to the query key; ties go left (reading R8).  Stops
    after R picks or when both sides are exhausted (Sec. 7.5: an exhausted
    cluster returns what it has).  Returns the window [s, e) it covered.
    """
    n = len(keys)
    left, right = p - 1, p
    taken = 0
    dl = dist_e(int(keys[left]), qkey, m, beta, B) if left >= 0 else None
    dr = dist_e(int(keys[right]), qkey, m, beta, B) if right < n else None
    while taken < R and (dl is not None or dr is not None):
        if dr is None or (dl is not None and dl <= dr):
            left -= 1
            dl = dist_e(int(keys[left]), qkey, m, beta, B) if left >= 0 else None
        else:
            right += 1
            dr = dist_e(int(keys[right]), qkey, m, beta, B) if right < n else None
        taken += 1
    return left + 1, right


# ----------------------------------------------------------------------------
# Clustering (Sec. 3.2, Sec. 3.3.2): k-means partition and centroid routing.
# Reading R4: nearest centroid = argmax x.mu - |mu|^2/2 (same order as L2).
# ----------------------------------------------------------------------------

def centroid_scores(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    C64 = C.astype(np.float64)
    return X.astype(np.float64) @ C64.T - 0.5 * np.sum(C64 * C64, axis=1)


def assign(X: np.ndarray, C: np.ndarray, chunk: int = 65536):
    """Nearest centroid per point (ties -> smaller index) and near-tie count
    (best two scores within 1e-9 relative)."""
    asg = np.empty(X.shape[0], dtype=np.int64)
    near = 0
    for s in range(0, X.shape[0], chunk):
        S = centroid_scores(X[s:s + chunk], C)
        asg[s:s + chunk] = np.argmax(S, axis=1)
        if S.shape[1] > 1:
            top2 = -np.partition(-S, 1, axis=1)[:, :2]
            near += int(np.count_nonzero(top2[:, 0] - top2[:, 1] <=
                                         1e-9 * np.maximum(1.0, np.abs(top2[:, 0]))))
    return asg, near


# Reading R24: the paper does not say how k-means starts.  Forgy
# initialisation: the initial centroids are `count` distinct rows of the
# training rows, drawn by Floyd's sampling algorithm (Bentley and Floyd, 1987)
# from the counter-based SplitMix64 generator (Steele, Lea and Flood, 2014):
# draw i (from 0) is mix64(seed + (i + 1) * GAMMA mod 2^64), and the integer
# uniform on [0, j] is that draw mod (j + 1).

SPLITMIX_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(seed: int, i: int) -> int:
    """Draw i of the SplitMix64 stream that starts from state `seed`."""
    z = (seed + (i + 1) * SPLITMIX_GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def forgy_rows(seed: int, n: int, count: int) -> np.ndarray:
    """`count` distinct indices of [0, n), ascending (Floyd's algorithm: for
    j = n - count .. n - 1 take t uniform on [0, j]; keep t, or j if t is
    already taken)."""
    if not 0 < count <= n:
        raise ValueError("forgy_rows: need 0 < count <= n")
    chosen: set[int] = set()
    for i, j in enumerate(range(n - count, n)):
        t = splitmix64(seed, i) % (j + 1)
        chosen.add(j if t in chosen else t)
    return np.array(sorted(chosen), dtype=np.int64)


def kmeans(X: np.ndarray, init: np.ndarray, iters: int) -> np.ndarray:
    """Lloyd's k-means from the given initial centroids (Sec. 3.2): `iters`
    rounds of assigning every row to its nearest centroid (FP64 scores) and
    moving each centroid to the mean of its rows.  Reading R25: centroids are
    stored in FP32, as the index keeps them, so each mean is taken in FP64 and
    rounded to FP32.  An emptied cluster keeps its previous centroid.  Returns
    the FP32 centroids."""
    C = init.astype(np.float32).copy()
    X64 = X.astype(np.float64)
    for _ in range(iters):
        asg, _ = assign(X, C)
        for j in range(C.shape[0]):
            sel = asg == j
            if np.any(sel):
                C[j] = X64[sel].mean(axis=0).astype(np.float32)
    return C


def route(Q: np.ndarray, C: np.ndarray, c: int):
    """Top-c centroids per query by score descending, ties -> smaller index.
    Also returns the near-tie flag (c-th and (c+1)-th within 1e-6 relative)."""
    S = centroid_scores(Q, C)
    nq, nclu = S.shape
    out = np.empty((nq, c), dtype=np.int64)
    near = np.zeros(nq, dtype=bool)
    for i in range(nq):
        order = np.lexsort((np.arange(nclu), -S[i]))
        out[i] = order[:c]
        if c < nclu:
            a, b = S[i, order[c - 1]], S[i, order[c]]
            near[i] = abs(a - b) <= 1e-6 * max(abs(a), abs(b), 1e-300)
    return out, near, S


# ----------------------------------------------------------------------------
# Index build and search
# ----------------------------------------------------------------------------

@dataclass
class CoreModel:
    """In-cluster retriever: L sorted hashkey arrays with one RMI each."""
    ids: np.ndarray                  # global ids of the cluster, ascending
    keys: list = field(default_factory=list)     # L x (n_c,) uint64 sorted
    sorted_ids: list = field(default_factory=list)   # L x (n_c,) int64
    flags: list = field(default_factory=list)    # L x (n_c,) bool (boundary)
    x_min: list = field(default_factory=list)
    x_max: list = field(default_factory=list)
    rmi: list = field(default_factory=list)


@dataclass
class Index:
    X: np.ndarray
    C: np.ndarray
    A: np.ndarray
    b: np.ndarray
    L: int
    m: int
    W: float
    F: int
    B: int
    hash_kind: int
    asg: np.ndarray
    asg_near_ties: int
    keys: np.ndarray        # (n, L) uint64
    kflags: np.ndarray      # (n, L) bool
    clamped: int
    cores: dict = field(default_factory=dict)
    raw_keys: bool = False          # RMIs learn raw key values (Sec. 7.4 ablation)
    centroid_model: "CoreModel | None" = None

    @property
    def beta(self) -> int:
        return element_bits(self.m, self.hash_kind)

    def cluster_ids(self, j: int) -> np.ndarray:
        return np.nonzero(self.asg == j)[0]

    def core(self, j: int, fit: bool = True) -> CoreModel:
        cached = self.cores.get(j)
        if cached is None or (fit and any(r is None for r in cached.rmi) and len(cached.ids)):
            self.cores[j] = build_core(self, j, fit)
        return self.cores[j]


def hash_keys(X, A, b, L, m, W, hash_kind=HASH_PSTABLE):
    """Keys (n, L) uint64, key boundary flags (n, L), clamp count."""
    if hash_kind == HASH_PSTABLE:
        t = projections_t(X, A, b, W)
    else:
        t = projections_t(X, A, np.zeros_like(b), 1.0)
    h, hflag = hash_values(t, hash_kind)
    keys, clamped = pack_keys(h, L, m, hash_kind)
    return keys, key_flags(hflag, L, m), clamped


def build_index(X, C, A, b, L, m, W, F, B=None, hash_kind=HASH_PSTABLE, raw_keys=False) -> Index:
    """Partition by nearest centroid, hash every point (projections shared by
    all clusters, reading R3).  Core models are built per cluster on demand."""
    if B is None:
        B = 3 if hash_kind == HASH_HYPERPLANE else 1
    asg, near = assign(X, C)
    keys, kflags, clamped = hash_keys(X, A, b, L, m, W, hash_kind)
    return Index(X, C, A, b, L, m, W, F, B, hash_kind, asg, near, keys, kflags, clamped, raw_keys=raw_keys)


def build_core(index: Index, j: int, fit: bool = True) -> CoreModel:
    """Sort each array by (key, id), re-scale, fit the RMI (Sec. 3.3.1)."""
    ids = index.cluster_ids(j)
    cm = CoreModel(ids=ids)
    for l in range(index.L):
        k = index.keys[ids, l]
        order = np.lexsort((ids, k))
        ks = k[order]
        cm.keys.append(ks)
        cm.sorted_ids.append(ids[order])
        cm.flags.append(index.kflags[ids[order], l])
        n_c = len(ks)
        if n_c == 0:
            cm.x_min.append(0)
            cm.x_max.append(0)
            cm.rmi.append(None)
            continue
        x_min, x_max = int(ks[0]), int(ks[-1])
        cm.x_min.append(x_min)
        cm.x_max.append(x_max)
        if fit:
            r = np.array([rescale(int(x), x_min, x_max, n_c, index.raw_keys) for x in ks])
            lb = np.searchsorted(ks, ks, side="left")
            cm.rmi.append(fit_rmi(r, lb, index.F))
        else:
            cm.rmi.append(None)
    return cm


@dataclass
class SearchResult:
    ids: np.ndarray            # (nq, k) int64, -1 padded
    scores: np.ndarray         # (nq, k) float64, -inf padded
    route: np.ndarray          # (nq, c)
    route_near: np.ndarray     # (nq,) bool
    qkeys: np.ndarray          # (nq, L) uint64
    qflags: np.ndarray         # (nq, L) bool
    pstar: np.ndarray          # (nq, c, L) lower bound in the cluster's array
    wstart: np.ndarray         # (nq, c, L) expansion window start
    wlen: np.ndarray           # (nq, c, L) expansion window length
    ucount: np.ndarray         # (nq, c) unique candidates per probed cluster


def search(index: Index, Q: np.ndarray, k: int, c: int, R: int, route_kind: int = ROUTE_EXACT,
           Rc: int | None = None) -> SearchResult:
    """LIDER batched search (Sec. 3.3.2): route, per probed cluster locate and
    expand on each array, union of candidates, exact scores, top-k.
    route_kind = ROUTE_CORE routes with the Layer-1 centroids retriever,
    expanding Rc positions per array (default r0 * c with r0 = R // k)."""
    nq = Q.shape[0]
    L, m, beta, B = index.L, index.m, index.beta, index.B
    qkeys, qflags, _ = hash_keys(Q, index.A, index.b, L, m, index.W, index.hash_kind)
    if route_kind == ROUTE_CORE:
        rt, near = route_core(index, Q, qkeys, qflags, c, (R // k) * c if Rc is None else Rc)
    else:
        rt, near, _ = route(Q, index.C, c)
    ids_out = np.full((nq, k), -1, dtype=np.int64)
    sc_out = np.full((nq, k), -np.inf)
    pstar = np.zeros((nq, c, L), dtype=np.int64)
    wstart = np.zeros((nq, c, L), dtype=np.int64)
    wlen = np.zeros((nq, c, L), dtype=np.int64)
    ucount = np.zeros((nq, c), dtype=np.int64)
    X = index.X
    for i in range(nq):
        q64 = Q[i].astype(np.float64)
        cand_all = []
        for pi in range(c):
            cm = index.core(int(rt[i, pi]), fit=False)
            cand = set()
            for l in range(L):
                ks = cm.keys[l]
                qk = int(qkeys[i, l])
                p = lower_bound(ks, qk)
                s, e = expand(ks, p, qk, R, m, beta, B)
                pstar[i, pi, l], wstart[i, pi, l], wlen[i, pi, l] = p, s, e - s
                cand.update(int(x) for x in cm.sorted_ids[l][s:e])
            ucount[i, pi] = len(cand)
            cand_all.extend(cand)
        if not cand_all:
            continue
        cid = np.array(sorted(cand_all), dtype=np.int64)
        s = X[cid].astype(np.float64) @ q64
        order = np.lexsort((cid, -s))[:k]
        ids_out[i, :len(order)] = cid[order]
        sc_out[i, :len(order)] = s[order]
    return SearchResult(ids_out, sc_out, rt, near, qkeys, qflags, pstar, wstart, wlen, ucount)


# ----------------------------------------------------------------------------
# Layer-1 centroids retriever (Sec. 3.2; Sec. 3.3.2 "a core model is created
# on the collection of the cluster centroids").  The same ESK-LSH projections
# hash the centroids into L sorted arrays; a query is located (exact lower
# bound) and expanded by Rc positions in each array (for this core model
# k_m = c_0, so Rc = r_0 * c_0, Sec. 6.2), and the
# candidates found are ranked by the routing score of reading R4.
# ----------------------------------------------------------------------------

def centroid_core(index: Index) -> CoreModel:
    """The centroids retriever's sorted arrays (entries are centroid indices,
    equal keys in ascending index order) and the centroids' key flags."""
    if index.centroid_model is None:
        ncl = index.C.shape[0]
        keys, kflags, _ = hash_keys(index.C, index.A, index.b, index.L, index.m, index.W, index.hash_kind)
        ids = np.arange(ncl, dtype=np.int64)
        cm = CoreModel(ids=ids)
        for l in range(index.L):
            order = np.lexsort((ids, keys[:, l]))
            cm.keys.append(keys[order, l])
            cm.sorted_ids.append(ids[order])
            cm.flags.append(kflags[order, l])
        index.centroid_model = cm
    return index.centroid_model


def route_core(index: Index, Q: np.ndarray, qkeys: np.ndarray, qflags: np.ndarray, c: int, Rc: int):
    """Top-c centroids found by the centroids retriever, score descending,
    ties -> smaller index.  Also returns a flag per query: its c-th and
    (c+1)-th candidate scores are within 1e-6 relative, or one of its query
    keys or of the centroid keys lies on a hash boundary (then a correct
    implementation may route it differently)."""
    cm = centroid_core(index)
    any_cflag = any(bool(np.any(f)) for f in cm.flags)
    nq = Q.shape[0]
    out = np.empty((nq, c), dtype=np.int64)
    near = np.zeros(nq, dtype=bool)
    for i in range(nq):
        cand = set()
        for l in range(index.L):
            ks = cm.keys[l]
            qk = int(qkeys[i, l])
            p = lower_bound(ks, qk)
            s, e = expand(ks, p, qk, Rc, index.m, index.beta, index.B)
            cand.update(int(j) for j in cm.sorted_ids[l][s:e])
        cid = np.array(sorted(cand), dtype=np.int64)
        S = centroid_scores(Q[i:i + 1], index.C[cid])[0]
        order = np.lexsort((cid, -S))
        out[i] = cid[order[:c]]
        flag = any_cflag or bool(np.any(qflags[i]))
        if len(cid) > c:
            a, b = S[order[c - 1]], S[order[c]]
            flag = flag or abs(a - b) <= 1e-6 * max(abs(a), abs(b), 1e-300)
        near[i] = flag
    return out, near


# ----------------------------------------------------------------------------
# RMI diagnostics (Sec. 7.4): a prediction is out of range (OOR) when it sits
# at either end of the array (where the clamp of negative and too-large
# predictions lands); it is a large error (LE) when it is more than k
# positions from the true location, the exact lower bound of the query key.
# ----------------------------------------------------------------------------

def rmi_diagnostics(index: Index, qkeys: np.ndarray, route: np.ndarray, k: int) -> tuple[int, int, int]:
    """(N_OOR, N_LE, N_overlap) over every (query, probed cluster, array) of a
    search whose routes are `route` (nq, c); empty clusters are skipped.  The
    RMIs are fitted here (re-scaled keys, or raw ones if index.raw_keys)."""
    n_oor = n_le = n_both = 0
    for i in range(route.shape[0]):
        for j in route[i]:
            cm = index.core(int(j), fit=True)
            for l in range(index.L):
                ks = cm.keys[l]
                n_c = len(ks)
                if n_c == 0:
                    continue
                qk = int(qkeys[i, l])
                r = rescale(qk, cm.x_min[l], cm.x_max[l], n_c, index.raw_keys)
                _, ph = cm.rmi[l].predict(r)
                p = lower_bound(ks, qk)
                oor = ph == 0 or ph == n_c - 1
                le = abs(ph - p) > k
                n_oor += oor
                n_le += le
                n_both += oor and le
    return n_oor, n_le, n_both


def exact_knn(X: np.ndarray, Q: np.ndarray, k: int, chunk: int = 262144):
    """Brute-force top-k by FP64 inner product (the 'Flat' index, Sec. 7.1.2);
    ties -> smaller id."""
    nq = Q.shape[0]
    Q64 = Q.astype(np.float64)
    S = np.empty((nq, X.shape[0]))
    for s in range(0, X.shape[0], chunk):
        S[:, s:s + chunk] = Q64 @ X[s:s + chunk].astype(np.float64).T
    ids = np.empty((nq, k), dtype=np.int64)
    sc = np.empty((nq, k))
    for i in range(nq):
        part = np.argpartition(-S[i], min(k, X.shape[0] - 1))[:k + 1] if X.shape[0] > k else np.arange(X.shape[0])
        kth = np.sort(S[i, part])[::-1][min(k, len(part)) - 1]
        pool = np.nonzero(S[i] >= kth)[0]
        order = pool[np.lexsort((pool, -S[i, pool]))][:k]
        ids[i, :len(order)] = order
        sc[i, :len(order)] = S[i, order]
    return ids, sc


def recall_at(found: np.ndarray, truth: np.ndarray, k: int) -> float:
    """Mean |found[:k] & truth[:k]| / k."""
    hit = 0
    for f, t in zip(found, truth):
        hit += len(set(int(x) for x in f[:k] if x >= 0) & set(int(x) for x in t[:k]))
    return hit / (k * len(truth))
