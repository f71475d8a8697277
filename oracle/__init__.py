"""FP64 CPU oracle for the SNAPS outlier-detection hot path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library never
imports, links or runs anything here, and this package imports nothing from
the CUDA library.  Inputs come from the shared ``snaps_inputs`` generator.

It follows Gowanlock et al., arXiv 2405.20176:

* :func:`normalise` -- features to [0, 1] (Sec. 3.3), NaN -> column mean
  (Sec. 2.1), rounded to float32 (the canonical input both sides use);
* :func:`join` -- brute-force DSSJ counts / distance sums (Sec. 3.5.1) and
  kNNSJ lists (Sec. 3.6) for one subspace, in C (``snaps_oracle.c``);
* :func:`scores` -- the four per-object metrics of Table 2: eps-neighbour
  count, mean eps-neighbour distance, kNN in-degree, mean kNN distance;
* :func:`ranks` -- the rankings of Sec. 3.4 as Table 2 prints them (dense,
  rank 0 = most outlying);
* :func:`top` -- the first ``n`` objects of each ranking, ties by index;
* :func:`normalised_scores` -- each metric mapped onto [0, 1] with 1 = most
  outlying, from population min / max.  The paper normalises features, not
  scores; this output is the library's own, defined here in FP64;
* :func:`similarity`, :func:`select_index`, :func:`select_eps`,
  :func:`select_k` -- the over-/underfitting parameter selection (Sec. 3.5.2,
  Eq. 2 and 3; Sec. 3.6.2), one full join per grid value;
* :func:`selectivity`, :func:`eps_for_selectivity` -- the selectivity of
  Sec. 3.5.3 by its definition, and the radius at which a sampled distance
  histogram reaches a target selectivity.

Every function states the passage it follows.  Parity: pinned by the Table 2
worked example, closed-form lattices and duplicates, invariants and an
independent brute force (``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snaps_oracle.c")
_SO = os.path.join(_HERE, "libsnaps_oracle.so")
_lib = None

N_SCORES = 4
EPS_COUNT, EPS_MEAN, KNN_INDEG, KNN_MEAN = range(N_SCORES)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) if it is missing or stale."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, u32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_double
        p = ctypes.c_void_p
        lib.snaps_oracle_normalise.argtypes = [p, i64, i32, i32, p]
        lib.snaps_oracle_normalise.restype = i32
        lib.snaps_oracle_join.argtypes = [p, i64, i32, u32, i32, dbl, p, i64, p, p, p, p, i32]
        lib.snaps_oracle_join.restype = i32
        lib.snaps_oracle_threads.argtypes = []
        lib.snaps_oracle_threads.restype = i32
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the oracle's join uses by default."""
    return int(_load().snaps_oracle_threads())


def popcount(mask: int) -> int:
    return bin(int(mask)).count("1")


def default_eps2(mask: int) -> float:
    """Squared default radius for a subspace of d = popcount(mask) features:
    eps = 0.05 * sqrt(d), so eps2 = 0.0025 * d (FP64)."""
    return 0.0025 * popcount(mask)


def normalise(x, nan_to_mean: bool = True) -> np.ndarray:
    """Min-max normalise each column to [0, 1] in FP64 and round to float32
    (Sec. 3.3; NaN -> column mean first, Sec. 2.1)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if x.ndim != 2:
        raise ValueError("x must be 2-D")
    out = np.empty(x.shape, dtype=np.float32)
    rc = _load().snaps_oracle_normalise(x.ctypes.data, x.shape[0], x.shape[1],
                                        1 if nan_to_mean else 0, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle normalise rejected its arguments")
    return out


@dataclass
class JoinResult:
    knn_idx: np.ndarray | None   # (nq, k) int32, nearest first
    knn_d2: np.ndarray | None    # (nq, k) float64 squared distances
    eps_count: np.ndarray | None  # (nq,) int64
    eps_sum: np.ndarray | None   # (nq,) float64, sum of distances


def join(x, mask: int, k: int, eps2: float | None, queries=None, nthreads: int = 0) -> JoinResult:
    """Brute-force DSSJ + kNNSJ of one subspace (Sec. 3.5, 3.6).

    ``x`` is the normalised (n, f) population; it is taken exactly (float32
    values are widened to double without change).  ``k = 0`` skips the kNN
    join, ``eps2 = None`` skips the eps join.  ``queries`` restricts which rows
    are evaluated (each still joined against all n rows)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    n, f = x.shape
    if queries is None:
        nq, qptr = n, None
    else:
        q = np.ascontiguousarray(np.asarray(queries, dtype=np.int64))
        nq, qptr = q.size, q.ctypes.data
    ki = np.zeros((nq, max(k, 0)), dtype=np.int32)
    kd = np.zeros((nq, max(k, 0)), dtype=np.float64)
    ec = np.zeros(nq, dtype=np.int64)
    es = np.zeros(nq, dtype=np.float64)
    e2 = -1.0 if eps2 is None else float(eps2)
    rc = _load().snaps_oracle_join(x.ctypes.data, n, f, int(mask), int(k), e2, qptr, nq,
                                   ki.ctypes.data, kd.ctypes.data, ec.ctypes.data,
                                   es.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError("oracle join rejected its arguments")
    return JoinResult(ki if k > 0 else None, kd if k > 0 else None,
                      ec if eps2 is not None else None, es if eps2 is not None else None)


def scores(res: JoinResult, n: int) -> np.ndarray:
    """The four per-object metrics (Table 2 columns), FP64, shape (4, n).

    0: number of eps-neighbours (DSSJ distance-oblivious, Sec. 3.5.1 item 1);
    1: mean distance to the eps-neighbours, 0 when there are none (item 2;
       Table 2 point 10);
    2: in-degree of the kNN graph, i.e. how many kNN lists hold the object
       (Sec. 3.6.1 item 1);
    3: mean distance to the k nearest neighbours (Sec. 3.6.1 item 2).
    Requires a join over all n queries (the in-degree needs every list)."""
    s = np.zeros((N_SCORES, n), dtype=np.float64)
    c = res.eps_count.astype(np.float64)
    s[EPS_COUNT] = c
    with np.errstate(invalid="ignore", divide="ignore"):
        s[EPS_MEAN] = np.where(c > 0, res.eps_sum / np.where(c > 0, c, 1.0), 0.0)
    s[KNN_INDEG] = np.bincount(res.knn_idx.ravel(), minlength=n).astype(np.float64)
    s[KNN_MEAN] = np.sqrt(res.knn_d2).mean(axis=1)
    return s


def _order_keys(s: np.ndarray):
    """Per-metric sort keys, smallest = most outlying (Sec. 3.4, Table 2):
    counts and in-degrees ascending, mean distances descending, and for the
    eps mean distance every object without eps-neighbours comes first."""
    keys = []
    keys.append((s[EPS_COUNT],))
    zero = (s[EPS_COUNT] == 0)
    keys.append((np.where(zero, 0, 1), np.where(zero, 0.0, -s[EPS_MEAN])))
    keys.append((s[KNN_INDEG],))
    keys.append((-s[KNN_MEAN],))
    return keys


def ranks(s: np.ndarray) -> np.ndarray:
    """Dense rankings (ties share a rank; rank 0 = most outlying), shape (4, n),
    as Table 2 prints them."""
    n = s.shape[1]
    out = np.zeros((N_SCORES, n), dtype=np.int64)
    for m, key in enumerate(_order_keys(s)):
        stacked = np.stack(key, axis=1)
        _, inv = np.unique(stacked, axis=0, return_inverse=True)
        out[m] = inv.ravel()
    return out


def top(s: np.ndarray, count: int = 100) -> np.ndarray:
    """The first ``count`` objects of each ranking, ordered by (rank, index)
    -- equal metric values are taken in index order (Sec. 4.3 keeps 'the first
    1%' of tied objects).  Shape (4, min(count, n)), int32."""
    n = s.shape[1]
    m = min(count, n)
    out = np.zeros((N_SCORES, m), dtype=np.int32)
    idx = np.arange(n)
    for r, key in enumerate(_order_keys(s)):
        order = np.lexsort((idx,) + tuple(reversed(key)))
        out[r] = order[:m]
    return out


def normalised_scores(s: np.ndarray) -> np.ndarray:
    """Each metric mapped onto [0, 1] with 1 = most outlying, in FP64 from the
    population's min and max (a constant metric maps to 0).  Objects without
    eps-neighbours get 1 for the eps mean distance (they rank first); the other
    objects' mean distances are scaled over the objects that have neighbours."""
    out = np.zeros_like(s, dtype=np.float64)

    def scale(v, lo, hi, up):
        span = hi - lo
        if not span > 0.0:
            return np.zeros_like(v)
        return (v - lo) / span if up else (hi - v) / span

    c = s[EPS_COUNT]
    out[EPS_COUNT] = scale(c, c.min(), c.max(), up=False)
    has = c > 0
    if has.any():
        v = s[EPS_MEAN][has]
        out[EPS_MEAN][has] = scale(v, v.min(), v.max(), up=True)
    out[EPS_MEAN][~has] = 1.0
    d = s[KNN_INDEG]
    out[KNN_INDEG] = scale(d, d.min(), d.max(), up=False)
    m = s[KNN_MEAN]
    out[KNN_MEAN] = scale(m, m.min(), m.max(), up=True)
    return out


@dataclass
class SubspaceResult:
    mask: int
    join: JoinResult
    scores: np.ndarray      # (4, n) FP64 metrics
    ranks: np.ndarray       # (4, n) dense ranks
    top: np.ndarray         # (4, min(100, n)) indices
    normalised: np.ndarray  # (4, n) in [0, 1]


def subspace(xn: np.ndarray, mask: int, k: int, eps: float | None = None,
             top_n: int = 100, nthreads: int = 0) -> SubspaceResult:
    """Everything the library reports for one subspace, by the definitions
    above: the join over all queries, the four metrics, ranks, top lists and
    normalised metrics.  ``eps`` defaults to 0.05 * sqrt(d)."""
    eps2 = default_eps2(mask) if eps is None else float(eps) * float(eps)
    res = join(xn, mask, k, eps2, nthreads=nthreads)
    s = scores(res, xn.shape[0])
    return SubspaceResult(int(mask), res, s, ranks(s), top(s, top_n), normalised_scores(s))


def default_eps(mask: int) -> float:
    """eps = 0.05 * sqrt(d) for a d-feature subspace."""
    return 0.05 * math.sqrt(popcount(mask))


# ---- parameter selection (Sec. 3.5.2, Eq. 2 and 3; Sec. 3.6.2) -------------------------------

def similarity(top_a, top_b) -> float:
    """Eq. 2: the fraction f of the n objects of top-n list ``top_a`` that are
    also in top-n list ``top_b`` (both of length n)."""
    n = len(top_a)
    return len(set(int(v) for v in top_a) & set(int(v) for v in top_b)) / n


def select_index(u_min, u_max) -> int:
    """Eq. 3: the grid index j minimising |U^min_j - U^max_j| (the smallest j
    when several minimise it -- the paper does not say; this is the reading)."""
    gap = np.abs(np.asarray(u_min, dtype=np.float64) - np.asarray(u_max, dtype=np.float64))
    return int(np.flatnonzero(gap == gap.min())[0])


def u_curves(tops) -> tuple[np.ndarray, np.ndarray]:
    """U^min and U^max (Sec. 3.5.2) of a grid of top-n lists ordered from the
    smallest to the largest grid value: each list compared with the first and
    with the last."""
    u_min = np.array([similarity(tops[0], t) for t in tops])
    u_max = np.array([similarity(tops[-1], t) for t in tops])
    return u_min, u_max


def eps_grid(eps_min: float, eps_max: float, count: int) -> np.ndarray:
    """``count`` evenly spaced radii over [eps_min, eps_max] (Sec. 3.5.2),
    computed in FP64 and rounded to FP32 (the library's radius precision)."""
    j = np.arange(count, dtype=np.float64)
    return (eps_min + j * (eps_max - eps_min) / (count - 1)).astype(np.float32)


def select_eps(xn: np.ndarray, mask: int, eps_min: float, eps_max: float, count: int, top_n: int):
    """eps selection for one subspace by definition: a full eps-join at every
    grid radius (eps^2 = eps * eps in FP32, as the library squares a given
    radius), the count and mean-distance rankings, their top-n lists, U^min,
    U^max and the selected index.  Returns (u, sel, tops) with u of shape
    (2 metrics, 2, count), sel of shape (2,) and tops of shape (count, 2, top_n)."""
    x64 = np.asarray(xn, dtype=np.float64)
    n = x64.shape[0]
    tops = []
    for e in eps_grid(eps_min, eps_max, count):
        e2 = float(np.float32(e) * np.float32(e))
        res = join(x64, mask, 0, e2)
        s = np.zeros((N_SCORES, n))
        c = res.eps_count.astype(np.float64)
        s[EPS_COUNT] = c
        s[EPS_MEAN] = np.where(c > 0, res.eps_sum / np.where(c > 0, c, 1.0), 0.0)
        tops.append(top(s, top_n)[[EPS_COUNT, EPS_MEAN]])
    tops = np.array(tops)
    u = np.zeros((2, 2, count))
    sel = np.zeros(2, dtype=np.int64)
    for r in range(2):
        u[r, 0], u[r, 1] = u_curves(tops[:, r])
        sel[r] = select_index(u[r, 0], u[r, 1])
    return u, sel, tops


def select_k(xn: np.ndarray, mask: int, k_grid, top_n: int):
    """k selection for one subspace by definition (Sec. 3.6.2): a full kNN join
    at every grid k, the in-degree and mean-distance rankings, their top-n
    lists, U^min, U^max and the selected index.  Returns (u, sel, tops) shaped
    (2, 2, len(k_grid)), (2,), (len(k_grid), 2, top_n)."""
    x64 = np.asarray(xn, dtype=np.float64)
    n = x64.shape[0]
    tops = []
    for kj in k_grid:
        res = join(x64, mask, int(kj), None)
        s = np.zeros((N_SCORES, n))
        s[KNN_INDEG] = np.bincount(res.knn_idx.ravel(), minlength=n).astype(np.float64)
        s[KNN_MEAN] = np.sqrt(res.knn_d2).mean(axis=1)
        tops.append(top(s, top_n)[[KNN_INDEG, KNN_MEAN]])
    tops = np.array(tops)
    u = np.zeros((2, 2, len(k_grid)))
    sel = np.zeros(2, dtype=np.int64)
    for r in range(2):
        u[r, 0], u[r, 1] = u_curves(tops[:, r])
        sel[r] = select_index(u[r, 0], u[r, 1])
    return u, sel, tops


# ---- eps range from selectivity (Sec. 3.5.3) ------------------------------------------------

def selectivity(xn: np.ndarray, mask: int, eps: float) -> float:
    """Sec. 3.5.3: s = (|A| - |D|) / |D|, the mean number of eps-neighbours per
    object with the object itself excluded, from a full eps-join (FP64,
    eps^2 = eps * eps)."""
    res = join(np.asarray(xn, dtype=np.float64), mask, 0, float(eps) * float(eps))
    return float(res.eps_count.mean())


def sample_rows(n: int, m: int) -> np.ndarray:
    """The m sampled objects of the selectivity estimate: original indices
    floor(s n / m), s = 0 .. m - 1 (evenly strided; all objects when m = n)."""
    return (np.arange(m, dtype=np.int64) * n) // m


def sample_distances(xn: np.ndarray, mask: int, n_sample: int) -> tuple[np.ndarray, int]:
    """Distances (FP64) from each of m = min(n_sample, n) sampled objects to
    every other object, concatenated; returns them and m."""
    x64 = np.asarray(xn, dtype=np.float64)
    n = x64.shape[0]
    m = min(int(n_sample), n)
    cols = [f for f in range(x64.shape[1]) if (mask >> f) & 1]
    xs = x64[:, cols]
    out = []
    for s in sample_rows(n, m):
        d = np.sqrt(((xs - xs[s]) ** 2).sum(axis=1))
        out.append(np.delete(d, s))
    return np.concatenate(out), m


def eps_for_selectivity(xn: np.ndarray, mask: int, targets, n_sample: int = 1024, n_bins: int = 4096):
    """Sec. 3.5.3, the sampled estimate of the radius for a selectivity, in the
    steps the paper gives: (1) the distances from a sample of objects to all
    others; (2) their mean eps_mean, the upper bound of a practical radius;
    (3) a histogram of the distances below eps_mean (n_bins bins of width
    w = eps_mean / n_bins, bin floor(d / w)); (4) its cumulative counts, which
    divided by the sample size m give the mean neighbour count at each bin's
    upper edge; (5) for every target, the first edge (b + 1) w at which that
    count reaches the target, eps_mean when none does.  Returns (eps, eps_mean)
    in FP64; all zeros when every distance is 0."""
    d, m = sample_distances(xn, mask, n_sample)
    eps_mean = float(d.mean())
    targets = np.atleast_1d(np.asarray(targets, dtype=np.float64))
    if eps_mean == 0.0:
        return np.zeros(targets.size), 0.0
    w = eps_mean / n_bins
    b = np.floor(d / w).astype(np.int64)
    cum = np.cumsum(np.bincount(b[b < n_bins], minlength=n_bins))
    eps = np.empty(targets.size)
    for t, s in enumerate(targets):
        hit = np.flatnonzero(cum >= s * m)
        eps[t] = (hit[0] + 1) * w if hit.size else eps_mean
    return eps, eps_mean
