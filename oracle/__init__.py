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
  scores; this output is the library's own, defined here in FP64.

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
