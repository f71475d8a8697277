"""Comparison rules between the CUDA library and the FP64 oracle.

The library decides neighbours and radius membership in FP32, the oracle in
FP64, so results may legitimately differ where a candidate's squared distance
lies within a relative band of the k-th distance or of eps^2.  The band is
2e-6 on squared distances (1e-6 on distances); the FP32 fold of <= 15 squared
differences is accurate to about (d + 2) * 2^-24 < 1.1e-6 relative.  Inside
the band the test checks that the library's answer is valid rather than
identical; outside it the answer must be identical.  Floating-point metrics
must agree within 1e-5 relative.
"""
from __future__ import annotations

import numpy as np

import oracle

BAND = 2e-6      # relative, on squared distances
SCORE_RTOL = 1e-5


def exact_d2(x64: np.ndarray, mask: int, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    cols = [c for c in range(x64.shape[1]) if (mask >> c) & 1]
    d = x64[i][..., cols] - x64[j][..., cols]
    return (d * d).sum(axis=-1)


def check_knn(x64, mask, gpu_idx, gpu_dist, ora_idx, ora_d2, queries=None):
    """Rank-wise: the library's p-th neighbour must sit at the oracle's p-th
    distance within the band (identical index outside the band); reported
    distances within SCORE_RTOL.  Returns the number of rows that differ."""
    nq, k = ora_idx.shape
    q = np.arange(nq) if queries is None else np.asarray(queries)
    assert gpu_idx.shape == (nq, k)
    assert np.all(gpu_idx >= 0) and np.all(gpu_idx < x64.shape[0])
    assert np.all(gpu_idx != q[:, None]), "a point is never its own neighbour"
    srt = np.sort(gpu_idx, axis=1)
    assert np.all(srt[:, 1:] != srt[:, :-1]), "neighbours are distinct"
    d2 = exact_d2(x64, mask, np.repeat(q[:, None], k, axis=1), gpu_idx)
    tol = BAND * ora_d2 + 1e-30
    bad = np.abs(d2 - ora_d2) > tol
    assert not bad.any(), (
        f"{bad.sum()} neighbours off the oracle's distance profile, e.g. row "
        f"{np.argwhere(bad)[0]}: gpu d2 {d2[bad][0]!r} vs oracle {ora_d2[bad][0]!r}")
    differ = np.any(gpu_idx != ora_idx, axis=1)
    # a differing index is only allowed where the oracle has another candidate
    # in the band around that rank's distance -- i.e. a near tie
    for r in np.flatnonzero(differ):
        for p in np.flatnonzero(gpu_idx[r] != ora_idx[r]):
            dp = ora_d2[r, p]
            near = np.abs(ora_d2[r] - dp) <= BAND * dp + 1e-30
            near_k = abs(ora_d2[r, k - 1] - dp) <= BAND * dp + 1e-30
            assert near.sum() > 1 or near_k, f"row {r} rank {p}: index differs without a near tie"
    if gpu_dist is not None:
        ref = np.sqrt(ora_d2)
        np.testing.assert_allclose(gpu_dist, ref, rtol=SCORE_RTOL, atol=1e-12)
    return int(differ.sum())


def eps_bounds(x64, mask, eps2, queries=None):
    """Oracle eps counts at the band's two edges."""
    lo = oracle.join(x64, mask, 0, eps2 * (1 - BAND), queries=queries).eps_count
    hi = oracle.join(x64, mask, 0, eps2 * (1 + BAND), queries=queries).eps_count
    return lo, hi


def check_eps(gpu_count, gpu_mean, ora, lo, hi):
    """Counts inside [lo, hi] and equal to the oracle outside the band;
    means within SCORE_RTOL wherever the count is unambiguous."""
    assert np.all(gpu_count >= lo) and np.all(gpu_count <= hi)
    sure = lo == hi
    np.testing.assert_array_equal(gpu_count[sure], ora.eps_count[sure])
    c = ora.eps_count[sure]
    ref = np.where(c > 0, ora.eps_sum[sure] / np.maximum(c, 1), 0.0)
    if gpu_mean is not None:
        np.testing.assert_allclose(gpu_mean[sure], ref, rtol=SCORE_RTOL, atol=1e-12)
    return int((~sure).sum())


def check_top(gpu_top, ora_scores, ora_top, metric):
    """The library's top list must be the oracle's, except that objects whose
    real-valued keys tie within SCORE_RTOL may swap."""
    if np.array_equal(gpu_top, ora_top):
        return 0
    s = ora_scores
    if metric in (oracle.EPS_COUNT, oracle.KNN_INDEG):
        raise AssertionError(f"integer-metric top list differs: {gpu_top[:10]} vs {ora_top[:10]}")
    key = -s[metric]
    if metric == oracle.EPS_MEAN:
        key = np.where(s[oracle.EPS_COUNT] == 0, -np.inf, key)
    gk, ok = key[gpu_top], key[ora_top]
    finite = np.isfinite(gk) & np.isfinite(ok)
    tol = SCORE_RTOL * np.maximum(np.abs(gk), np.abs(ok)) + 1e-12
    diff = np.abs(np.where(finite, gk, 0.0) - np.where(finite, ok, 0.0))
    assert np.all(np.where(finite, diff <= tol, gk == ok)), \
        "top-list keys differ beyond the tolerance"
    return int((gpu_top != ora_top).sum())


NORM_ATOL = 1e-7  # FP32 output of a value in [0, 1]: half an ulp is <= 3e-8


def check_norm(gpu_norm, gpu_scores, ora_scores, ora_norm=None):
    """Normalised metrics (4, n).

    (a) The normalisation step on its own: the library's output must be the
        oracle's FP64 normalisation of the library's own raw metrics, to
        NORM_ATOL.
    (b) End to end against the oracle's FP64 metrics.  Integer metrics whose
        rows agree exactly must agree to NORM_ATOL; mean distances within
        SCORE_RTOL relative move z = (v - lo) / (hi - lo) by at most
        SCORE_RTOL (|v| + 2 |lo| + |hi|) / (hi - lo), which is the tolerance
        (the eps mean distance only where the counts agree, since the counts
        decide which objects take part in its statistics).
    Returns the largest end-to-end error per metric (None where not compared)."""
    g64 = np.asarray(gpu_scores, dtype=np.float64)
    ref = oracle.normalised_scores(g64)
    np.testing.assert_allclose(gpu_norm, ref, rtol=0, atol=NORM_ATOL,
                               err_msg="normalisation of the library's own metrics")
    if ora_norm is None:
        ora_norm = oracle.normalised_scores(ora_scores)
    errs = [None] * 4
    for m in (oracle.EPS_COUNT, oracle.KNN_INDEG):
        if np.array_equal(g64[m], ora_scores[m]):
            np.testing.assert_allclose(gpu_norm[m], ora_norm[m], rtol=0, atol=NORM_ATOL)
            errs[m] = float(np.abs(gpu_norm[m] - ora_norm[m]).max())
    for m in (oracle.EPS_MEAN, oracle.KNN_MEAN):
        if m == oracle.EPS_MEAN and not np.array_equal(g64[oracle.EPS_COUNT], ora_scores[oracle.EPS_COUNT]):
            continue
        v = ora_scores[m]
        use = ora_scores[oracle.EPS_COUNT] > 0 if m == oracle.EPS_MEAN else np.ones(v.size, bool)
        if not use.any():
            continue
        lo, hi = v[use].min(), v[use].max()
        if not hi > lo:
            np.testing.assert_array_equal(gpu_norm[m][use], 0.0)
            continue
        tol = SCORE_RTOL * (np.abs(v) + 2 * abs(lo) + abs(hi)) / (hi - lo) + NORM_ATOL
        d = np.abs(gpu_norm[m] - ora_norm[m])
        assert np.all(d <= tol), f"metric {m}: normalised value off by {d.max():.3g}"
        errs[m] = float(d.max())
    return errs
