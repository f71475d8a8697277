"""Pin the oracle's join against a second, independent brute force written
with whole-matrix NumPy operations (full distance matrix, lexicographic sort)
on small populations."""
import numpy as np
import pytest

import oracle
import snaps_inputs


def _numpy_join(x, mask, k, eps2):
    cols = [c for c in range(x.shape[1]) if (mask >> c) & 1]
    y = x[:, cols].astype(np.float64)
    d2 = ((y[:, None, :] - y[None, :, :]) ** 2).sum(axis=-1)
    n = x.shape[0]
    idx = np.arange(n)
    knn = np.zeros((n, k), dtype=np.int64)
    kd = np.zeros((n, k))
    for i in range(n):
        row = d2[i].copy()
        row[i] = np.inf
        order = np.lexsort((idx, row))[:k]
        knn[i], kd[i] = order, row[order]
    near = (d2 <= eps2) & ~np.eye(n, dtype=bool)
    cnt = near.sum(axis=1)
    sm = np.where(near, np.sqrt(d2), 0.0).sum(axis=1)
    return knn, kd, cnt, sm


@pytest.mark.parametrize("seed,n,mask,k", [
    (0, 300, (1 << 15) - 1, 10),
    (1, 257, 0b11, 10),
    (2, 150, 0b100000000000001, 5),
    (3, 64, 0b011011011011011, 20),
    (4, 33, 0b111, 32),
])
def test_join_matches_numpy_brute_force(seed, n, mask, k):
    x = oracle.normalise(snaps_inputs.population(n, seed))
    eps2 = oracle.default_eps2(mask)
    ref_knn, ref_d2, ref_cnt, ref_sum = _numpy_join(x, mask, k, eps2)
    got = oracle.join(x, mask, k, eps2)
    np.testing.assert_array_equal(got.knn_idx, ref_knn)
    np.testing.assert_allclose(got.knn_d2, ref_d2, rtol=1e-12, atol=0)
    np.testing.assert_array_equal(got.eps_count, ref_cnt)
    np.testing.assert_allclose(got.eps_sum, ref_sum, rtol=1e-12, atol=1e-15)


def test_integer_grid_ties_match_numpy():
    # coarse integer coordinates force many exact distance ties
    rng = np.random.default_rng(9)
    x = rng.integers(0, 4, size=(120, 3)).astype(np.float64)
    ref_knn, ref_d2, ref_cnt, ref_sum = _numpy_join(x, 0b111, 12, 2.0)
    got = oracle.join(x, 0b111, 12, 2.0)
    np.testing.assert_array_equal(got.knn_idx, ref_knn)
    np.testing.assert_array_equal(got.knn_d2, ref_d2)
    np.testing.assert_array_equal(got.eps_count, ref_cnt)
