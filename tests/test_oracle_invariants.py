"""Invariants implied by the definitions, on seeded synthetic populations:
kNN distances non-decreasing, eps-counts symmetric (even total), in-degrees
summing to N*k, subspace monotonicity, and permutation equivariance."""
import numpy as np
import pytest

import oracle
import snaps_inputs


@pytest.fixture(scope="module")
def pop():
    return oracle.normalise(snaps_inputs.population(400, 11))


@pytest.mark.parametrize("mask", [0b11, 0b101010101, (1 << 15) - 1, 0b110000000000011])
def test_basic_invariants(pop, mask):
    k = 10
    r = oracle.subspace(pop, mask, k)
    d2 = r.join.knn_d2
    assert np.all(np.diff(d2, axis=1) >= 0.0)
    assert r.join.eps_count.sum() % 2 == 0
    assert r.scores[oracle.KNN_INDEG].sum() == pop.shape[0] * k
    for i in range(pop.shape[0]):
        assert i not in r.join.knn_idx[i]
        assert len(set(r.join.knn_idx[i].tolist())) == k
    # eps-neighbour mean distance never exceeds eps
    eps = oracle.default_eps(mask)
    assert np.all(r.scores[oracle.EPS_MEAN] <= eps * (1 + 1e-12))
    # the top list starts with a rank-0 object for every metric
    for m in range(4):
        assert r.ranks[m][r.top[m][0]] == 0


def test_subspace_monotonicity(pop):
    # dist_S <= dist_S' for S subset of S': fewer eps-neighbours (same eps)
    # and a larger k-th distance in the superspace
    sub, sup = 0b000100100011, 0b010110100111
    assert sub & sup == sub
    e2 = 0.01
    a = oracle.join(pop, sub, 10, e2)
    b = oracle.join(pop, sup, 10, e2)
    assert np.all(a.eps_count >= b.eps_count)
    assert np.all(a.knn_d2[:, -1] <= b.knn_d2[:, -1])
    assert np.all(a.knn_d2[:, 0] <= b.knn_d2[:, 0])


def test_permutation_equivariance(pop):
    mask = 0b111100001111
    rng = np.random.default_rng(2)
    perm = rng.permutation(pop.shape[0])
    a = oracle.join(pop, mask, 7, 0.02)
    b = oracle.join(pop[perm], mask, 7, 0.02)
    # row perm[q] of the original is row q of the permuted population
    np.testing.assert_array_equal(b.eps_count, a.eps_count[perm])
    np.testing.assert_allclose(b.eps_sum, a.eps_sum[perm], rtol=1e-12)
    inv = np.argsort(perm)
    for q in range(pop.shape[0]):
        assert sorted(perm[b.knn_idx[q]].tolist()) == sorted(a.knn_idx[perm[q]].tolist())


def test_query_subset_matches_full_run(pop):
    mask = 0b1011
    full = oracle.join(pop, mask, 10, 0.005)
    q = np.array([3, 77, 399, 0, 200])
    part = oracle.join(pop, mask, 10, 0.005, queries=q)
    np.testing.assert_array_equal(part.knn_idx, full.knn_idx[q])
    np.testing.assert_array_equal(part.eps_count, full.eps_count[q])
    np.testing.assert_array_equal(part.eps_sum, full.eps_sum[q])
