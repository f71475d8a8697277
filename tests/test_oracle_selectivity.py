"""Pins of the oracle's selectivity estimate (Sec. 3.5.3) against closed forms
on a lattice, the selectivity definition evaluated by the brute-force join,
and a pure-Python quantile on a tiny case."""
import math

import numpy as np

import oracle
import snaps_inputs


def lattice(n):
    """n objects evenly spaced on feature 0 over [0, 1]; feature 1 constant."""
    x = np.zeros((n, 2))
    x[:, 0] = np.arange(n) / (n - 1)
    x[:, 1] = 0.5
    return x


def lattice_selectivity(n, t):
    """Mean neighbours within t lattice steps, self excluded: object i has
    min(i, t) + min(n - 1 - i, t) of them, summing to 2t(n-1) - t^2 + t."""
    return (2 * t * (n - 1) - t * t + t) / n


def test_sample_rows():
    np.testing.assert_array_equal(oracle.sample_rows(10, 4), [0, 2, 5, 7])
    np.testing.assert_array_equal(oracle.sample_rows(5, 5), [0, 1, 2, 3, 4])
    np.testing.assert_array_equal(oracle.sample_rows(7, 1), [0])


def test_lattice_mean_distance_closed_form():
    # ordered pairs of an n-point lattice: sum |i - j| = n (n - 1) (n + 1) / 3,
    # so the mean distance is (n + 1) / (3 (n - 1))
    for n in (2, 11, 101):
        _, em = oracle.eps_for_selectivity(lattice(n), 0b11, [1.0], n_sample=n, n_bins=10)
        assert math.isclose(em, (n + 1) / (3 * (n - 1)), rel_tol=1e-12)


def test_lattice_radius_brackets_the_exact_step():
    # at target s_t (the selectivity of radius t steps), the estimate is the
    # first bin edge above t h: eps in (t h, t h + w]
    n, n_bins = 101, 1000
    h = 1.0 / (n - 1)
    targets = [lattice_selectivity(n, t) for t in (1, 3, 10, 25)]
    eps, em = oracle.eps_for_selectivity(lattice(n), 0b11, targets, n_sample=n, n_bins=n_bins)
    w = em / n_bins
    for t, e in zip((1, 3, 10, 25), eps):
        assert t * h < e <= t * h + w + 1e-15, (t, e, t * h, w)
    # the closed form itself is the definition's value (brute-force join)
    for t in (1, 3, 10):
        assert math.isclose(oracle.selectivity(lattice(n), 0b11, (t + 0.5) * h),
                            lattice_selectivity(n, t), rel_tol=1e-12)


def test_radius_meets_the_definition_on_the_full_population():
    # with every object sampled, the estimate at the returned radius is the
    # selectivity of Sec. 3.5.3 itself: it reaches the target there and not
    # one bin below
    x = oracle.normalise(snaps_inputs.population(400, 11))
    n = x.shape[0]
    mask = 0b100000100010
    n_bins = 512
    targets = [0.001 * n, 0.15 * n, 3.0, 0.4 * n]
    eps, em = oracle.eps_for_selectivity(x, mask, targets, n_sample=n, n_bins=n_bins)
    w = em / n_bins
    for s, e in zip(targets, eps):
        assert e <= em
        if e < em:
            assert oracle.selectivity(x, mask, e) >= s
        assert oracle.selectivity(x, mask, e - w * (1 + 1e-9)) < s


def test_radius_brackets_the_sample_quantile():
    # the ceil(s m)-th smallest sampled distance q lies in [eps - w, eps)
    rng = np.random.default_rng(4)
    x = rng.random((40, 3))
    m, n_bins = 7, 64
    rows = [int(r) for r in oracle.sample_rows(40, m)]
    dist = sorted(math.dist(x[r], x[j]) for r in rows for j in range(40) if j != r)
    em_exact = sum(dist) / len(dist)
    for s in (0.5, 2.0, 9.0, 17.5):
        eps, em = oracle.eps_for_selectivity(x, 0b111, [s], n_sample=m, n_bins=n_bins)
        assert math.isclose(em, em_exact, rel_tol=1e-12)
        q = dist[math.ceil(s * m) - 1]
        if q < em:
            assert eps[0] - em / n_bins <= q < eps[0]
        else:
            assert eps[0] == em


def test_unreachable_target_and_identical_objects():
    x = oracle.normalise(snaps_inputs.population(200, 2))
    eps, em = oracle.eps_for_selectivity(x, 0b11, [199.0], n_sample=200, n_bins=100)
    assert eps[0] == em   # every other object lies within eps_mean of none
    same = np.full((30, 4), 0.25)
    eps, em = oracle.eps_for_selectivity(same, 0b1111, [1.0, 29.0], n_sample=30, n_bins=16)
    assert em == 0.0 and np.all(eps == 0.0)
