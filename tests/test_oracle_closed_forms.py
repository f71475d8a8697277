"""Pin the oracle to closed forms: Eq. 1's subspace count, normalisation of
known columns, lattices (distances h, h*sqrt(2), ... and Gauss-circle counts),
duplicates at distance 0, and the degenerate radii and k."""
import itertools
import math

import numpy as np
import pytest

import oracle
import snaps_inputs


def test_eq1_subspace_count():
    m = snaps_inputs.all_masks(15)
    assert m.size == sum(math.comb(15, i) for i in range(2, 16)) == 32752
    pc = np.array([bin(int(v)).count("1") for v in m])
    assert pc.min() == 2 and pc.max() == 15
    assert np.all(np.diff(m.astype(np.int64)) > 0)
    assert snaps_inputs.pairs_and_full().size == 106


def test_normalise_known_columns():
    x = np.array([[2.0, -1.0, 5.0],
                  [4.0, np.nan, 5.0],
                  [6.0, 3.0, 5.0],
                  [3.0, 1.0, 5.0]])
    z = oracle.normalise(x, nan_to_mean=True)
    assert z.dtype == np.float32
    np.testing.assert_array_equal(z[:, 0], np.float32([0.0, 0.5, 1.0, 0.25]))
    # NaN -> mean of (-1, 3, 1) = 1 -> (1 - -1) / 4 = 0.5
    np.testing.assert_array_equal(z[:, 1], np.float32([0.0, 0.5, 1.0, 0.5]))
    # constant column -> 0
    np.testing.assert_array_equal(z[:, 2], np.float32([0, 0, 0, 0]))
    # rounding: value 1/3 of the span rounds to the nearest float32
    z2 = oracle.normalise(np.array([[0.0], [1.0], [3.0]]))
    assert z2[1, 0] == np.float32(1.0 / 3.0)


def _lattice(m, h, dims=2):
    pts = np.array(list(itertools.product(range(m), repeat=dims)), dtype=np.float64)
    return pts * h, pts.astype(np.int64)


def _ball_count(c, m, r2, dims):
    """Integer points of the m^dims lattice (other than c) within squared
    radius r2 of c, by enumeration of offsets -- independent of the oracle."""
    rad = int(math.isqrt(r2))
    cnt = 0
    for off in itertools.product(range(-rad, rad + 1), repeat=dims):
        if all(o == 0 for o in off):
            continue
        if sum(o * o for o in off) > r2:
            continue
        q = [c[t] + off[t] for t in range(dims)]
        if all(0 <= v < m for v in q):
            cnt += 1
    return cnt


@pytest.mark.parametrize("r2", [1, 2, 4, 5, 8, 9])
def test_lattice_eps_counts_gauss_circle(r2):
    m, h = 12, 0.125  # h = 2^-3: every coordinate and squared distance is exact
    x, ij = _lattice(m, h)
    eps2 = r2 * h * h
    res = oracle.join(x, 0b11, 0, eps2)
    expect = np.array([_ball_count(c, m, r2, 2) for c in ij])
    np.testing.assert_array_equal(res.eps_count, expect)
    # interior points see the full Gauss-circle count N(r) - 1
    interior = {1: 4, 2: 8, 4: 12, 5: 20, 8: 24, 9: 28}[r2]
    c = (m // 2) * m + m // 2
    assert res.eps_count[c] == interior


def test_lattice_knn_distances_and_order():
    m, h = 12, 0.125
    x, ij = _lattice(m, h)
    res = oracle.join(x, 0b11, 8, None)
    for a in range(1, m - 1):
        for b in range(1, m - 1):
            i = a * m + b
            np.testing.assert_array_equal(res.knn_d2[i], [h * h] * 4 + [2 * h * h] * 4)
            axis = sorted([(a - 1) * m + b, a * m + b - 1, a * m + b + 1, (a + 1) * m + b])
            diag = sorted([(a - 1) * m + b - 1, (a - 1) * m + b + 1,
                           (a + 1) * m + b - 1, (a + 1) * m + b + 1])
            assert res.knn_idx[i].tolist() == axis + diag


def test_lattice_3d_eps_counts():
    m, h = 5, 0.25
    x, ij = _lattice(m, h, dims=3)
    for r2 in (1, 2, 3, 4):
        res = oracle.join(x, 0b111, 0, r2 * h * h)
        expect = np.array([_ball_count(c, m, r2, 3) for c in ij])
        np.testing.assert_array_equal(res.eps_count, expect)


def test_projection_makes_duplicates():
    # a 4x4x4 lattice seen in features {0, 1}: every point has 3 exact
    # duplicates (same (a, b), other c) at distance 0, nearest first by index
    m, h = 4, 0.25
    x, ij = _lattice(m, h, dims=3)
    res = oracle.join(x, 0b011, 3, 0.0)
    np.testing.assert_array_equal(res.eps_count, np.full(m ** 3, 3))
    np.testing.assert_array_equal(res.eps_sum, np.zeros(m ** 3))
    for i in range(m ** 3):
        same = [j for j in range(m ** 3) if j != i and ij[j][0] == ij[i][0] and ij[j][1] == ij[i][1]]
        assert res.knn_idx[i].tolist() == same
        assert np.all(res.knn_d2[i] == 0.0)


def test_duplicates_come_first_in_index_order():
    rng = np.random.default_rng(3)
    x = rng.random((50, 4))
    dup_rows = [7, 19, 33, 41]
    for r in dup_rows[1:]:
        x[r] = x[dup_rows[0]]
    res = oracle.join(x, 0b1111, 5, None)
    for r in dup_rows:
        others = [d for d in dup_rows if d != r]
        assert res.knn_idx[r][:3].tolist() == others
        assert np.all(res.knn_d2[r][:3] == 0.0)
        assert res.knn_d2[r][3] > 0.0


def test_eps_beyond_diameter_counts_everyone():
    x = snaps_inputs.population(200, 4)
    xn = oracle.normalise(x)
    d = 15
    res = oracle.join(xn, (1 << d) - 1, 0, float(d) + 1e-9)   # eps = sqrt(d) = diameter of [0,1]^d
    np.testing.assert_array_equal(res.eps_count, np.full(200, 199))


def test_eps_below_min_distance_counts_nobody():
    x = snaps_inputs.population(200, 5)
    xn = oracle.normalise(x)
    r = oracle.subspace(xn, 0b111, 4, eps=1e-7)
    assert np.all(r.join.eps_count == 0)
    assert np.all(r.scores[oracle.EPS_MEAN] == 0.0)
    assert np.all(r.ranks[oracle.EPS_MEAN] == 0)
    assert np.all(r.ranks[oracle.EPS_COUNT] == 0)
    np.testing.assert_array_equal(r.top[oracle.EPS_COUNT], np.arange(100))


def test_k_all_others_gives_full_in_degree():
    x = snaps_inputs.population(60, 6)
    xn = oracle.normalise(x)
    r = oracle.subspace(xn, 0b1010101, 59)
    np.testing.assert_array_equal(r.scores[oracle.KNN_INDEG], np.full(60, 59))
    # every row holds all the other rows
    for i in range(60):
        assert sorted(r.join.knn_idx[i].tolist()) == [j for j in range(60) if j != i]


def test_bad_arguments_are_rejected():
    x = np.zeros((5, 3))
    with pytest.raises(ValueError):
        oracle.join(x, 0b1000, 1, None)      # bit beyond f
    with pytest.raises(ValueError):
        oracle.join(x, 0b11, 5, None)        # k > n - 1
