"""The seeded population generator follows its stated recipe: fixed bytes per
(n, seed), 15 float32 columns on [0, 1], the per-family shapes (symmetric
normal, right-skewed lognormal and Beta(2, 5), a bimodal mixture), and 0.5 %
of the rows replaced by uniform outliers.  Also the subspace lists: Eq. 1's
count, and the 105 pairs plus the full subspace."""
import numpy as np

import snaps_inputs


def test_same_seed_same_bytes_other_seed_other_bytes():
    a = snaps_inputs.population(3000, 4)
    b = snaps_inputs.population(3000, 4)
    c = snaps_inputs.population(3000, 5)
    assert a.dtype == np.float32 and a.shape == (3000, 15) and a.flags.c_contiguous
    assert a.tobytes() == b.tobytes()
    assert a.tobytes() != c.tobytes()


def test_columns_span_the_unit_interval():
    x = snaps_inputs.population(20000, 0)
    assert np.all(x >= 0.0) and np.all(x <= 1.0)
    # each column's own sample range maps onto [0, 1] (outliers are drawn inside it)
    assert np.all(x.min(axis=0) <= 0.01) and np.all(x.max(axis=0) >= 0.99)


def _skew(v):
    v = v.astype(np.float64)
    return float(np.mean((v - v.mean()) ** 3) / v.std() ** 3)


def test_feature_families_have_their_shapes():
    x = snaps_inputs.population(100000, 1)
    normal, lognormal, beta, mix = x[:, 0:5], x[:, 5:9], x[:, 9:12], x[:, 12:15]
    assert all(abs(_skew(normal[:, j])) < 0.1 for j in range(5))
    # LogNormal(0, 0.5) has skewness about 1.75; Beta(2, 5) about 0.6
    assert all(_skew(lognormal[:, j]) > 1.2 for j in range(4))
    assert all(0.4 < _skew(beta[:, j]) < 0.8 for j in range(3))
    for j in range(3):
        h, _ = np.histogram(mix[:, j], bins=20, range=(0, 1))
        lo_mode, hi_mode, valley = h[4:8].max(), h[12:16].max(), h[9:11].min()
        assert valley < 0.2 * min(lo_mode, hi_mode), "the mixture columns are bimodal"
        assert lo_mode > hi_mode, "the 0.6-weight component is the larger mode"


def test_outlier_fraction():
    n = 200000
    x = snaps_inputs.population(n, 2).astype(np.float64)
    # uniform outliers sit far from the normal columns' centre far more often than
    # the normal rows do: count rows whose five normal-family features are all
    # beyond 0.25 of the column centre, which a Normal(0.5, 0.12) row almost never is
    c = np.median(x[:, 0:5], axis=0)
    far = np.all(np.abs(x[:, 0:5] - c) > 0.25, axis=1)
    # a uniform value is beyond 0.25 of the centre with probability 1/2 per feature
    expect = snaps_inputs.OUTLIER_FRACTION * n * 0.5 ** 5
    assert 0.5 * expect < far.sum() < 2.0 * expect


def test_subspace_lists():
    m = snaps_inputs.all_masks()
    assert m.size == 2 ** 15 - 1 - 15 == 32752  # Eq. 1: subsets of 2..15 of 15 features
    assert np.all(np.diff(m.astype(np.int64)) > 0)
    pc = np.array([bin(int(v)).count("1") for v in m])
    assert pc.min() == 2 and pc.max() == 15
    pf = snaps_inputs.pairs_and_full()
    assert pf.size == 106 and int(pf[-1]) == (1 << 15) - 1
    s = snaps_inputs.mask_sample(64, 1)
    assert s.size == 64 and np.all(np.isin(s, m)) and np.unique(s).size == 64


def test_chunk_sample_is_whole_chunks():
    m = snaps_inputs.chunk_sample(8, 1)
    assert m.dtype == np.uint16 and m.size == 8 * 32
    assert np.all(np.diff(m.astype(np.int64)) > 0)  # ascending, distinct
    highs = np.unique(m >> 5)
    assert highs.size == 8
    for h in highs:
        assert bin(int(h)).count("1") >= 2
        np.testing.assert_array_equal(m[(m >> 5) == h] & 31, np.arange(32))
    # every mask is a valid subspace of 2..15 features
    assert all(2 <= bin(int(v)).count("1") <= 15 for v in m)
    np.testing.assert_array_equal(snaps_inputs.chunk_sample(8, 1), m)
