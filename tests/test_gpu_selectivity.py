"""The eps range from selectivity (snaps_eps_selectivity; Sec. 3.5.3) through
the C ABI against the FP64 oracle: the same eps_mean (to the rounding of
FP32 distances) and the same bin edge for every target, give or take one bin
where an FP32 distance falls on the other side of an edge; and the invalid
requests it must reject."""
import numpy as np
import pytest

import oracle
import paper_2405_20176_b300 as snaps
import snaps_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = snaps.snaps_create(0)
    yield c
    snaps.snaps_destroy(c)


def check_against_oracle(xn, masks, targets, eps, em, n_sample, n_bins):
    for s, m in enumerate(masks):
        e_or, em_or = oracle.eps_for_selectivity(xn, int(m), targets, n_sample, n_bins)
        np.testing.assert_allclose(em[s], em_or, rtol=1e-5, err_msg=f"eps_mean, mask {int(m):#x}")
        w = em_or / n_bins
        # bin indices: exact except where a target sits on an edge that an FP32 distance crossed
        b_gpu = np.rint(eps[s].astype(np.float64) / (em[s] / n_bins)).astype(np.int64)
        b_or = np.rint(e_or / w).astype(np.int64)
        assert np.all(np.abs(b_gpu - b_or) <= 1), (hex(int(m)), b_gpu, b_or)
        np.testing.assert_allclose(eps[s], e_or, atol=w * 1.001 + 1e-6, rtol=0)
        yield int(np.sum(b_gpu == b_or))


@pytest.mark.parametrize("n,seed,n_sample,n_bins", [(3000, 0, 512, 4096), (2049, 7, 4000, 300),
                                                    (613, 5, 37, 64)])
def test_selectivity_matches_oracle(ctx, n, seed, n_sample, n_bins):
    x = snaps_inputs.population(n, seed)
    masks = np.array([0b11, 0b100100010000100, 0b111111110000000, (1 << 15) - 1], dtype=np.uint16)
    targets = [0.001 * n, 0.15 * n, 2.5, 0.5 * n, n - 1]
    pop = snaps.snaps_index(ctx, x)
    try:
        eps, em = snaps.snaps_eps_selectivity(pop, masks, targets, n_sample, n_bins)
    finally:
        snaps.snaps_release(pop)
    xn = oracle.normalise(x)
    equal = sum(check_against_oracle(xn, masks, targets, eps, em, n_sample, n_bins))
    assert equal >= len(masks) * len(targets) - 2
    # n - 1 neighbours on average is out of reach below eps_mean
    np.testing.assert_array_equal(eps[:, -1], em)


def test_selectivity_range_wrapper(ctx):
    n = 1200
    x = snaps_inputs.population(n, 9)
    masks = np.array([0b1110, 0b111000111], dtype=np.uint16)
    pop = snaps.snaps_index(ctx, x)
    try:
        lo, hi = snaps.snaps_eps_range(pop, n, masks, n_sample=n)
        eps, _ = snaps.snaps_eps_selectivity(pop, masks, [0.001 * n, 0.15 * n], n_sample=n)
    finally:
        snaps.snaps_release(pop)
    np.testing.assert_array_equal(lo, eps[:, 0])
    np.testing.assert_array_equal(hi, eps[:, 1])
    assert np.all(lo < hi)
    # the radii reach their selectivities (the definition, by the brute-force join)
    xn = oracle.normalise(x)
    for s, m in enumerate(masks):
        assert oracle.selectivity(xn, int(m), float(hi[s])) >= 0.15 * n * (1 - 1e-3)


def test_selectivity_identical_objects(ctx):
    x = np.full((100, 5), 3.0, dtype=np.float32)
    pop = snaps.snaps_index(ctx, x)
    try:
        eps, em = snaps.snaps_eps_selectivity(pop, np.array([0b11, 0b11111], dtype=np.uint16), [1.0, 50.0], 100,
                                              128)
    finally:
        snaps.snaps_release(pop)
    assert np.all(em == 0.0) and np.all(eps == 0.0)


def test_selectivity_rejects_bad_requests(ctx):
    x = snaps_inputs.population(300, 2)
    masks = np.array([0b110], dtype=np.uint16)
    pop = snaps.snaps_index(ctx, x)
    try:
        for kw in (dict(targets=[0.0]),                   # not above 0
                   dict(targets=[300.0]),                 # above n - 1
                   dict(targets=list(range(1, 34))),      # too many targets
                   dict(targets=[3.0], n_sample=0),
                   dict(targets=[3.0], n_sample=70000),
                   dict(targets=[3.0], n_bins=0),
                   dict(targets=[3.0], n_bins=4097)):
            with pytest.raises(snaps.SnapsError) as e:
                snaps.snaps_eps_selectivity(pop, masks, **kw)
            assert e.value.status == snaps.SNAPS_EINVAL
        with pytest.raises(snaps.SnapsError):
            snaps.snaps_eps_selectivity(pop, np.array([0b1], dtype=np.uint16), [3.0])
    finally:
        snaps.snaps_release(pop)
