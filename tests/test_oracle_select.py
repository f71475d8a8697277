"""Pins of the oracle's parameter selection (Sec. 3.5.2, Eq. 2 and 3;
Sec. 3.6.2) against the paper's worked example and against properties the
definitions force."""
import numpy as np

import oracle
import snaps_inputs


def test_worked_example_of_eq2_and_eq3():
    # the illustrative example of Sec. 3.5.2 (n = 10, |G| = 3)
    e1 = [1, 2, 3, 4, 5, 16, 17, 18, 19, 20]
    e2 = [1, 2, 3, 4, 8, 9, 10, 100, 101, 102]
    e3 = [1, 2, 8, 9, 10, 11, 12, 13, 14, 15]
    u_min, u_max = oracle.u_curves([e1, e2, e3])
    np.testing.assert_allclose(u_min, [1.0, 0.4, 0.2])
    np.testing.assert_allclose(u_max, [0.2, 0.5, 1.0])
    # |U^min - U^max| = {0.8, 0.1, 0.8}: the middle radius is selected
    assert oracle.select_index(u_min, u_max) == 1


def test_similarity_is_a_set_overlap():
    assert oracle.similarity([3, 1, 2], [2, 3, 1]) == 1.0   # order does not matter
    assert oracle.similarity([1, 2, 3, 4], [5, 6, 7, 8]) == 0.0
    assert oracle.similarity([1, 2, 3, 4], [4, 9, 1, 7]) == 0.5


def test_select_index_takes_the_first_of_equal_gaps():
    assert oracle.select_index([1.0, 0.6, 0.4, 0.2], [0.2, 0.4, 0.6, 1.0]) == 1


def test_grids_and_curve_ends():
    g = oracle.eps_grid(0.05, 0.25, 5)
    np.testing.assert_allclose(g, [0.05, 0.1, 0.15, 0.2, 0.25], rtol=1e-7)
    assert g.dtype == np.float32
    x = oracle.normalise(snaps_inputs.population(400, 3))
    mask = 0b101100000000110
    u, sel, tops = oracle.select_eps(x, mask, 0.05, 0.4, 6, 8)
    # a list compared with itself matches fully: U^min_1 = U^max_G = 1
    assert np.all(u[:, 0, 0] == 1.0) and np.all(u[:, 1, -1] == 1.0)
    assert np.all((u >= 0.0) & (u <= 1.0))
    assert tops.shape == (6, 2, 8)
    for r in range(2):
        assert sel[r] == oracle.select_index(u[r, 0], u[r, 1])
    uk, selk, topk = oracle.select_k(x, mask, [2, 4, 8, 16], 8)
    assert np.all(uk[:, 0, 0] == 1.0) and np.all(uk[:, 1, -1] == 1.0)
    assert topk.shape == (4, 2, 8)


def test_select_eps_grid_end_matches_a_plain_join():
    # the ranking at a grid radius is the one snaps_scores defines for that radius
    x = oracle.normalise(snaps_inputs.population(300, 5))
    mask = 0b11000000011
    _, _, tops = oracle.select_eps(x, mask, 0.1, 0.3, 3, 10)
    r = oracle.subspace(x, mask, 1, eps=float(np.float32(0.3)), top_n=10)
    np.testing.assert_array_equal(tops[-1, 0], r.top[oracle.EPS_COUNT])
    np.testing.assert_array_equal(tops[-1, 1], r.top[oracle.EPS_MEAN])
