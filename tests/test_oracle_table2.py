"""Pin the oracle to the paper's worked example: Fig. 1 points, eps = 0.67,
k = 3, and every metric value and ranking of Table 2 plus the kNN graph of
Fig. 1b.  The expected numbers are the paper's, stored in tests/golden."""
import json
import os

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def table2(golden_dir):
    with open(os.path.join(golden_dir, "table2.json")) as fh:
        return json.load(fh)


def _run(points, eps, k):
    return oracle.subspace(points, 0b11, k, eps=eps, top_n=10)


@pytest.mark.parametrize("scale", [1, 100])
def test_table2_values_and_ranks(table2, scale):
    # scale 100 turns every coordinate into an integer, so all squared
    # distances are exact and the tie of Fig. 1b point 1 is an exact tie.
    pts = np.array(table2["points"], dtype=np.float64)
    pts = np.rint(pts * 100) if scale == 100 else pts
    eps = table2["eps"] * scale
    r = _run(pts, eps, table2["k"])
    s = r.scores
    np.testing.assert_array_equal(s[oracle.EPS_COUNT], table2["dssj_num_neighbors"])
    np.testing.assert_allclose(s[oracle.EPS_MEAN] / scale, table2["dssj_mean_distance"], atol=5e-5)
    np.testing.assert_array_equal(s[oracle.KNN_INDEG], table2["knn_in_degree"])
    np.testing.assert_allclose(s[oracle.KNN_MEAN] / scale, table2["knn_mean_distance"], atol=5e-5)
    np.testing.assert_array_equal(r.ranks[oracle.EPS_COUNT], table2["dssj_num_neighbors_rank"])
    np.testing.assert_array_equal(r.ranks[oracle.EPS_MEAN], table2["dssj_mean_distance_rank"])
    np.testing.assert_array_equal(r.ranks[oracle.KNN_INDEG], table2["knn_in_degree_rank"])
    np.testing.assert_array_equal(r.ranks[oracle.KNN_MEAN], table2["knn_mean_distance_rank"])


@pytest.mark.parametrize("scale", [1, 100])
def test_fig1b_knn_graph(table2, scale):
    pts = np.array(table2["points"], dtype=np.float64)
    pts = np.rint(pts * 100) if scale == 100 else pts
    r = _run(pts, table2["eps"] * scale, table2["k"])
    for src, dst in table2["knn_edges_1based"].items():
        got = sorted((r.join.knn_idx[int(src) - 1] + 1).tolist())
        assert got == sorted(dst), (src, got, dst)
    # nearest first: point 1's list is 3, 7, then the tie (2 before 4)
    assert (r.join.knn_idx[0] + 1).tolist() == [3, 7, 2]


def test_table2_top_lists_follow_ranks(table2):
    pts = np.rint(np.array(table2["points"]) * 100)
    r = _run(pts, 67.0, 3)
    for m, name in enumerate(["dssj_num_neighbors_rank", "dssj_mean_distance_rank",
                              "knn_in_degree_rank", "knn_mean_distance_rank"]):
        rk = np.array(table2[name])
        expect = np.lexsort((np.arange(10), rk))
        np.testing.assert_array_equal(r.top[m], expect)
    # point 10 is rank 0 in all four rankings (Sec. 3.7)
    assert all(r.top[m][0] == 9 for m in range(4))


def test_table2_normalised_scores(table2):
    pts = np.rint(np.array(table2["points"]) * 100)
    r = _run(pts, 67.0, 3)
    z = r.normalised
    assert z.min() >= 0.0 and z.max() <= 1.0
    # point 10 is the most outlying object under every metric
    assert np.all(z[:, 9] == 1.0)
    # counts: 4 neighbours (point 3) is the least outlying -> 0
    assert z[oracle.EPS_COUNT][2] == 0.0
    # the normalised value is monotone in the rank for every metric
    for m in range(4):
        order = np.argsort(r.ranks[m], kind="stable")
        assert np.all(np.diff(z[m][order]) <= 0.0)
