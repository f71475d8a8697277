"""Pin the oracle's normalised metrics to values worked out by hand: Table 2's
printed metrics mapped onto [0, 1] (4-decimal inputs, so a 1e-3 tolerance),
and a four-point example whose metrics are exact.  A mis-scaling that keeps
the ranking -- for instance the eps mean distance scaled over all objects,
those without neighbours included -- fails these values."""
import json
import os

import numpy as np
import pytest

import oracle

NAMES = ["eps_count", "eps_mean", "knn_indeg", "knn_mean"]


@pytest.fixture(scope="module")
def golden(golden_dir):
    with open(os.path.join(golden_dir, "normalised.json")) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def table2(golden_dir):
    with open(os.path.join(golden_dir, "table2.json")) as fh:
        return json.load(fh)


def test_table2_normalised_values(golden, table2):
    # integer coordinates (x100): exact distances, the figure's tie exact
    pts = np.rint(np.array(table2["points"]) * 100)
    z = oracle.subspace(pts, 0b11, table2["k"], eps=table2["eps"] * 100, top_n=10).normalised
    exp = golden["table2"]
    np.testing.assert_allclose(z[oracle.EPS_COUNT], exp["eps_count"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(z[oracle.KNN_INDEG], exp["knn_indeg"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(z[oracle.EPS_MEAN], exp["eps_mean"], rtol=0, atol=1e-3)
    np.testing.assert_allclose(z[oracle.KNN_MEAN], exp["knn_mean"], rtol=0, atol=1e-3)


def test_line_normalised_values_exact(golden):
    g = golden["line"]
    r = oracle.subspace(np.array(g["points"]), 0b11, g["k"], eps=g["eps"], top_n=4)
    for m, name in enumerate(NAMES):
        np.testing.assert_allclose(r.normalised[m], g[name], rtol=0, atol=1e-15, err_msg=name)


def test_constant_metric_maps_to_zero():
    # unit square: every corner has two eps-neighbours at distance 1
    pts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    r = oracle.subspace(pts, 0b11, 1, eps=1.0, top_n=4)
    assert np.all(r.scores[oracle.EPS_COUNT] == 2) and np.all(r.scores[oracle.EPS_MEAN] == 1.0)
    assert np.all(r.normalised[oracle.EPS_COUNT] == 0.0)
    assert np.all(r.normalised[oracle.EPS_MEAN] == 0.0)
    assert np.all(r.normalised[oracle.KNN_MEAN] == 0.0)


def test_nobody_has_neighbours():
    # eps below every distance: every object ranks first for the eps mean distance
    pts = np.array([[0.0, 0.0], [1.0, 0.0], [3.0, 0.0]])
    r = oracle.subspace(pts, 0b11, 1, eps=0.5, top_n=3)
    assert np.all(r.normalised[oracle.EPS_MEAN] == 1.0)
    assert np.all(r.normalised[oracle.EPS_COUNT] == 0.0)
