"""Parity of the CUDA library (through the C ABI) with the FP64 oracle, element
by element, on seeded populations: normalisation, both joins, the four
metrics, normalised metrics and top-n lists, across tile boundaries, ragged
tails, both kNN-list capacities, the subspace-batched and lane-per-subspace
kernels, and the degenerate cases."""
import numpy as np
import pytest

import oracle
import paper_2405_20176_b300 as snaps
import snaps_inputs
from parity import BAND, check_eps, check_knn, check_norm, check_top

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = snaps.snaps_create(0)
    yield c
    snaps.snaps_destroy(c)


def gpu_all(ctx, x, masks, k, eps=None, flags=snaps.SNAPS_NORM_MINMAX, top_n=100):
    """Run every entry point on device outputs and return host copies."""
    masks = np.asarray(masks, dtype=np.uint16)
    pop = snaps.snaps_index(ctx, np.ascontiguousarray(x, dtype=np.float32), flags)
    try:
        n, f = snaps.snaps_pop_shape(pop)
        m = masks.size
        dev = torch.device("cuda")
        feat = np.zeros((n, f), dtype=np.float32)
        snaps.snaps_pop_features(pop, feat)
        sc = torch.empty((m, 4, n), dtype=torch.float32, device=dev)
        nz = torch.empty((m, 4, n), dtype=torch.float32, device=dev)
        top_n = min(top_n, n)
        tp = torch.empty((m, 4, top_n), dtype=torch.int32, device=dev)
        snaps.snaps_scores(pop, masks, k, eps=eps, scores=sc, norm=nz, top=tp, top_n=top_n)
        idx = torch.empty((m, n, k), dtype=torch.int32, device=dev)
        dist = torch.empty((m, n, k), dtype=torch.float32, device=dev)
        snaps.snaps_knn_selfjoin(pop, masks, k, idx, dist)
        cnt = torch.empty((m, n), dtype=torch.int32, device=dev)
        mean = torch.empty((m, n), dtype=torch.float32, device=dev)
        snaps.snaps_eps_selfjoin(pop, masks, eps, cnt, mean)
        torch.cuda.synchronize()
        return dict(features=feat, scores=sc.cpu().numpy(), norm=nz.cpu().numpy(),
                    top=tp.cpu().numpy(), idx=idx.cpu().numpy(), dist=dist.cpu().numpy(),
                    count=cnt.cpu().numpy(), mean=mean.cpu().numpy())
    finally:
        snaps.snaps_release(pop)


def compare(g, xn, masks, k, eps=None, top_n=100):
    """Full comparison of one gpu_all result with the oracle."""
    x64 = xn.astype(np.float64)
    n = xn.shape[0]
    stats = {"knn_rows_differ": 0, "eps_in_band": 0}
    for s, mask in enumerate(np.asarray(masks, dtype=np.uint16)):
        mask = int(mask)
        e = None if eps is None else float(eps[s])
        r = oracle.subspace(xn, mask, k, eps=e, top_n=min(top_n, n))
        e2 = oracle.default_eps2(mask) if e is None else float(np.float64(np.float32(e)) ** 2)
        # kNN lists (two entry points must agree exactly with each other)
        stats["knn_rows_differ"] += check_knn(x64, mask, g["idx"][s], g["dist"][s],
                                              r.join.knn_idx, r.join.knn_d2)
        # eps join
        lo, hi = oracle.join(x64, mask, 0, e2 * (1 - BAND)).eps_count, \
            oracle.join(x64, mask, 0, e2 * (1 + BAND)).eps_count
        ora_eps = oracle.join(x64, mask, 0, e2)
        stats["eps_in_band"] += check_eps(g["count"][s], g["mean"][s], ora_eps, lo, hi)
        sc = g["scores"][s]
        np.testing.assert_array_equal(sc[0], g["count"][s])
        np.testing.assert_array_equal(sc[1], g["mean"][s])
        if stats["knn_rows_differ"] == 0:
            np.testing.assert_array_equal(sc[2], r.scores[oracle.KNN_INDEG])
        assert sc[2].sum() == n * k
        np.testing.assert_allclose(sc[3], r.scores[oracle.KNN_MEAN], rtol=1e-5, atol=1e-12)
        # normalised metrics, all four: the step itself and end to end
        check_norm(g["norm"][s], sc, r.scores, r.normalised)
        # top lists
        for m in range(4):
            if m in (oracle.EPS_COUNT,) and not np.array_equal(sc[0], r.scores[0]):
                continue
            if m == oracle.KNN_INDEG and not np.array_equal(sc[2], r.scores[2]):
                continue
            check_top(g["top"][s][m], r.scores, r.top[m], m)
    return stats


def test_normalisation_is_bit_exact(ctx):
    x = snaps_inputs.population(3001, 7)
    x[:, 3] = x[:, 3] * 37.5 - 4.0
    x[:, 9] = 0.25   # constant column
    pop = snaps.snaps_index(ctx, x)
    try:
        feat = np.zeros_like(x)
        snaps.snaps_pop_features(pop, feat)
    finally:
        snaps.snaps_release(pop)
    np.testing.assert_array_equal(feat, oracle.normalise(x))


def test_nan_to_mean(ctx):
    x = np.array([[0.0, 1.0], [np.nan, 3.0], [2.0, np.nan], [4.0, 5.0]], dtype=np.float32)
    pop = snaps.snaps_index(ctx, x, snaps.SNAPS_NORM_MINMAX | snaps.SNAPS_NAN_TO_MEAN)
    try:
        feat = np.zeros_like(x)
        snaps.snaps_pop_features(pop, feat)
    finally:
        snaps.snaps_release(pop)
    np.testing.assert_array_equal(feat, oracle.normalise(x, nan_to_mean=True))
    with pytest.raises(snaps.SnapsError) as ei:
        snaps.snaps_index(ctx, x, snaps.SNAPS_NORM_MINMAX)
    assert ei.value.status == snaps.SNAPS_EINVAL


def test_table2_worked_example(ctx, golden_dir):
    import json
    import os
    with open(os.path.join(golden_dir, "table2.json")) as fh:
        t2 = json.load(fh)
    # integer coordinates (x100): exact in FP32, so the figure's tie is exact
    x = np.rint(np.array(t2["points"]) * 100).astype(np.float32)
    g = gpu_all(ctx, x, [0b11], 3, eps=[67.0], flags=0, top_n=10)
    sc = g["scores"][0]
    np.testing.assert_array_equal(sc[0], t2["dssj_num_neighbors"])
    np.testing.assert_allclose(sc[1] / 100, t2["dssj_mean_distance"], atol=5e-5)
    np.testing.assert_array_equal(sc[2], t2["knn_in_degree"])
    np.testing.assert_allclose(sc[3] / 100, t2["knn_mean_distance"], atol=5e-5)
    for s, edges in t2["knn_edges_1based"].items():
        assert sorted((g["idx"][0][int(s) - 1] + 1).tolist()) == sorted(edges)
    assert (g["idx"][0][0] + 1).tolist() == [3, 7, 2]
    for m, name in enumerate(["dssj_num_neighbors_rank", "dssj_mean_distance_rank",
                              "knn_in_degree_rank", "knn_mean_distance_rank"]):
        expect = np.lexsort((np.arange(10), np.array(t2[name])))
        np.testing.assert_array_equal(g["top"][0][m], expect)
    # normalised metrics worked out by hand from the printed Table 2 values
    with open(os.path.join(golden_dir, "normalised.json")) as fh:
        z = json.load(fh)["table2"]
    for m, name, tol in [(0, "eps_count", 1e-7), (1, "eps_mean", 1e-3), (2, "knn_indeg", 1e-7),
                         (3, "knn_mean", 1e-3)]:
        np.testing.assert_allclose(g["norm"][0][m], z[name], rtol=0, atol=tol, err_msg=name)


def test_config1_full_space(ctx):
    """N = 2,000, full 15-feature subspace, k = 10, eps = 0.05 sqrt(15)."""
    x = snaps_inputs.population(2000, 0)
    g = gpu_all(ctx, x, [(1 << 15) - 1], 10)
    xn = oracle.normalise(x)
    np.testing.assert_array_equal(g["features"], xn)
    st = compare(g, xn, [(1 << 15) - 1], 10)
    assert st["knn_rows_differ"] <= 2


@pytest.mark.parametrize("n,seed", [(700, 1), (257, 2), (513, 3)])
def test_dense_chunks_tree_kernel(ctx, n, seed):
    """Whole 32-subspace chunks (the batched tree kernel) plus lone masks."""
    x = snaps_inputs.population(n, seed)
    allm = snaps_inputs.all_masks()
    chunk_a = allm[(allm >> 5) == 0b0000010011]          # one dense chunk
    chunk_b = allm[(allm >> 5) == 0b1111111111]          # the top chunk (contains the full mask)
    lone = np.array([0b11, 0b100000000000001, 0b010101010101010], dtype=np.uint16)
    masks = np.concatenate([chunk_a, chunk_b, lone])
    g = gpu_all(ctx, x, masks, 10)
    st = compare(g, oracle.normalise(x), masks, 10)
    assert st["knn_rows_differ"] <= max(2, n * masks.size // 2000)


@pytest.mark.parametrize("k", [1, 5, 16, 17, 20, 32])
def test_k_range(ctx, k):
    x = snaps_inputs.population(300, 40 + k)
    allm = snaps_inputs.all_masks()
    masks = np.concatenate([allm[(allm >> 5) == 3][:12], [0b111000]]).astype(np.uint16)
    g = gpu_all(ctx, x, masks, k)
    compare(g, oracle.normalise(x), masks, k)


@pytest.mark.parametrize("n", [2, 3, 40, 64, 65, 255, 256])
def test_tiny_and_ragged_sizes(ctx, n):
    x = snaps_inputs.population(n, 100 + n)
    k = min(10, n - 1)
    allm = snaps_inputs.all_masks()
    masks = np.concatenate([allm[(allm >> 5) == 0b1000000000][:20], [0b11, 0b110]]).astype(np.uint16)
    g = gpu_all(ctx, x, masks, k, top_n=min(100, n))
    compare(g, oracle.normalise(x), masks, k, top_n=min(100, n))


def test_custom_eps_and_extremes(ctx):
    x = snaps_inputs.population(400, 9)
    masks = np.array([0b11, 0b111, 0b1111, 0b11111, (1 << 15) - 1], dtype=np.uint16)
    # eps beyond the diameter: everyone; below any distance: nobody
    g = gpu_all(ctx, x, masks, 10, eps=[2.0, 2.0, 1e-9, 0.0, 4.0])
    assert np.all(g["count"][0] == 399) and np.all(g["count"][4] == 399)
    assert np.all(g["count"][2] == 0) and np.all(g["scores"][2][1] == 0)
    compare(g, oracle.normalise(x), masks, 10, eps=[2.0, 2.0, 1e-9, 0.0, 4.0])


@pytest.mark.parametrize("case", ["no_neighbours", "crowded_bin"])
def test_top_lists_crowded_rows(ctx, case):
    """Rows whose top-100 boundary falls in a crowded part of the ranking: every
    object tied (no eps-neighbours anywhere: the lowest indices win), and
    99 far outliers above a cluster of 8,901 objects whose kNN mean distances
    all fall in one code bin of the finishing kernel."""
    rng = np.random.default_rng(77)
    if case == "no_neighbours":
        x = rng.uniform(0.0, 1.0, size=(9000, 2)).astype(np.float32)
        eps = [0.0]
    else:
        cluster = rng.uniform(0.0, 0.01, size=(8901, 2))
        line = 1.0 + 0.5 * np.arange(99)[:, None] * np.ones((1, 2))
        x = np.concatenate([cluster, line])[rng.permutation(9000)].astype(np.float32)
        eps = [0.002]
    g = gpu_all(ctx, x, [0b11], 10, eps=eps, flags=0)
    compare(g, x, [0b11], 10, eps=eps)
    if case == "no_neighbours":
        assert np.all(g["scores"][0][0] == 0)
        for m in (oracle.EPS_COUNT, oracle.EPS_MEAN):
            np.testing.assert_array_equal(g["top"][0][m], np.arange(100))


def test_lattice_ties_and_duplicates_exact(ctx):
    # 2-D lattice with spacing 1/8: every squared distance is exact in FP32,
    # so neighbours (ties broken by index) and counts must match exactly
    m = 16
    pts = np.array([(a, b) for a in range(m) for b in range(m)], dtype=np.float64) / 8
    x = np.concatenate([pts, pts[:7]]).astype(np.float32)   # 7 exact duplicates
    masks = [0b11]
    g = gpu_all(ctx, x, masks, 8, eps=[0.25], flags=0)
    r = oracle.subspace(x.astype(np.float64), 0b11, 8, eps=0.25)
    np.testing.assert_array_equal(g["idx"][0], r.join.knn_idx)
    np.testing.assert_array_equal(g["count"][0], r.join.eps_count)
    np.testing.assert_array_equal(g["scores"][0][2], r.scores[oracle.KNN_INDEG])
    for mm in range(4):
        check_top(g["top"][0][mm], r.scores, r.top[mm], mm)


def test_host_and_device_outputs_agree(ctx):
    x = snaps_inputs.population(1000, 12)
    masks = snaps_inputs.mask_sample(40, 3)
    pop = snaps.snaps_index(ctx, x)
    try:
        n = 1000
        sc_h = np.zeros((masks.size, 4, n), dtype=np.float32)
        tp_h = np.zeros((masks.size, 4, 100), dtype=np.int32)
        snaps.snaps_scores(pop, masks, 10, scores=sc_h, top=tp_h, top_n=100)
        sc_d = torch.empty((masks.size, 4, n), device="cuda")
        tp_d = torch.empty((masks.size, 4, 100), dtype=torch.int32, device="cuda")
        snaps.snaps_scores(pop, masks, 10, scores=sc_d, top=tp_d, top_n=100)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(sc_h, sc_d.cpu().numpy())
        np.testing.assert_array_equal(tp_h, tp_d.cpu().numpy())
        # a device-resident input population gives the same bits
        pop2 = snaps.snaps_index(ctx, torch.from_numpy(x).cuda())
        try:
            sc2 = np.zeros_like(sc_h)
            snaps.snaps_scores(pop2, masks, 10, scores=sc2)
            np.testing.assert_array_equal(sc_h, sc2)
        finally:
            snaps.snaps_release(pop2)
    finally:
        snaps.snaps_release(pop)


def test_subset_of_masks_matches_full_batch(ctx):
    """Results for a subspace do not depend on what else is in the batch
    (tree vs lane-per-subspace kernels give the same bits)."""
    x = snaps_inputs.population(600, 21)
    allm = snaps_inputs.all_masks()
    chunk = allm[(allm >> 5) == 0b0110000001]
    pop = snaps.snaps_index(ctx, x)
    try:
        full = np.zeros((chunk.size, 4, 600), dtype=np.float32)
        snaps.snaps_scores(pop, chunk, 10, scores=full)
        for s in range(0, chunk.size, 7):
            one = np.zeros((1, 4, 600), dtype=np.float32)
            snaps.snaps_scores(pop, chunk[s:s + 1], 10, scores=one)
            np.testing.assert_array_equal(one[0], full[s])
    finally:
        snaps.snaps_release(pop)


def test_invalid_requests(ctx):
    x = snaps_inputs.population(50, 1)
    pop = snaps.snaps_index(ctx, x)
    try:
        out = np.zeros((1, 4, 50), dtype=np.float32)
        for masks, k in [([0b1], 5), ([1 << 15], 5), ([0b11], 0), ([0b11], 50), ([0b11], 33)]:
            with pytest.raises(snaps.SnapsError) as ei:
                snaps.snaps_scores(pop, masks, k, scores=out)
            assert ei.value.status == snaps.SNAPS_EINVAL
        with pytest.raises(snaps.SnapsError):
            snaps.snaps_index(ctx, np.zeros((1, 3), dtype=np.float32))
        bad = x.copy()
        bad[3, 2] = np.inf
        with pytest.raises(snaps.SnapsError):
            snaps.snaps_index(ctx, bad)
    finally:
        snaps.snaps_release(pop)
