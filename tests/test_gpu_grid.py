"""The grid-indexed join for subspaces of <= 4 features (sort-by-cell index,
Sec. 3.8.1; DSSJ, Sec. 3.5; kNNSJ, Sec. 3.6) returns the brute-force join's
results bit for bit -- same canonical FP32 distances, same exact decisions --
across populations, k, radii that give one cell or the largest grid, sparse
points that need the kNN ring search, and the tensor-core form (whose mean
eps distances come from its accumulator, within 1e-5); at a size
where the library picks the grid on its own, it matches the FP64 oracle on
sampled queries."""
import numpy as np
import pytest

import oracle
import paper_2405_20176_b300 as snaps
import snaps_inputs
from parity import SCORE_RTOL, check_eps, check_knn, check_top, eps_bounds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRID = snaps.SNAPS_INDEX_GRID
NONE = snaps.SNAPS_INDEX_NONE


@pytest.fixture(scope="module")
def ctx():
    c = snaps.snaps_create(0)
    snaps.snaps_set_tc_min_fill(c, 1)  # the tensor-core form's subspaces on the tensor cores
    yield c
    snaps.snaps_destroy(c)


def low_d_masks(n3, seed):
    """All 105 two-feature subspaces, n3 three-feature ones and n3 / 2 of four
    features (indexed on their three highest features, refined on all four)."""
    allm = snaps_inputs.all_masks()
    pc = np.array([bin(int(v)).count("1") for v in allm])
    rng = np.random.default_rng(seed)
    three = rng.choice(allm[pc == 3], size=n3, replace=False)
    four = rng.choice(allm[pc == 4], size=max(2, n3 // 2), replace=False)
    return np.concatenate([allm[pc == 2], np.sort(three), np.sort(four)]).astype(np.uint16)


def scores_with(ctx, x, masks, k, precision, eps=None, flags=snaps.SNAPS_NORM_MINMAX, top_n=100):
    masks = np.asarray(masks, dtype=np.uint16)
    pop = snaps.snaps_index(ctx, np.ascontiguousarray(x, dtype=np.float32), flags)
    try:
        n = x.shape[0]
        top_n = min(top_n, n)
        sc = torch.empty((masks.size, 4, n), device="cuda")
        nz = torch.empty((masks.size, 4, n), device="cuda")
        tp = torch.empty((masks.size, 4, top_n), dtype=torch.int32, device="cuda")
        snaps.snaps_trace(ctx, True)
        snaps.snaps_scores(pop, masks, k, eps=eps, precision=precision, scores=sc, norm=nz, top=tp,
                           top_n=top_n)
        torch.cuda.synchronize()
        tr = snaps.snaps_trace_read(ctx)
        snaps.snaps_trace(ctx, False)
        return sc.cpu().numpy(), nz.cpu().numpy(), tp.cpu().numpy(), tr
    finally:
        snaps.snaps_release(pop)


def assert_grid_equals_brute(ctx, x, masks, k, eps=None, form=snaps.SNAPS_FP32):
    g = scores_with(ctx, x, masks, k, form | GRID, eps)
    b = scores_with(ctx, x, masks, k, form | NONE, eps)
    assert g[3]["grid"][1] > 0, "the grid path ran"
    assert b[3]["grid"][1] == 0, "brute force took no grid"
    if form == snaps.SNAPS_FP32:
        for u, v, name in zip(g[:3], b[:3], ("scores", "norm", "top")):
            np.testing.assert_array_equal(u, v, err_msg=name)
        return
    # the tensor-core join's mean eps distances come from its accumulator: the
    # other metrics and their rankings are the grid's bits, those within 1e-5
    same = [0, 2, 3]
    for u, v, name in zip(g[:3], b[:3], ("scores", "norm", "top")):
        np.testing.assert_array_equal(u[:, same], v[:, same], err_msg=name)
    np.testing.assert_allclose(b[0][:, 1], g[0][:, 1], rtol=SCORE_RTOL, atol=1e-6)
    for s in range(g[0].shape[0]):
        check_top(b[2][s, 1], g[0][s].astype(np.float64), g[2][s, 1], oracle.EPS_MEAN)


@pytest.mark.parametrize("n,seed", [(2000, 0), (3001, 4), (513, 2)])
def test_grid_equals_brute_force(ctx, n, seed):
    assert_grid_equals_brute(ctx, snaps_inputs.population(n, seed), low_d_masks(30, seed), 10)


@pytest.mark.parametrize("k", [1, 17, 32])
def test_grid_k_range(ctx, k):
    assert_grid_equals_brute(ctx, snaps_inputs.population(1500, 10 + k), low_d_masks(10, k), k)


def test_grid_radius_extremes(ctx):
    x = snaps_inputs.population(1200, 3)
    masks = low_d_masks(6, 3)
    m = masks.size
    # a radius far below the grid's smallest cell (the cell cap binds), one that
    # covers everything (a single cell), and zero
    for e in (1e-4, 2.0, 0.0):
        assert_grid_equals_brute(ctx, x, masks, 10, eps=np.full(m, e, dtype=np.float32))


def test_grid_sparse_points_need_rings(ctx):
    # a tight cluster plus scattered points: the scattered points' k-th
    # neighbour lies many cells away, so the ring search must reach it
    rng = np.random.default_rng(7)
    x = np.clip(rng.normal(0.5, 0.01, size=(900, 15)), 0, 1)
    x[:40] = rng.random((40, 15))
    x = x.astype(np.float32)
    assert_grid_equals_brute(ctx, x, low_d_masks(8, 7), 20)


def test_grid_tensor_core_form(ctx):
    assert_grid_equals_brute(ctx, snaps_inputs.population(1800, 5), low_d_masks(12, 5), 10,
                             form=snaps.SNAPS_TC_F16)


def test_grid_chosen_at_scale_matches_oracle(ctx):
    # n >= SNAPS_GRID_AUTO_N: the library takes the grid by itself for these
    # subspaces; checked against the FP64 oracle on sampled queries
    n = snaps.SNAPS_GRID_AUTO_N + 4463
    x = snaps_inputs.population(n, 11)
    masks = np.array([0b11, 0b1000000000100, 0b100100000010000, 0b110000001000100], dtype=np.uint16)
    k = 10
    pop = snaps.snaps_index(ctx, x)
    try:
        m = masks.size
        idx = torch.empty((m, n, k), dtype=torch.int32, device="cuda")
        dist = torch.empty((m, n, k), dtype=torch.float32, device="cuda")
        cnt = torch.empty((m, n), dtype=torch.int32, device="cuda")
        mean = torch.empty((m, n), dtype=torch.float32, device="cuda")
        snaps.snaps_trace(ctx, True)
        snaps.snaps_knn_selfjoin(pop, masks, k, idx, dist)
        snaps.snaps_eps_selfjoin(pop, masks, None, cnt, mean)
        torch.cuda.synchronize()
        tr = snaps.snaps_trace_read(ctx)
        snaps.snaps_trace(ctx, False)
        assert tr["grid"][1] > 0 and tr["join_tree"][1] == 0 and tr["join_lane"][1] == 0
        idx, dist, cnt, mean = (t.cpu().numpy() for t in (idx, dist, cnt, mean))
    finally:
        snaps.snaps_release(pop)
    xn = oracle.normalise(x)
    x64 = xn.astype(np.float64)
    q = np.sort(np.random.default_rng(12).choice(n, size=160, replace=False))
    for s, mask in enumerate(masks):
        mask = int(mask)
        e2 = oracle.default_eps2(mask)
        r = oracle.join(x64, mask, k, e2, queries=q)
        check_knn(x64, mask, idx[s][q], dist[s][q], r.knn_idx, r.knn_d2, queries=q)
        lo, hi = eps_bounds(x64, mask, e2, queries=q)
        check_eps(cnt[s][q], mean[s][q], r, lo, hi)


@pytest.mark.parametrize("cells", [2, 3])
def test_finer_cells_equal_brute_force(ctx, cells):
    # cells 1/R of eps wide search a (2R + 1)^D block; the same bits as brute
    # force, including the kNN rings of scattered points and a radius of zero
    try:
        for n, k in ((2000, 10), (900, 20)):
            for d in (2, 3, 4):
                snaps.snaps_autotune_set(ctx, n, k, d, True, 1.0 / cells)
        assert_grid_equals_brute(ctx, snaps_inputs.population(2000, 11), low_d_masks(16, 11), 10)
        rng = np.random.default_rng(8)
        x = np.clip(rng.normal(0.5, 0.01, size=(900, 15)), 0, 1)
        x[:40] = rng.random((40, 15))
        masks = low_d_masks(8, 8)
        assert_grid_equals_brute(ctx, x.astype(np.float32), masks, 20)
        assert_grid_equals_brute(ctx, x.astype(np.float32), masks, 20, eps=np.zeros(masks.size, np.float32))
    finally:
        snaps.snaps_autotune_clear(ctx)
