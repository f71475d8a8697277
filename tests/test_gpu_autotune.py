"""The index-route autotuner (snaps_autotune): it reports a measurement and a
choice for subspaces of 2, 3 and 4 features, and whatever it chooses, the
auto route and the forced grid return the same bits as brute force; on a
population above the tuning size it times a sample.  Invalid k is rejected."""
import numpy as np
import pytest

import paper_2405_20176_b300 as snaps
import snaps_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MASKS = np.array([0b11, 0b110000000000000, 0b100000000001, 0b111, 0b101000000000100, 0b1111,
                  0b110000000000011, 0b111111111111111, 0b1010101], dtype=np.uint16)


@pytest.fixture()
def ctx():
    c = snaps.snaps_create(0)
    yield c
    snaps.snaps_destroy(c)


def scores_of(pop, n, k, precision):
    sc = torch.empty((MASKS.size, 4, n), device="cuda")
    top = torch.empty((MASKS.size, 4, 100), dtype=torch.int32, device="cuda")
    snaps.snaps_scores(pop, MASKS, k, precision=precision, scores=sc, top=top, top_n=100)
    torch.cuda.synchronize()
    return sc.cpu().numpy(), top.cpu().numpy()


@pytest.mark.parametrize("n,k", [(20000, 10), (70001, 20)])
def test_autotune_keeps_results(ctx, n, k):
    x = snaps_inputs.population(n, 5)
    pop = snaps.snaps_index(ctx, x)
    try:
        ref = scores_of(pop, n, k, snaps.SNAPS_FP32 | snaps.SNAPS_INDEX_NONE)
        rep = snaps.snaps_autotune(pop, k)
        assert [e["d"] for e in rep] == [2, 3, 4]
        for e in rep:
            assert e["ms_brute"] > 0 and all(t > 0 for t in e["ms_grid"])
            widths = [1.0, np.float32(0.5), np.float32(1.0 / 3.0)]
            assert e["cell_mult"] in widths
            best = min(e["ms_grid"])
            assert e["grid"] == (best < e["ms_brute"])
            assert e["ms_grid"][widths.index(e["cell_mult"])] == best
        for prec in (snaps.SNAPS_FP32, snaps.SNAPS_FP32 | snaps.SNAPS_INDEX_GRID):
            got = scores_of(pop, n, k, prec)
            np.testing.assert_array_equal(got[0], ref[0])
            np.testing.assert_array_equal(got[1], ref[1])
        snaps.snaps_autotune_clear(ctx)
        got = scores_of(pop, n, k, snaps.SNAPS_FP32)
        np.testing.assert_array_equal(got[0], ref[0])
    finally:
        snaps.snaps_release(pop)


def test_autotune_rejects_bad_k(ctx):
    pop = snaps.snaps_index(ctx, snaps_inputs.population(500, 1))
    try:
        for k in (0, 33, -1):
            with pytest.raises(snaps.SnapsError) as e:
                snaps.snaps_autotune(pop, k)
            assert e.value.status == snaps.SNAPS_EINVAL
    finally:
        snaps.snaps_release(pop)


def test_tuned_choice_applies_to_lone_subspaces(ctx):
    # below SNAPS_GRID_AUTO_N the grid serves a lone subspace once the tuner
    # chose it, while subspaces that share a chunk stay in the tree join
    n = 20000
    pop = snaps.snaps_index(ctx, snaps_inputs.population(n, 6))
    try:
        rep = snaps.snaps_autotune(pop, 10)
        sc = torch.empty((32, 4, n), device="cuda")
        chunk0 = np.array([m for m in range(32) if bin(m).count("1") >= 2], dtype=np.uint16)

        def grid_launches(masks):
            snaps.snaps_trace(ctx, True)
            snaps.snaps_scores(pop, masks, 10, scores=sc[:masks.size])
            torch.cuda.synchronize()
            tr = snaps.snaps_trace_read(ctx)
            snaps.snaps_trace(ctx, False)
            return tr["grid"][1], tr["join_tree"][1]

        g_lone, _ = grid_launches(np.array([0b11], dtype=np.uint16))
        assert (g_lone > 0) == rep[0]["grid"]
        g_chunk, t_chunk = grid_launches(chunk0)
        assert g_chunk == 0 and t_chunk > 0
    finally:
        snaps.snaps_release(pop)


def tc_launches(ctx, pop, masks, n, precision):
    """Scores of one call, and its tensor-core and subspace-at-a-time launches."""
    sc = torch.empty((masks.size, 4, n), device="cuda")
    snaps.snaps_trace(ctx, True)
    snaps.snaps_scores(pop, masks, 10, precision=precision | snaps.SNAPS_INDEX_NONE, scores=sc)
    torch.cuda.synchronize()
    tr = snaps.snaps_trace_read(ctx)
    snaps.snaps_trace(ctx, False)
    return sc.cpu().numpy(), tr["join_tc"][1], tr["join_lane"][1]


def test_tc_blocks_need_their_minimum_fill(ctx):
    # a tensor-core block is formed only with at least the minimum fill of
    # subspaces; the rest take the plain routes and return the plain bits
    n = 4000
    pop = snaps.snaps_index(ctx, snaps_inputs.population(n, 7))
    try:
        few = snaps_inputs.mask_sample(40, 3)
        plain, t, _ = tc_launches(ctx, pop, few, n, snaps.SNAPS_FP32)
        assert t == 0
        got, t, lone = tc_launches(ctx, pop, few, n, snaps.SNAPS_TC_F16)  # built-in fill: 128
        assert t == 0 and lone > 0
        np.testing.assert_array_equal(got, plain)
        snaps.snaps_set_tc_min_fill(ctx, 1)
        got, t, _ = tc_launches(ctx, pop, few, n, snaps.SNAPS_TC_F16)
        assert t == 1
        np.testing.assert_array_equal(got[:, [0, 2, 3]], plain[:, [0, 2, 3]])
        np.testing.assert_allclose(got[:, 1], plain[:, 1], rtol=1e-5, atol=1e-6)
        snaps.snaps_set_tc_min_fill(ctx, snaps.SNAPS_TC_NEVER)
        got, t, _ = tc_launches(ctx, pop, few, n, snaps.SNAPS_TC_BF16)
        assert t == 0
        np.testing.assert_array_equal(got, plain)
        # one full block of 256 and a tail of 44 below the fill: one block on the
        # tensor cores, the tail (the highest dimensions) joined plain
        snaps.snaps_set_tc_min_fill(ctx, 0)
        many = snaps_inputs.mask_sample(300, 4)
        ref, _, _ = tc_launches(ctx, pop, many, n, snaps.SNAPS_FP32)
        got, t, lone = tc_launches(ctx, pop, many, n, snaps.SNAPS_TC_F16)
        assert t == 1 and lone > 0
        np.testing.assert_array_equal(got[:, [0, 2, 3]], ref[:, [0, 2, 3]])
        np.testing.assert_allclose(got[:, 1], ref[:, 1], rtol=1e-5, atol=1e-6)
        order = sorted(range(many.size), key=lambda m: (bin(int(many[m])).count("1"), int(many[m])))
        tail = order[256:]
        np.testing.assert_array_equal(got[tail], ref[tail])
        for bad in (-1, snaps.SNAPS_TC_NEVER + 1):
            with pytest.raises(snaps.SnapsError) as e:
                snaps.snaps_set_tc_min_fill(ctx, bad)
            assert e.value.status == snaps.SNAPS_EINVAL
    finally:
        snaps.snaps_set_tc_min_fill(ctx, 0)
        snaps.snaps_release(pop)


def test_autotune_tc_fill_applies(ctx):
    n = 20000
    pop = snaps.snaps_index(ctx, snaps_inputs.population(n, 8))
    try:
        rep = snaps.snaps_autotune_tc(pop, 10)
        assert rep["ms_block"] > 0 and rep["ms_lone"] > 0
        expect = min(snaps.SNAPS_TC_NEVER, max(1, int(np.ceil(rep["ms_block"] / rep["ms_lone"]))))
        assert abs(rep["min_fill"] - expect) <= 1  # ceil of the same ratio, in FP64 both
        fill = rep["min_fill"]
        if 2 <= fill <= 256:
            masks = snaps_inputs.mask_sample(fill, 9)
            _, t, _ = tc_launches(ctx, pop, masks, n, snaps.SNAPS_TC_F16)
            assert t == 1
            _, t, _ = tc_launches(ctx, pop, masks[:fill - 1], n, snaps.SNAPS_TC_F16)
            assert t == 0
        snaps.snaps_autotune_clear(ctx)  # back to the built-in fill
        _, t, _ = tc_launches(ctx, pop, snaps_inputs.mask_sample(127, 9), n, snaps.SNAPS_TC_F16)
        assert t == 0
        _, t, _ = tc_launches(ctx, pop, snaps_inputs.mask_sample(128, 9), n, snaps.SNAPS_TC_F16)
        assert t == 1
        with pytest.raises(snaps.SnapsError) as e:
            snaps.snaps_autotune_tc(pop, 10, precision=snaps.SNAPS_FP32)
        assert e.value.status == snaps.SNAPS_EINVAL
    finally:
        snaps.snaps_release(pop)
    wide = snaps.snaps_index(ctx, (snaps_inputs.population(500, 1) * 3.0).astype(np.float32), flags=0)
    try:
        with pytest.raises(snaps.SnapsError) as e:
            snaps.snaps_autotune_tc(wide, 10)
        assert e.value.status == snaps.SNAPS_EINVAL
    finally:
        snaps.snaps_release(wide)
