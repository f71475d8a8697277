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
