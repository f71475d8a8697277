"""snaps_scores_static, the scoring call for callers that cannot let a
library allocate device memory: through the C ABI, two calls in a row, each
equal to the regular snaps_index + snaps_scores result.  This file is named
to run last, so a failure here stops a `-x` run only after every other test."""
import numpy as np
import pytest

import paper_2405_20176_b300 as snaps
import snaps_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _regular(x, masks, k, top_n):
    ctx = snaps.snaps_create(0)
    try:
        pop = snaps.snaps_index(ctx, x)
        try:
            sc = np.zeros((masks.size, 4, x.shape[0]), dtype=np.float32)
            tp = np.zeros((masks.size, 4, top_n), dtype=np.int32)
            snaps.snaps_scores(pop, masks, k, scores=sc, top=tp, top_n=top_n)
            return sc, tp
        finally:
            snaps.snaps_release(pop)
    finally:
        snaps.snaps_destroy(ctx)


def test_static_scoring_matches_regular_twice_in_a_row():
    allm = snaps_inputs.all_masks()
    cases = [
        (snaps_inputs.population(2000, 0), np.concatenate([allm[(allm >> 5) == 0b1111111111],
                                                           [0b11, 0b101000000000001]]), 10),
        (snaps_inputs.population(1500, 7), snaps_inputs.mask_sample(70, 4), 5),
    ]
    outs = []
    for x, masks, k in cases:
        masks = masks.astype(np.uint16)
        n = x.shape[0]
        feat = torch.from_numpy(x).cuda()
        sc = torch.full((masks.size, 4, n), -1.0, device="cuda")
        tp = torch.full((masks.size, 4, 100), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        snaps.snaps_scores_static(0, feat, masks, k, scores=sc, top=tp, top_n=100)
        outs.append((sc.cpu().numpy(), tp.cpu().numpy()))
    for (x, masks, k), (sc, tp) in zip(cases, outs):
        ref_sc, ref_tp = _regular(x, masks.astype(np.uint16), k, 100)
        np.testing.assert_array_equal(sc, ref_sc)
        np.testing.assert_array_equal(tp, ref_tp)


def test_static_scoring_rejects_sizes_beyond_its_limits():
    x = torch.zeros((snaps.SNAPS_STATIC_MAX_N + 1, 15), device="cuda")
    sc = torch.empty((1, 4, snaps.SNAPS_STATIC_MAX_N + 1), device="cuda")
    with pytest.raises(snaps.SnapsError) as ei:
        snaps.snaps_scores_static(0, x, [0b11], 10, scores=sc)
    assert ei.value.status == snaps.SNAPS_EINVAL
    assert "allocation-free" in str(ei.value)
    host = np.zeros((100, 4), dtype=np.float32)
    with pytest.raises(snaps.SnapsError) as ei:
        snaps.snaps_scores_static(0, host, [0b11], 10, scores=np.zeros((1, 4, 100), np.float32))
    assert ei.value.status == snaps.SNAPS_EINVAL
