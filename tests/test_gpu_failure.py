"""Failure detection without a GPU fault: the tensor-core join's pipeline
waits are bounded, and with the bound set to a single try they give up for
real (a copy, B rows or an MMA batch not ready yet).  The call must return
SNAPS_ETIMEOUT -- every warp leaves in order, waiting for its own copies and
MMAs in flight and freeing tensor memory -- and the same context must then
give correct results with the default bound."""
import numpy as np
import pytest

import oracle
import paper_2405_20176_b300 as snaps
import snaps_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_waits_give_up_and_the_context_recovers():
    ctx = snaps.snaps_create(0)
    try:
        snaps.snaps_set_tc_min_fill(ctx, 1)  # the 40 subspaces form a tensor-core block
        x = snaps_inputs.population(3000, 5)
        masks = snaps_inputs.mask_sample(40, 5)
        pop = snaps.snaps_index(ctx, x)
        try:
            n, m = x.shape[0], masks.size
            plain = np.zeros((m, 4, n), dtype=np.float32)
            snaps.snaps_scores(pop, masks, 10, scores=plain)
            for form in (snaps.SNAPS_TC_F16, snaps.SNAPS_TC_BF16, snaps.SNAPS_TC_TF32):
                snaps.snaps_set_wait_limit(ctx, 1)
                out = np.zeros((m, 4, n), dtype=np.float32)
                with pytest.raises(snaps.SnapsError) as ei:
                    snaps.snaps_scores(pop, masks, 10, precision=form, scores=out)
                assert ei.value.status == snaps.SNAPS_ETIMEOUT
                # the default bound again: the context works and the results hold
                snaps.snaps_set_wait_limit(ctx, 0)
                snaps.snaps_scores(pop, masks, 10, precision=form, scores=out)
                np.testing.assert_array_equal(out[:, [0, 2, 3]], plain[:, [0, 2, 3]])
                np.testing.assert_allclose(out[:, 1], plain[:, 1], rtol=1e-5, atol=1e-6)
            # and the plain path on the same context agrees with the oracle
            snaps.snaps_scores(pop, masks[:2], 10, scores=plain[:2])
            r = oracle.subspace(oracle.normalise(x), int(masks[0]), 10)
            np.testing.assert_allclose(plain[0][3], r.scores[oracle.KNN_MEAN], rtol=1e-5)
        finally:
            snaps.snaps_release(pop)
    finally:
        snaps.snaps_destroy(ctx)
