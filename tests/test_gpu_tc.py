"""The tensor-core filtered joins (SNAPS_TC_F16, SNAPS_TC_BF16, SNAPS_TC_TF32) against the
plain FP32 path and the FP64 oracle, across block fills, subspace mixes, k,
ragged N and extreme radii (every candidate passing stresses the exact
recompute).  eps counts, kNN lists, in-degrees and kNN mean distances are the
plain path's bits (every decision near eps or the k-th distance is made on the
canonical FP32 distance); the mean eps distance takes the accumulator's
distances and agrees to 1e-5 relative (plus two quantisation steps of
eps / 2^20); its ranking may differ only where keys tie within that."""
import numpy as np
import pytest

import oracle
import paper_2405_20176_b300 as snaps
import snaps_inputs
from parity import SCORE_RTOL, check_eps, check_knn, check_norm, check_top

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = snaps.snaps_create(0)
    # these tests exercise the tensor-core kernel itself: every block is formed
    # however few subspaces it carries
    snaps.snaps_set_tc_min_fill(c, 1)
    yield c
    snaps.snaps_destroy(c)


def run_both(ctx, x, masks, k, eps=None, top_n=100):
    masks = np.asarray(masks, dtype=np.uint16)
    pop = snaps.snaps_index(ctx, x)
    try:
        n = x.shape[0]
        top_n = min(top_n, n)
        out = {}
        for prec in (snaps.SNAPS_FP32, snaps.SNAPS_TC_F16, snaps.SNAPS_TC_BF16, snaps.SNAPS_TC_TF32):
            sc = np.zeros((masks.size, 4, n), dtype=np.float32)
            nz = np.zeros_like(sc)
            tp = np.zeros((masks.size, 4, top_n), dtype=np.int32)
            snaps.snaps_scores(pop, masks, k, eps=eps, precision=prec, scores=sc, norm=nz,
                               top=tp, top_n=top_n)
            out[prec] = (sc, nz, tp)
        return out
    finally:
        snaps.snaps_release(pop)


SAME = [oracle.EPS_COUNT, oracle.KNN_INDEG, oracle.KNN_MEAN]


def assert_tc_matches_plain(out, eps2):
    """eps2: per-subspace squared radius (the quantisation step of the mean
    eps distance is sqrt(eps2) / 2^20)."""
    a_sc, a_nz, a_tp = out[snaps.SNAPS_FP32]
    step = np.sqrt(np.maximum(np.asarray(eps2, dtype=np.float64), 0.0)) / 2.0 ** 20
    for form in (snaps.SNAPS_TC_F16, snaps.SNAPS_TC_BF16, snaps.SNAPS_TC_TF32):
        sc, nz, tp = out[form]
        np.testing.assert_array_equal(sc[:, SAME], a_sc[:, SAME], err_msg=f"metrics, form {form}")
        np.testing.assert_array_equal(nz[:, SAME], a_nz[:, SAME], err_msg=f"normalised, form {form}")
        np.testing.assert_array_equal(tp[:, SAME], a_tp[:, SAME], err_msg=f"top lists, form {form}")
        for s in range(sc.shape[0]):
            np.testing.assert_allclose(sc[s, 1], a_sc[s, 1], rtol=SCORE_RTOL, atol=2 * step[s],
                                       err_msg=f"eps mean, subspace {s}, form {form}")
            check_top(tp[s, oracle.EPS_MEAN], a_sc[s].astype(np.float64), a_tp[s, oracle.EPS_MEAN],
                      oracle.EPS_MEAN)
            check_norm(nz[s], sc[s], a_sc[s].astype(np.float64))


def eps2_of(masks, eps=None):
    masks = np.asarray(masks, dtype=np.uint16)
    if eps is None:
        return np.array([oracle.default_eps2(int(m)) for m in masks])
    return np.asarray(eps, dtype=np.float32).astype(np.float64) ** 2


@pytest.mark.parametrize("n,seed", [(2000, 0), (257, 1), (513, 2), (1100, 3)])
def test_tc_equals_plain_on_mixed_subspaces(ctx, n, seed):
    allm = snaps_inputs.all_masks()
    masks = np.concatenate([allm[(allm >> 5) == 0b1111111111], snaps_inputs.mask_sample(50, seed),
                            [0b11, (1 << 15) - 1]])
    assert_tc_matches_plain(run_both(ctx, snaps_inputs.population(n, seed), masks, 10), eps2_of(masks))


@pytest.mark.parametrize("k", [1, 5, 16, 17, 32])
def test_tc_k_range(ctx, k):
    masks = snaps_inputs.mask_sample(70, 10 + k)
    assert_tc_matches_plain(run_both(ctx, snaps_inputs.population(700, 20 + k), masks, k), eps2_of(masks))


def test_tc_extreme_radii_and_large_k(ctx):
    # eps beyond the diameter: every candidate passes the filter and the kNN
    # buffers overflow mid-tile; tiny eps: only duplicates
    x = snaps_inputs.population(900, 31)
    x[5] = x[17]
    masks = np.array([0b11, 0b111, 0b1010101010101, (1 << 15) - 1, 0b110000000000011], dtype=np.uint16)
    big, tiny = [4.0] * 5, [0.0, 1e-9, 0.0, 1e-9, 0.0]
    assert_tc_matches_plain(run_both(ctx, x, masks, 32, eps=big), eps2_of(masks, big))
    assert_tc_matches_plain(run_both(ctx, x, masks, 10, eps=tiny), eps2_of(masks, tiny))


@pytest.mark.parametrize("form", ["f16", "bf16", "tf32"])
def test_tc_matches_oracle(ctx, form):
    prec = {"f16": snaps.SNAPS_TC_F16, "bf16": snaps.SNAPS_TC_BF16, "tf32": snaps.SNAPS_TC_TF32}[form]
    x = snaps_inputs.population(1500, 41)
    masks = snaps_inputs.mask_sample(12, 41)
    pop = snaps.snaps_index(ctx, x)
    try:
        n, m = 1500, masks.size
        idx = torch.empty((m, n, 10), dtype=torch.int32, device="cuda")
        dist = torch.empty((m, n, 10), device="cuda")
        sc = np.zeros((m, 4, n), dtype=np.float32)
        nz = np.zeros((m, 4, n), dtype=np.float32)
        tp = np.zeros((m, 4, 100), dtype=np.int32)
        snaps.snaps_scores(pop, masks, 10, precision=prec, scores=sc, norm=nz, top=tp, top_n=100)
        snaps.snaps_knn_selfjoin(pop, masks, 10, idx, dist)
        torch.cuda.synchronize()
    finally:
        snaps.snaps_release(pop)
    xn = oracle.normalise(x)
    x64 = xn.astype(np.float64)
    for s, mask in enumerate(masks):
        r = oracle.subspace(xn, int(mask), 10)
        check_knn(x64, int(mask), idx[s].cpu().numpy(), dist[s].cpu().numpy(),
                  r.join.knn_idx, r.join.knn_d2)
        e2 = oracle.default_eps2(int(mask))
        lo = oracle.join(x64, int(mask), 0, e2 * (1 - 2e-6)).eps_count
        hi = oracle.join(x64, int(mask), 0, e2 * (1 + 2e-6)).eps_count
        check_eps(sc[s][0].astype(np.int64), sc[s][1], oracle.join(x64, int(mask), 0, e2), lo, hi)
        np.testing.assert_allclose(sc[s][3], r.scores[oracle.KNN_MEAN], rtol=1e-5)
        for mm in (oracle.EPS_MEAN, oracle.KNN_MEAN):
            check_top(tp[s][mm], r.scores, r.top[mm], mm)
        check_norm(nz[s], sc[s], r.scores, r.normalised)


def test_tc_rejects_wide_features(ctx):
    x = (snaps_inputs.population(300, 3) * 10).astype(np.float32)
    pop = snaps.snaps_index(ctx, x, flags=0)
    try:
        for prec in (snaps.SNAPS_TC_F16, snaps.SNAPS_TC_BF16, snaps.SNAPS_TC_TF32, 4):
            with pytest.raises(snaps.SnapsError) as ei:
                snaps.snaps_scores(pop, [0b11], 5, precision=prec,
                                   scores=np.zeros((1, 4, 300), np.float32))
            assert ei.value.status == snaps.SNAPS_EINVAL
    finally:
        snaps.snaps_release(pop)
