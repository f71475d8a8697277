"""The precision workload at its full size: N = 250,000 objects (seed 0), the
plain FP32 join against the three tensor-core forms (FP16, BF16 and TF32
high/low parts) on 256 subspaces -- eight whole 32-subspace chunks drawn with seed 1,
one full tensor-core block -- with k = 10 and eps = 0.05 sqrt(d).

Per form and per metric, against the FP64 oracle on 64 evenly spaced
queries of every subspace (band rules of tests/parity.py): eps counts, mean
eps distances and kNN mean distances, and the kNN lists of the kNN-join
entry point (the plain join) rank by rank.  The
in-degree of an object needs every query's list, which the oracle cannot
afford at this size: the tensor-core forms must return the plain form's
in-degrees bit for bit, and every subspace's in-degrees sum to N k.  The
largest error seen per metric is printed (pytest -s)."""
import numpy as np
import pytest

import oracle
import paper_2405_20176_b300 as snaps
import snaps_inputs
from parity import SCORE_RTOL, check_eps, check_knn, eps_bounds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, K = 250_000, 10
FORMS = {"fp32": snaps.SNAPS_FP32, "tc_f16": snaps.SNAPS_TC_F16, "tc_bf16": snaps.SNAPS_TC_BF16,
         "tc_tf32": snaps.SNAPS_TC_TF32}


def test_precision_workload_against_the_oracle():
    x = snaps_inputs.population(N, 0)
    masks = snaps_inputs.chunk_sample(8, 1)
    queries = np.linspace(0, N - 1, 64).round().astype(np.int64)
    qt = torch.from_numpy(queries).cuda()
    ctx = snaps.snaps_create(0)
    got = {}
    try:
        pop = snaps.snaps_index(ctx, torch.from_numpy(x).cuda())
        try:
            # kNN lists (plain FP32 join, which the kNN-join entry point runs)
            idx = torch.empty((masks.size, N, K), dtype=torch.int32, device="cuda")
            dist = torch.empty((masks.size, N, K), device="cuda")
            snaps.snaps_knn_selfjoin(pop, masks, K, idx, dist)
            torch.cuda.synchronize()
            lists = {"idx": idx[:, qt].cpu().numpy(), "dist": dist[:, qt].cpu().numpy()}
            del idx, dist
            for name, prec in FORMS.items():
                sc = torch.empty((masks.size, 4, N), device="cuda")
                snaps.snaps_trace(ctx, True)
                snaps.snaps_scores(pop, masks, K, precision=prec, scores=sc)
                torch.cuda.synchronize()
                tr = snaps.snaps_trace_read(ctx)
                snaps.snaps_trace(ctx, False)
                if prec != snaps.SNAPS_FP32:
                    assert tr["join_tc"][1] == 1, "one full block on the tensor cores"
                assert torch.all(sc[:, 2].to(torch.int64).sum(dim=1) == N * K)
                got[name] = {"indeg": sc[:, 2].cpu().numpy(), "q": sc[:, :, qt].cpu().numpy()}
                del sc
        finally:
            snaps.snaps_release(pop)
    finally:
        snaps.snaps_destroy(ctx)
    for name in ("tc_f16", "tc_bf16", "tc_tf32"):
        np.testing.assert_array_equal(got[name]["indeg"], got["fp32"]["indeg"], err_msg=name)

    x64 = oracle.normalise(x).astype(np.float64)
    err = {name: {"eps_count_differ": 0, "eps_count_in_band": 0, "eps_mean_max_rel": 0.0,
                  "knn_mean_max_rel": 0.0} for name in FORMS}
    knn_rows_in_band = 0
    for s, mask in enumerate(masks):
        mask = int(mask)
        e2 = oracle.default_eps2(mask)
        j = oracle.join(x64, mask, K, e2, queries=queries)
        lo, hi = eps_bounds(x64, mask, e2, queries=queries)
        sure = lo == hi
        c = j.eps_count
        ref_mean = np.where(c > 0, j.eps_sum / np.maximum(c, 1), 0.0)
        ref_knn = np.sqrt(j.knn_d2).mean(axis=1)
        for name in FORMS:
            g = got[name]
            q = g["q"][s]
            err[name]["eps_count_in_band"] += check_eps(q[0], q[1], j, lo, hi)
            err[name]["eps_count_differ"] += int((q[0] != c).sum())
            ok = sure & (q[0] == c) & (c > 0)
            if ok.any():
                rel = np.abs(q[1][ok] - ref_mean[ok]) / ref_mean[ok]
                err[name]["eps_mean_max_rel"] = max(err[name]["eps_mean_max_rel"], float(rel.max()))
            np.testing.assert_allclose(q[3], ref_knn, rtol=SCORE_RTOL, atol=1e-12)
            err[name]["knn_mean_max_rel"] = max(err[name]["knn_mean_max_rel"],
                                                float((np.abs(q[3] - ref_knn) / ref_knn).max()))
        knn_rows_in_band += check_knn(x64, mask, lists["idx"][s], lists["dist"][s], j.knn_idx, j.knn_d2,
                                      queries=queries)
    print(f"\nprecision workload N={N}, {masks.size} subspaces, {queries.size} queries each; "
          f"kNN lists rank by rank, {knn_rows_in_band} rows with a neighbour in the band:")
    for name in FORMS:
        print(f"  {name}: {err[name]}")
    for name in FORMS:
        assert err[name]["eps_mean_max_rel"] <= SCORE_RTOL
