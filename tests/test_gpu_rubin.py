"""Rubin scale: N = 5,000,000 objects (seed 0), two of the two-feature
subspaces through the grid index in the benchmark's call, k = 10,
eps = 0.05 sqrt(2).  Invariants on both subspaces, and 64 evenly spaced
queries against the FP64 oracle under the band rules of tests/parity.py:
eps counts and means, kNN mean distances, and the kNN lists rank by rank."""
import numpy as np
import pytest

import oracle
import paper_2405_20176_b300 as snaps
import snaps_inputs
from parity import SCORE_RTOL, check_eps, check_knn, eps_bounds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, K = 5_000_000, 10


def test_rubin_scale_pairs():
    x = snaps_inputs.population(N, 0)
    masks = np.array([0b11, 0b110000000000000], dtype=np.uint16)
    ctx = snaps.snaps_create(0)
    try:
        pop = snaps.snaps_index(ctx, torch.from_numpy(x).cuda())
        sc = torch.empty((masks.size, 4, N), dtype=torch.float32, device="cuda")
        snaps.snaps_trace(ctx, True)
        snaps.snaps_scores(pop, masks, K, scores=sc)
        torch.cuda.synchronize()
        tr = snaps.snaps_trace_read(ctx)
        idx = torch.empty((masks.size, N, K), dtype=torch.int32, device="cuda")
        dist = torch.empty((masks.size, N, K), dtype=torch.float32, device="cuda")
        snaps.snaps_knn_selfjoin(pop, masks, K, idx, dist)
        torch.cuda.synchronize()
        snaps.snaps_release(pop)
        assert tr["grid"][1] > 0, "the grid index serves two-feature subspaces at this size"
        assert torch.all(sc[:, 2].to(torch.int64).sum(dim=1) == N * K)
        assert torch.all(sc[:, 0].to(torch.int64).sum(dim=1) % 2 == 0)
        g = sc.cpu().numpy()
        queries = np.linspace(0, N - 1, 64).round().astype(np.int64)
        q_idx = idx[:, queries].cpu().numpy()
        q_dist = dist[:, queries].cpu().numpy()
        del idx, dist
    finally:
        snaps.snaps_destroy(ctx)
    x64 = oracle.normalise(x).astype(np.float64)
    for s, mask in enumerate(masks):
        mask = int(mask)
        e2 = oracle.default_eps2(mask)
        j = oracle.join(x64, mask, K, e2, queries=queries)
        lo, hi = eps_bounds(x64, mask, e2, queries=queries)
        check_eps(g[s, 0][queries], g[s, 1][queries], j, lo, hi)
        np.testing.assert_allclose(g[s, 3][queries], np.sqrt(j.knn_d2).mean(axis=1), rtol=SCORE_RTOL,
                                   atol=1e-12)
        check_knn(x64, mask, q_idx[s], q_dist[s], j.knn_idx, j.knn_d2, queries=queries)
