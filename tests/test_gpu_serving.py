"""The continuous-batching request loop (snaps_submit / snaps_poll): each
request's result is bit-identical alone (a synchronous snaps_scores call) and
in a mix of concurrent requests of different sizes, subspace sets and k;
admission, cancellation and in-use populations behave as documented."""
import numpy as np
import pytest

import paper_2405_20176_b300 as snaps
import snaps_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _request_mix(seed, count):
    rng = np.random.default_rng(seed)
    allm = snaps_inputs.all_masks()
    out = []
    for r in range(count):
        n = int(np.exp(rng.uniform(np.log(300), np.log(4000))))
        n_masks = int(rng.integers(1, 80))
        d = rng.integers(2, 16, size=n_masks)
        masks = []
        for dd in d:
            feats = rng.choice(15, size=int(dd), replace=False)
            masks.append(int(sum(1 << int(f) for f in feats)))
        if r % 3 == 0:   # some requests take whole dense chunks
            h = int(rng.integers(1, 1024))
            masks += [int(m) for m in allm[(allm >> 5) == h]]
        k = int(rng.choice([5, 10, 20]))
        out.append((n, int(rng.integers(0, 1 << 30)), np.array(masks, dtype=np.uint16), k))
    return out


def test_results_alone_equal_results_in_the_mix():
    ctx = snaps.snaps_create(0)
    try:
        snaps.snaps_set_slots(ctx, 4)
        mix = _request_mix(5, 16)
        pops, reqs, outs = [], [], []
        for n, seed, masks, k in mix:
            pop = snaps.snaps_index(ctx, snaps_inputs.population(n, seed))
            pops.append(pop)
            sc = torch.empty((masks.size, 4, n), device="cuda")
            tp = torch.empty((masks.size, 4, min(100, n)), dtype=torch.int32, device="cuda")
            nz = np.zeros((masks.size, 4, n), dtype=np.float32)     # a host output too
            outs.append((sc, tp, nz))
        torch.cuda.synchronize()
        for (n, seed, masks, k), pop, (sc, tp, nz) in zip(mix, pops, outs):
            reqs.append(snaps.snaps_submit(ctx, pop, masks, k, scores=sc, norm=nz, top=tp,
                                           top_n=min(100, n)))
        lat = []
        for r in reqs:
            res = snaps.snaps_poll(ctx, r, timeout_us=-1)
            assert res.status == snaps.SNAPS_OK
            assert res.latency_us >= res.queue_us >= 0
            lat.append(res.latency_us)
        torch.cuda.synchronize()
        for (n, seed, masks, k), pop, (sc, tp, nz) in zip(mix, pops, outs):
            a_sc = np.zeros((masks.size, 4, n), dtype=np.float32)
            a_nz = np.zeros_like(a_sc)
            a_tp = np.zeros((masks.size, 4, min(100, n)), dtype=np.int32)
            snaps.snaps_scores(pop, masks, k, scores=a_sc, norm=a_nz, top=a_tp, top_n=min(100, n))
            np.testing.assert_array_equal(sc.cpu().numpy(), a_sc)
            np.testing.assert_array_equal(tp.cpu().numpy(), a_tp)
            np.testing.assert_array_equal(nz, a_nz)
        for pop in pops:
            snaps.snaps_release(pop)
    finally:
        snaps.snaps_destroy(ctx)


def test_cancel_release_and_admission():
    ctx = snaps.snaps_create(0, 2 << 30)
    try:
        snaps.snaps_set_slots(ctx, 1)
        pop = snaps.snaps_index(ctx, snaps_inputs.population(6000, 3))
        allm = snaps_inputs.all_masks()[:512]
        outs = [torch.empty((allm.size, 4, 6000), device="cuda") for _ in range(3)]
        torch.cuda.synchronize()
        reqs = [snaps.snaps_submit(ctx, pop, allm, 10, scores=o) for o in outs]
        # the last request is still queued behind the single slot
        snaps.snaps_cancel(ctx, reqs[2])
        with pytest.raises(snaps.SnapsError) as ei:
            snaps.snaps_release(pop)
        assert ei.value.status == snaps.SNAPS_EBUSY
        st = [snaps.snaps_poll(ctx, r, -1).status for r in reqs]
        assert st == [snaps.SNAPS_OK, snaps.SNAPS_OK, snaps.SNAPS_ECANCELED]
        with pytest.raises(snaps.SnapsError) as ei:
            snaps.snaps_poll(ctx, reqs[0], 0)      # a finished ticket is forgotten
        assert ei.value.status == snaps.SNAPS_EINVAL
        # a request larger than the whole budget is refused at submit
        big = torch.empty(1, device="cuda")
        with pytest.raises(snaps.SnapsError) as ei:
            snaps.snaps_submit(ctx, pop, snaps_inputs.all_masks(), 10, top=big, top_n=100)
        assert ei.value.status == snaps.SNAPS_ENOMEM
        snaps.snaps_release(pop)
    finally:
        snaps.snaps_destroy(ctx)


def test_poll_timeout_returns_eagain():
    ctx = snaps.snaps_create(0)
    try:
        pop = snaps.snaps_index(ctx, snaps_inputs.population(20000, 8))
        masks = snaps_inputs.all_masks()[:2048]
        out = torch.empty((masks.size, 4, 20000), device="cuda")
        torch.cuda.synchronize()
        r = snaps.snaps_submit(ctx, pop, masks, 10, scores=out)
        first = snaps.snaps_poll(ctx, r, 0)
        res = first if first is not None else snaps.snaps_poll(ctx, r, -1)
        assert res.status == snaps.SNAPS_OK
        assert res.objects_x_subspaces == 20000 * masks.size
        snaps.snaps_release(pop)
    finally:
        snaps.snaps_destroy(ctx)


def test_small_requests_share_launches():
    """Continuous batching: small requests on several populations, with
    different k, queued behind a slot that is busy, are joined by shared
    launches; each result is the same as the request alone."""
    ctx = snaps.snaps_create(0)
    try:
        snaps.snaps_set_slots(ctx, 1)
        rng = np.random.default_rng(11)
        allm = snaps_inputs.all_masks()
        # a large request keeps the one slot busy while the small ones queue
        big_pop = snaps.snaps_index(ctx, snaps_inputs.population(9000, 2))
        big_out = torch.empty((512, 4, 9000), device="cuda")
        pops = [snaps.snaps_index(ctx, snaps_inputs.population(int(n), int(s)))
                for n, s in [(700, 1), (1500, 2), (2300, 3)]]
        sizes = [700, 1500, 2300]
        small = []
        for r in range(24):
            pi = int(rng.integers(0, 3))
            masks = rng.choice(allm, size=int(rng.integers(1, 6)), replace=False).astype(np.uint16)
            k = int(rng.choice([5, 10, 20]))
            n = sizes[pi]
            sc = torch.empty((masks.size, 4, n), device="cuda")
            tp = torch.empty((masks.size, 4, min(100, n)), dtype=torch.int32, device="cuda")
            small.append((pi, masks, k, sc, tp))
        torch.cuda.synchronize()
        tickets = [snaps.snaps_submit(ctx, big_pop, allm[:512], 10, scores=big_out)]
        for pi, masks, k, sc, tp in small:
            tickets.append(snaps.snaps_submit(ctx, pops[pi], masks, k, scores=sc, top=tp,
                                              top_n=min(100, sizes[pi])))
        for t in tickets:
            assert snaps.snaps_poll(ctx, t, -1).status == snaps.SNAPS_OK
        launches, served = snaps.snaps_serving_stats(ctx)
        assert launches >= 1 and served >= 2 * launches, (launches, served)
        torch.cuda.synchronize()
        for pi, masks, k, sc, tp in small:
            n = sizes[pi]
            a_sc = np.zeros((masks.size, 4, n), dtype=np.float32)
            a_tp = np.zeros((masks.size, 4, min(100, n)), dtype=np.int32)
            snaps.snaps_scores(pops[pi], masks, k, scores=a_sc, top=a_tp, top_n=min(100, n))
            np.testing.assert_array_equal(sc.cpu().numpy(), a_sc)
            np.testing.assert_array_equal(tp.cpu().numpy(), a_tp)
        for p in pops + [big_pop]:
            snaps.snaps_release(p)
    finally:
        snaps.snaps_destroy(ctx)


def test_large_request_runs_in_parts_and_lets_small_ones_through():
    """A request of more than 2e11 pair evaluations runs in parts of its
    subspace list; small requests queued behind it on the one slot are served
    between parts, so they finish before it does.  Every result equals the
    request alone."""
    ctx = snaps.snaps_create(0)
    try:
        snaps.snaps_set_slots(ctx, 1)
        allm = snaps_inputs.all_masks()
        big_n = 20000
        big_pop = snaps.snaps_index(ctx, snaps_inputs.population(big_n, 4))
        big_masks = allm[::16][:1536]          # 4e8 pairs x 1,536 subspaces: three parts or more
        big_sc = torch.empty((big_masks.size, 4, big_n), device="cuda")
        big_tp = np.zeros((big_masks.size, 4, 100), dtype=np.int32)  # a host output too
        pop = snaps.snaps_index(ctx, snaps_inputs.population(900, 5))
        rng = np.random.default_rng(4)
        small = []
        for _ in range(6):
            masks = rng.choice(allm, size=3, replace=False).astype(np.uint16)
            small.append((masks, torch.empty((3, 4, 900), device="cuda")))
        torch.cuda.synchronize()
        t_big = snaps.snaps_submit(ctx, big_pop, big_masks, 10, scores=big_sc, top=big_tp, top_n=100)
        t_small = [snaps.snaps_submit(ctx, pop, m, 10, scores=sc) for m, sc in small]
        r_small = [snaps.snaps_poll(ctx, t, -1) for t in t_small]
        r_big = snaps.snaps_poll(ctx, t_big, -1)
        assert r_big.status == snaps.SNAPS_OK and all(r.status == snaps.SNAPS_OK for r in r_small)
        # every small request was done while the large one still ran
        assert max(r.latency_us for r in r_small) < r_big.latency_us
        torch.cuda.synchronize()
        a_sc = np.zeros((big_masks.size, 4, big_n), dtype=np.float32)
        a_tp = np.zeros_like(big_tp)
        snaps.snaps_scores(big_pop, big_masks, 10, scores=a_sc, top=a_tp, top_n=100)
        np.testing.assert_array_equal(big_sc.cpu().numpy(), a_sc)
        np.testing.assert_array_equal(big_tp, a_tp)
        for masks, sc in small:
            a = np.zeros((3, 4, 900), dtype=np.float32)
            snaps.snaps_scores(pop, masks, 10, scores=a)
            np.testing.assert_array_equal(sc.cpu().numpy(), a)
        snaps.snaps_release(pop)
        snaps.snaps_release(big_pop)
    finally:
        snaps.snaps_destroy(ctx)
