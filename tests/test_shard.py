"""Subspaces shared out across ranks (Sec. 3.8.2), on the CPU: the
longest-first least-loaded assignment covers every requested subspace exactly
once, keeps every 32-subspace chunk on one rank, balances the all-subspace
workload, and two gloo ranks gather their per-subspace results on rank 0
into exactly what one rank computing everything would hold."""
import os
import socket

import numpy as np
import pytest

import snaps_inputs
from paper_2405_20176_b300 import shard

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_all_subspaces_once_and_balances(world):
    masks = snaps_inputs.all_masks()
    parts, load = shard.partition(masks, 31693, world)
    allpos = np.concatenate(parts)
    assert allpos.size == masks.size
    assert np.array_equal(np.sort(allpos), np.arange(masks.size))
    # whole chunks: no high part on two ranks
    owner = {}
    for r, p in enumerate(parts):
        for h in set((masks[p] >> 5).tolist()):
            assert owner.setdefault(h, r) == r
    # the longest-first greedy is within one unit of the mean load here
    biggest = max(c for c, _ in shard.units(masks, 31693))
    assert max(load) - min(load) <= biggest
    assert max(load) <= 1.01 * (sum(load) / world) + biggest


def test_partition_is_deterministic_and_handles_lone_and_repeated_subspaces():
    rng = np.random.default_rng(3)
    masks = snaps_inputs.mask_sample(200, 9)
    masks = np.concatenate([masks, masks[:5]])      # repeats
    masks = masks[rng.permutation(masks.size)]
    a, _ = shard.partition(masks, 5000, 3)
    b, _ = shard.partition(masks, 5000, 3)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert np.array_equal(np.sort(np.concatenate(a)), np.arange(masks.size))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fake_results(masks, positions, n):
    """Stand-in per-subspace outputs that depend on the subspace alone."""
    m = masks[positions].astype(np.float64)
    scores = (m[:, None, None] * 1e-3 + np.arange(4)[None, :, None] + np.arange(n)[None, None, :] * 1e-6)
    top = (masks[positions].astype(np.int32)[:, None, None] + np.arange(4 * 7).reshape(1, 4, 7)) % n
    return {"scores": scores.astype(np.float32), "top": top.astype(np.int32)}


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    from paper_2405_20176_b300 import shard as sh
    import snaps_inputs as si
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        masks = si.mask_sample(300, 4)
        n = 50
        parts, _ = sh.partition(masks, n, world)
        mine = parts[rank]
        got = sh.gather(_fake_results(masks, mine, n), mine, masks.size, rank, world, tdist)
        if rank == 0:
            out["gathered"] = got
            out["sizes"] = [p.size for p in parts]
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_two_ranks_gather_what_one_rank_computes():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    masks = snaps_inputs.mask_sample(300, 4)
    single = _fake_results(masks, np.arange(masks.size), 50)
    assert all(s > 0 for s in res["sizes"]), "both ranks got work"
    for name in single:
        np.testing.assert_array_equal(res["gathered"][name], single[name])


def test_gather_rejects_overlap_and_gaps():
    masks = snaps_inputs.mask_sample(10, 1)
    full = _fake_results(masks, np.arange(10), 5)
    assert np.array_equal(shard.gather(full, np.arange(10), 10, 0, 1)["top"], full["top"])
    with pytest.raises(ValueError):
        shard.gather(_fake_results(masks, np.arange(9), 5), np.arange(9), 10, 0, 1)
