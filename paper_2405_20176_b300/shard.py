"""Subspaces shared out across GPUs, one process per GPU (Sec. 3.8.2).

The paper assigns feature spaces to GPUs dynamically, the next one to the
least loaded GPU.  Here every rank computes the same static assignment
without talking to the others: units are taken in order of falling cost
and each goes to the rank with the least cost so far (the longest-first
greedy form of least-loaded scheduling, within 4/3 of the best assignment).
A unit is a whole 32-subspace chunk -- the subspaces (H << 5) | L that share
one high part H, which the subspace-batched join evaluates together -- when
four or more of its subspaces are requested (the library's threshold for that
kernel), and otherwise a single subspace; splitting a chunk would repeat its
shared arithmetic on two GPUs.  No data
moves between ranks while they compute; per-subspace results are gathered on
rank 0 afterwards.

The cost model counts candidate pairs times the work per pair of the kernel
that takes the unit (in FP32-pipe operations, as the library's kernels spend
them): about 45 per pair for a chunk's shared walk plus 3 per requested
subspace for its events, and 1.25 d + 8 per pair for a subspace joined on its
own.  It only has to rank units against each other; its error moves load
between ranks but never changes a result.

Host-side plumbing only: no arithmetic of the method lives here.
"""
from __future__ import annotations

from collections import defaultdict

import numpy as np

LOW_BITS = 5  # subspaces per chunk: 2^5
TREE_MIN_ACTIVE = 4  # requested subspaces from which a chunk takes the subspace-batched join


def units(masks, n: int):
    """The scheduling units of a request: a list of (cost, positions), the
    positions indexing `masks`.  A subspace requested twice forms a unit of
    its own for the repeat (it is joined on its own, as the library does)."""
    masks = np.asarray(masks, dtype=np.uint16)
    by_chunk = defaultdict(list)
    seen = set()
    extra = []
    for pos, m in enumerate(masks.tolist()):
        if m in seen:
            extra.append(pos)
            continue
        seen.add(m)
        by_chunk[m >> LOW_BITS].append(pos)
    pairs = float(n) * float(n - 1)
    out = []
    for _, members in sorted(by_chunk.items()):
        if len(members) >= TREE_MIN_ACTIVE:
            out.append((pairs * (45.0 + 3.0 * len(members)), members))
        else:
            extra.extend(members)
    for pos in sorted(extra):
        d = bin(int(masks[pos])).count("1")
        out.append((pairs * (1.25 * d + 8.0), [pos]))
    return out


def partition(masks, n: int, world: int):
    """Positions of `masks` for each of `world` ranks (a list of sorted int64
    arrays), and each rank's estimated cost.  Deterministic: every rank gets
    the same answer from the same arguments."""
    if world < 1:
        raise ValueError("world must be >= 1")
    us = units(masks, n)
    # falling cost, ties by first position, so that the order is total
    us.sort(key=lambda u: (-u[0], u[1][0]))
    load = [0.0] * world
    share = [[] for _ in range(world)]
    for cost, members in us:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += cost
        share[r].extend(members)
    return [np.array(sorted(s), dtype=np.int64) for s in share], load


def gather(local: dict, positions, n_total: int, rank: int, world: int, dist=None):
    """Collect per-subspace outputs on rank 0.

    local: {name: array whose first axis runs over this rank's subspaces, in
    the order of `positions`}.  Returns, on rank 0, {name: array whose first
    axis runs over all n_total subspaces in request order}; None elsewhere.
    Uses torch.distributed's object gather (host side) when world > 1."""
    mine = (np.asarray(positions, dtype=np.int64), {k: np.asarray(v) for k, v in local.items()})
    if world == 1:
        parts = [mine]
    else:
        parts = [None] * world if rank == 0 else None
        dist.gather_object(mine, parts, dst=0)
        if rank != 0:
            return None
    out = {}
    for name in local:
        first = next(p[1][name] for p in parts if p[1][name].shape[0] > 0) if any(
            p[1][name].shape[0] > 0 for p in parts) else np.asarray(local[name])
        full = np.zeros((n_total,) + first.shape[1:], dtype=first.dtype)
        filled = np.zeros(n_total, dtype=bool)
        for pos, arrays in parts:
            if filled[pos].any():
                raise ValueError("a subspace was computed on two ranks")
            full[pos] = arrays[name]
            filled[pos] = True
        if not filled.all():
            raise ValueError("a subspace was computed on no rank")
        out[name] = full
    return out
