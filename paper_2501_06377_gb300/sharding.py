"""Realizations across processes (one process per GPU).

Realizations are independent (the paper never splits a grid across ranks,
Sec. 4.1), so the multi-GPU path has no collective on its data path: each
rank advances its own shard.  This module holds the host logic:

* ``lpt_shards``: longest-processing-time-first bin packing of realizations
  by cost (cells x RKL2 stages x steps) over ranks;
* ``requeue``: hand the realizations of failed ranks to the survivors;
* ``max_over_ranks``: the timing reduction of a benchmark (the only
  collective, outside the timed data path);
* ``checked_barrier``: a barrier that names the ranks that did not arrive
  within a timeout (gloo's monitored barrier) instead of hanging;
* ``run_sharded``: the launcher: plan the shards, advance this rank's own
  realizations with no collective, then gather every rank's FP64
  diagnostics records to rank 0 (host objects, after the run);
* ``grid_advance``: the shard step of ``run_sharded`` on this rank's GPU.
"""
from __future__ import annotations

import heapq


def lpt_shards(costs, world):
    """Assign realization indices to ``world`` ranks, largest cost first to
    the least-loaded rank (Graham's LPT rule: makespan <= 4/3 optimal)."""
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(s) for s in out]


def shard_costs(shapes, stages, steps=1):
    """Cost of each realization: cells x (RKL2 stages + 4 advection stages) x steps."""
    return [nt * nph * (s + 4) * steps for (nt, nph), s in zip(shapes, stages)]


def requeue(shards, costs, failed):
    """New shards after the ranks in ``failed`` dropped out: their
    realizations go to the surviving ranks, least loaded first."""
    alive = [r for r in range(len(shards)) if r not in set(failed)]
    if not alive:
        raise RuntimeError("no rank left to take the realizations")
    loads = {r: sum(costs[i] for i in shards[r]) for r in alive}
    heap = [(loads[r], r) for r in alive]
    heapq.heapify(heap)
    out = {r: list(shards[r]) for r in alive}
    orphans = sorted((i for r in failed for i in shards[r]), key=lambda i: (-costs[i], i))
    for i in orphans:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(out[r]) if r in out else [] for r in range(len(shards))]


def max_over_ranks(x, device=None):
    """Maximum of a scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def checked_barrier(timeout_s=5.0):
    """Barrier that raises (naming the missing ranks) after ``timeout_s``
    instead of waiting forever; needs a gloo process group."""
    import datetime

    import torch.distributed as dist
    dist.monitored_barrier(timeout=datetime.timedelta(seconds=timeout_s), wait_all_ranks=True)


def gather_records(records, world, dst=0):
    """Every rank's list of (realization index, record) on rank ``dst``, in
    realization order (None on the other ranks; the local list without a
    process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or world == 1:
        return sorted(records, key=lambda x: x[0])
    rank = dist.get_rank()
    out = [None] * world if rank == dst else None
    dist.gather_object(records, out, dst=dst)
    if rank != dst:
        return None
    return sorted((x for part in out for x in part), key=lambda x: x[0])


def run_sharded(costs, advance, world, rank):
    """Plan the shards by cost (LPT), advance this rank's realizations with
    ``advance(indices) -> [(index, record), ...]`` (no collective inside),
    and gather all records on rank 0.  Returns (shards, records on rank 0 or
    None, this rank's seconds)."""
    import time
    shards = lpt_shards(costs, world)
    t0 = time.perf_counter()
    mine = advance(shards[rank]) if shards[rank] else []
    sec = time.perf_counter() - t0
    return shards, gather_records(mine, world), sec


def grid_advance(shapes, params, start_map, t_target, stream=None):
    """The shard step on this rank's GPU: one batched Grid over the given
    realizations (FP32), each started from ``start_map(shape)``, advanced to
    t_target hours; returns the ``advance`` callable of run_sharded, whose
    records are the realizations' FP64 diagnostics (sft_flux_diagnostics)."""
    def advance(idx):
        from .sft import Grid
        g = Grid([shapes[i] for i in idx], "fp32", stream=stream)
        for q, i in enumerate(idx):
            g.set_state(q, start_map(shapes[i]))
        g.set_flows([params[i] for i in idx])
        g.step(t_target)
        diag = g.diagnostics()
        g.close()
        return [(i, d) for i, d in zip(idx, diag)]
    return advance
