"""Independent systems spread over ranks, one GPU per rank.

The batched workload (many independent systems) needs no exchange while it is solved:
the systems are partitioned over the ranks by longest-processing-time-first list
scheduling on an estimated cost (n * nnz), each rank sets up and solves its share as
one block-diagonal hierarchy, and the only communication is one gather of the
per-system statuses, iteration counts and final residuals at the end. The single-system
workloads do not shard (they would need halo exchanges and reductions every step); they
run as independent replicas.
"""
from __future__ import annotations

import numpy as np


def system_cost(n: int, nnz: int) -> int:
    """Estimated cost of one system: set-up and solve both grow with its size and density."""
    return int(n) * int(nnz)


def lpt_partition(costs, nparts: int) -> list[list[int]]:
    """Longest processing time first: systems in decreasing cost (ties: lower index first), each to the
    part with the smallest load so far (ties: lower part). Returns the system indices of every part,
    ascending. The largest load is at most sum/nparts + (1 - 1/nparts) * max(costs)."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    order = sorted(range(len(costs)), key=lambda q: (-costs[q], q))
    loads = [0] * nparts
    parts = [[] for _ in range(nparts)]
    for q in order:
        r = min(range(nparts), key=lambda p: (loads[p], p))
        parts[r].append(q)
        loads[r] += costs[q]
    for p in parts:
        p.sort()
    return parts


def solve_sharded(systems, rank: int, world: int, solve_fn, group=None):
    """Solve this rank's LPT share of `systems` with solve_fn(list of systems) -> (status, iters, rel), one
    entry per system, then gather every rank's results. Returns (status, iters, rel) arrays over all
    systems in their original order, on every rank."""
    import torch.distributed as dist
    parts = lpt_partition([system_cost(s.n, s.nnz) for s in systems], world)
    mine = parts[rank]
    st, it, rel = solve_fn([systems[q] for q in mine]) if mine else ([], [], [])
    local = (list(mine), [int(v) for v in st], [int(v) for v in it], [float(v) for v in rel])
    if world > 1:
        got = [None] * world
        dist.all_gather_object(got, local, group=group)
    else:
        got = [local]
    status = np.full(len(systems), -1, np.int32)
    iters = np.zeros(len(systems), np.int32)
    rels = np.full(len(systems), np.nan)
    for ids, s_, i_, r_ in got:
        status[ids] = s_
        iters[ids] = i_
        rels[ids] = r_
    return status, iters, rels


def gpu_batched_solve(systems, tol=1e-8, max_iter=2000, cycle=1, **opts):
    """The systems as one block-diagonal hierarchy on the current GPU (lair_setup_batched and
    lair_solve_batched); per system: status 0 when its relative residual reached tol, else 7."""
    import torch
    import workloads as W
    from . import lair
    A, offs = W.block_diagonal(systems)
    dev = torch.device("cuda", torch.cuda.current_device())
    rp, col, val, b = (torch.from_numpy(a).to(dev) for a in (A.row_ptr, A.col, A.val, A.b))
    x = torch.zeros(A.n, dtype=torch.float64, device=dev)
    G = lair.Hierarchy.batched(rp, col, val, offs, **opts)
    _, its, rel, _ = G.solve_batched(b, x, tol=tol, cycle=cycle, max_iter=max_iter)
    G.close()
    rel = np.asarray(rel)
    return np.where(rel <= tol, 0, 7), np.asarray(its), rel
