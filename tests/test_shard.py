"""Batched systems over ranks (CPU): the LPT partition and the final gather, with two gloo ranks.
The per-rank solve is the CPU oracle here (the GPU path plugs the CUDA batched solve into the same
driver); no data-path collective runs, only the gather of statuses and iteration counts."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_lpt_partition_each_system_once_and_within_bound():
    from paper_1708_06065_gb300.shard import lpt_partition
    rng = np.random.default_rng(0)
    for nparts in (1, 2, 3, 8):
        costs = list(rng.integers(1, 10**6, 97))
        parts = lpt_partition(costs, nparts)
        flat = sorted(q for p in parts for q in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[q] for q in p) for p in parts]
        assert max(loads) <= sum(costs) / nparts + (1 - 1 / nparts) * max(costs)
    # by hand: 7 -> part 0, 7 -> 1, 6 -> 0 (loads 7, 7: ties go to the lower part), 6 -> 1, 5 -> 0, 5 -> 1
    assert lpt_partition([7, 7, 6, 6, 5, 5], 2) == [[0, 2, 4], [1, 3, 5]]
    # 9 -> 0, 8 -> 1, 4 -> 1 (8 < 9), 3 -> 0 (9 < 12): loads 12 and 12
    assert lpt_partition([3, 9, 4, 8], 2) == [[0, 1], [2, 3]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_solve(systems):
    from oracle import oracle as O
    import workloads as W
    A, offs = W.block_diagonal(systems)
    H = O.Hierarchy(A, seg=offs, prec=1)
    x, rep = H.solve_batched(A.b, tol=1e-8, cycle=1)
    return np.where(rep["rel"] <= 1e-8, 0, 7), rep["iters"], rep["rel"]


def _rank_main(rank, world, port, out):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import workloads as W
    from paper_1708_06065_gb300.shard import solve_sharded
    dist.init_process_group("gloo", rank=rank, world_size=world)
    systems = W.batched_fd(count=7, side_lo=8, side_hi=20)
    st, it, rel = solve_sharded(systems, rank, world, _oracle_solve)
    out.put((rank, st.tolist(), it.tolist(), rel.tolist()))
    dist.destroy_process_group()


def test_sharded_batch_gathers_every_system():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (s, i, l)) for r, s, i, l in (q.get(timeout=180) for _ in range(2)))
    for p in procs:
        p.join(60)
    assert all(p.exitcode == 0 for p in procs)
    assert got[0] == got[1]                      # every rank holds the gathered results
    st, it, rel = (np.asarray(v) for v in got[0])
    # each part solved by itself gives the gathered entries of its systems (a batch's hierarchy depth is
    # common to its systems, so results are per part, not per system alone)
    from paper_1708_06065_gb300.shard import lpt_partition, system_cost
    systems = W.batched_fd(count=7, side_lo=8, side_hi=20)
    assert (st == 0).all()
    for part in lpt_partition([system_cost(s.n, s.nnz) for s in systems], 2):
        s1, i1, r1 = _oracle_solve([systems[q] for q in part])
        assert np.array_equal(st[part], s1) and np.array_equal(it[part], i1)
        np.testing.assert_array_equal(rel[part], r1)
