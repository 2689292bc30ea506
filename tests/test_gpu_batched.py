"""Batched independent systems (one block-diagonal hierarchy) against the oracle.

The oracle builds the same block-diagonal hierarchy (splitting blocks inside systems) and
runs the same per-system stationary refinement; structure must match bit for bit, each
system's solution must match its own sparse direct solve.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import oracle as O
from tests.helpers import compare_hierarchies, entrywise_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lair():
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair as L
    return L


def batch(count, lo, hi):
    systems = W.batched_fd(count=count, side_lo=lo, side_hi=hi)
    A, offs = W.block_diagonal(systems)
    return systems, A, offs


@pytest.mark.parametrize("kw", [dict(precision=1), dict(precision=0, rs_block=512), dict(cf_mode=0, precision=1),
                                dict(cf_mode=1, precision=1, distance=2)])
def test_batched_hierarchy_matches_oracle(lair, kw):
    import torch
    systems, A, offs = batch(24, 16, 64)
    rp = torch.from_numpy(A.row_ptr).cuda()
    col = torch.from_numpy(A.col).cuda()
    val = torch.from_numpy(A.val).cuda()
    G = lair.Hierarchy.batched(rp, col, val, offs, **kw)
    okw = {("prec" if k == "precision" else k): v for k, v in kw.items()}
    H = O.Hierarchy(A, seg=offs, **okw)
    assert H.status == 0
    compare_hierarchies(G, H, 1e-5 if kw.get("precision") == 1 else 1e-12)


@pytest.mark.parametrize("cycle", [0, 1])
def test_batched_solve_per_system(lair, cycle):
    import torch
    systems, A, offs = batch(40, 16, 96)
    rp = torch.from_numpy(A.row_ptr).cuda()
    col = torch.from_numpy(A.col).cuda()
    val = torch.from_numpy(A.val).cuda()
    G = lair.Hierarchy.batched(rp, col, val, offs, precision=1)
    x, its, rel, st = G.solve_batched(torch.from_numpy(A.b).cuda(), tol=1e-8, max_iter=2000, cycle=cycle)
    H = O.Hierarchy(A, seg=offs, prec=1)
    xo, ro = H.solve_batched(A.b, tol=1e-8, max_iter=2000, cycle=cycle)
    assert st == 0 and ro["status"] == 0
    assert (rel <= 1e-8).all()
    assert np.abs(its - ro["iters"]).max() <= 1
    xg = x.cpu().numpy()
    for k, s in enumerate(systems):
        ref = spla.spsolve(s.to_scipy().tocsc(), s.b)
        xs = xg[offs[k]:offs[k + 1]]
        r = np.linalg.norm(s.b - s.to_scipy() @ xs) / np.linalg.norm(s.b)
        assert r <= 1.01e-8
        assert np.linalg.norm(xs - xo[offs[k]:offs[k + 1]]) <= 1e-6 * np.linalg.norm(ref)


def test_batch_setup_solve_convenience(lair):
    import ctypes
    systems = W.batched_fd(count=6, side_lo=20, side_hi=40)
    keep = []
    arr = (lair.lair_csr * len(systems))()
    bp = (ctypes.c_void_p * len(systems))()
    xp = (ctypes.c_void_p * len(systems))()
    xs = []
    for q, s in enumerate(systems):
        rp, col, val, b = (np.ascontiguousarray(s.row_ptr), np.ascontiguousarray(s.col), np.ascontiguousarray(s.val),
                           np.ascontiguousarray(s.b))
        x = np.zeros(s.n)
        keep += [rp, col, val, b, x]
        xs.append(x)
        arr[q] = lair.lair_csr(s.n, s.nnz, rp.ctypes.data, col.ctypes.data, val.ctypes.data, 0)
        bp[q] = b.ctypes.data
        xp[q] = x.ctypes.data
    its = np.zeros(len(systems), np.int32)
    rel = np.zeros(len(systems))
    o = lair.options(precision=1)
    st = lair.lib.lair_batch_setup_solve(len(systems), arr, bp, xp, ctypes.byref(o), 1e-8, 1, 400, its.ctypes.data,
                                         rel.ctypes.data)
    assert st == 0 and (rel <= 1e-8).all()
    for s, x in zip(systems, xs):
        assert np.linalg.norm(s.b - s.to_scipy() @ x) / np.linalg.norm(s.b) <= 1.01e-8


@pytest.mark.parametrize("count", [4, 10])
def test_batched_vcycle_matches_oracle(lair, count):
    """One V-cycle on a batch equals the oracle's entry by entry (FP32 cycle: within 1e-5 of the largest entry)."""
    import torch
    systems, A, offs = batch(count, 16, 96)
    G = lair.Hierarchy.batched(torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col).cuda(),
                               torch.from_numpy(A.val).cuda(), offs, precision=1)
    H = O.Hierarchy(A, seg=offs, prec=1)
    v = np.random.default_rng(0).uniform(-1, 1, A.n)
    z = G.precond(torch.from_numpy(v).cuda()).cpu().numpy()
    zo = H.precond(v)
    assert np.isfinite(z).all()
    assert entrywise_rel(z, zo) <= 1e-5


@pytest.mark.parametrize("cycle", [0, 1])
def test_stopped_systems_leave_no_trace(lair, cycle):
    """The cycle skips the rows of systems that have stopped. A system with b = 0 stops before its first cycle,
    so its rows never run in that solve; the other systems still reach their tolerance against their own
    direct solves, the zero system keeps x = 0, and a later solve on the same hierarchy gives the bits of a
    fresh hierarchy's solve (no run flag or cycle buffer carries over)."""
    import torch
    systems, A, offs = batch(8, 20, 48)
    opts = dict(cf_mode=1, interp=1, lump_tol=0.05, precision=1)
    b = A.b.copy()
    b[offs[2]:offs[3]] = 0.0
    G = lair.Hierarchy.batched(torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col).cuda(),
                               torch.from_numpy(A.val).cuda(), offs, **opts)
    x, its, rel, st = G.solve_batched(torch.from_numpy(b).cuda(), tol=1e-8, cycle=cycle, max_iter=2000)
    assert st == 0 and its[2] == 0 and (rel <= 1e-8).all()
    x = x.cpu().numpy()
    assert not x[offs[2]:offs[3]].any()
    for q, s in enumerate(systems):
        if q == 2:
            continue
        xr = spla.spsolve(s.to_scipy().tocsc(), b[offs[q]:offs[q + 1]])
        assert np.linalg.norm(x[offs[q]:offs[q + 1]] - xr) <= 1e-6 * np.linalg.norm(xr)
    # a second solve on the same hierarchy: the bits of a fresh hierarchy's first solve
    x2, its2, _, st2 = G.solve_batched(torch.from_numpy(A.b).cuda(), tol=1e-8, cycle=cycle, max_iter=2000)
    F = lair.Hierarchy.batched(torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col).cuda(),
                               torch.from_numpy(A.val).cuda(), offs, **opts)
    xf, itsf, _, stf = F.solve_batched(torch.from_numpy(A.b).cuda(), tol=1e-8, cycle=cycle, max_iter=2000)
    assert st2 == 0 and stf == 0 and np.array_equal(its2, itsf)
    assert torch.equal(x2, xf)
    # and outside the batched loops every system runs again: one preconditioner application of the whole batch
    v = torch.from_numpy(np.random.default_rng(5).uniform(-1, 1, A.n)).cuda()
    assert torch.equal(G.precond(v), F.precond(v))
