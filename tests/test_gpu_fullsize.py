"""Parity at the sizes the benchmark runs, with the benchmark's options and launch path.

The DG workload at full size (786,432 unknowns: PMIS through the cooperative kernel, distance-2
neighbourhoods with CTA-team local solves on the coarse levels, one-point P, block scaling,
mixed precision); the 3D FD workload at 96^3 and at its full 192^3 (7,077,888 unknowns, PMIS,
one-point P with the thread-per-row fused Galerkin product); and
the first 16 systems of the batched workload (sides up to 243). Every level's integer structure
must equal the oracle's bit for bit and its values must agree within 1e-5 of the row's largest
entry (FP32 local solves); one V-cycle is compared entry by entry, within 1e-5 of the largest
entry of the oracle's output.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import oracle as O
from tests.helpers import compare_hierarchies, entrywise_rel

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def lair():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair as L
    torch.cuda.init()
    return L


def oracle_kw(kw):
    m = dict(cf_mode="cf_mode", distance="distance", strength_abs="strength_abs", interp="interp",
             block_size="block_size", precision="prec", lump_tol="lump_tol", theta="theta")
    return {m[k]: v for k, v in kw.items()}


def device_hierarchy(lair, s, offs=None, **kw):
    """The hierarchy as bench.py builds it: device-resident CSR, a side stream, timers on."""
    import torch
    stream = torch.cuda.Stream()
    rp, col, val = (torch.from_numpy(a).cuda() for a in (s.row_ptr, s.col, s.val))
    if offs is None:
        G = lair.Hierarchy(rp, col, val, stream=stream, timing=1, **kw)
    else:
        G = lair.Hierarchy.batched(rp, col, val, offs, stream=stream, timing=1, **kw)
    torch.cuda.synchronize()
    return G


def check_cycle(G, H, n, seed):
    import torch
    v = np.random.default_rng(seed).uniform(-1, 1, n)
    z = G.precond(torch.from_numpy(v).cuda()).cpu().numpy()
    zo = H.precond(v)
    assert np.isfinite(z).all()
    err = entrywise_rel(z, zo)
    assert err <= TOL32, err


@pytest.mark.parametrize("name,scale", [("dg_p2_256", None), ("fd3d_192", 96), ("fd3d_192", None)])
def test_full_size_hierarchy_and_cycle(lair, name, scale):
    """The 3D system at 96^3 and at its full 192^3 (7,077,888 unknowns, the bench's default workload)."""
    s = W.config(name, scale=scale)
    kw = dict(W.BENCH_OPTIONS[name]["opts"], precision=lair.MIXED)
    G = device_hierarchy(lair, s, **kw)
    H = O.Hierarchy(s, **oracle_kw(kw))
    assert H.status == 0
    worst = compare_hierarchies(G, H, TOL32)
    assert max(worst.values()) <= TOL32
    check_cycle(G, H, s.n, 5)


def test_batched_first_16_systems(lair):
    import torch
    systems = W.config("batched_512", scale=16)
    assert max(s.n for s in systems) >= 240 ** 2
    A, offs = W.block_diagonal(systems)
    kw = dict(W.BENCH_OPTIONS["batched_512"]["opts"], precision=lair.MIXED)
    G = device_hierarchy(lair, A, offs, **kw)
    H = O.Hierarchy(A, seg=offs, **oracle_kw(kw))
    assert H.status == 0
    compare_hierarchies(G, H, TOL32)
    check_cycle(G, H, A.n, 6)
    x, its, rel, st = G.solve_batched(torch.from_numpy(A.b).cuda(), tol=1e-8, max_iter=2000, cycle=lair.FGMRES)
    assert st == 0 and (rel <= 1e-8).all()
    xg = x.cpu().numpy()
    for q, s in enumerate(systems):
        xs = xg[offs[q]:offs[q + 1]]
        assert np.linalg.norm(s.b - s.to_scipy() @ xs) / np.linalg.norm(s.b) <= 1.01e-8
        ref = spla.spsolve(s.to_scipy().tocsc(), s.b)
        assert np.linalg.norm(xs - ref) <= 1e-5 * np.linalg.norm(ref)
