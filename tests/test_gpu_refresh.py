"""Hierarchy refresh on the GPU (lair_refresh through the C ABI) against the oracle's refresh.

A hierarchy is set up for one matrix and refreshed with the values of another on the same pattern
(the backward Euler matrix I + dt S of Sec. 4.1.1 with a new dt, or new coefficients). Integer
structure must be the set-up's and identical on both sides; values within 1e-12 (FP64) or 1e-5
(mixed precision) of the row's largest entry; the cycle and the solve must agree with the oracle's.
Refreshing with the set-up's own values must reproduce the set-up bit for bit.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import oracle as O
from tests.helpers import backward_euler, compare_hierarchies, entrywise_rel

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


@pytest.fixture(scope="module")
def lair():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair as L
    torch.cuda.init()
    return L


def okw(kw):
    m = dict(cf_mode="cf_mode", distance="distance", theta="theta", strength_abs="strength_abs", interp="interp",
             lump_tol="lump_tol", lump_level0="lump_level0", coarse_max="coarse_max", max_levels="max_levels",
             block_size="block_size", precision="prec")
    return {m[k]: v for k, v in kw.items()}


def _fd2d(c):
    return W.fd_adr_2d(64, 3 * math.pi / 16, 1e-3, c)


def _be(S, dt):
    return backward_euler(S, dt)


CASES = {
    # new coefficients: reaction-dominated to advection-dominated
    "fd2d_reaction_laip_d2": (lambda: _fd2d(50.0), lambda: _fd2d(0.5), dict(distance=2)),
    # backward Euler with a new time step
    "fd2d_be_onepoint_mixed": (lambda: _be(W.config("fd2d_64"), 0.05), lambda: _be(W.config("fd2d_64"), 0.4),
                               dict(distance=2, interp=1, precision=1)),
    "fd3d_20_be_d1": (lambda: _be(W.config("fd3d_192", scale=20), 0.1),
                      lambda: _be(W.config("fd3d_192", scale=20), 1.0), dict(distance=1)),
    "dg_p2_16_dt": (lambda: W.dg_p2_advection(16), lambda: W.dg_p2_advection(16, dt=0.5 / 16),
                    dict(distance=2, interp=1, strength_abs=1, block_size=6, precision=1)),
    "dg_p2_12_dt_laip": (lambda: W.dg_p2_advection(12), lambda: W.dg_p2_advection(12, dt=2.0 / 12),
                         dict(distance=2, interp=0, strength_abs=1, block_size=6)),
    "fd2d_lump0_pmis": (lambda: _fd2d(5.0), lambda: _fd2d(0.5),
                        dict(distance=2, cf_mode=1, lump_tol=1e-2, lump_level0=1)),
    "fd2d_laip_mixed_d3": (lambda: _fd2d(2.0), lambda: _fd2d(0.2), dict(distance=3, precision=1)),
}


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("case", sorted(CASES))
def test_refresh_matches_oracle_refresh(lair, case):
    make1, make2, kw = CASES[case]
    s1, s2 = make1(), make2()
    assert np.array_equal(s1.col, s2.col) and np.array_equal(s1.row_ptr, s2.row_ptr)
    G = lair.Hierarchy.from_system(s1, device=True, **kw)
    H = O.Hierarchy(s1, **okw(kw))
    assert H.status == 0
    G.refresh(_dev(s2.val))
    assert H.refresh(s2) == 0
    tol = TOL32 if kw.get("precision") == 1 else TOL64
    compare_hierarchies(G, H, tol)
    # the cycle on the refreshed hierarchy (views, diagonals, coarsest inverse refreshed in place)
    rng = np.random.default_rng(3)
    v = rng.uniform(-1, 1, s2.n)
    z = G.precond(_dev(v)).cpu().numpy()
    zo = H.precond(v)
    assert entrywise_rel(z, zo) <= tol
    x, rep = G.solve(_dev(s2.b), tol=1e-10)
    assert rep.status == 0
    xh = x.cpu().numpy()
    assert np.linalg.norm(s2.b - s2.to_scipy() @ xh) / np.linalg.norm(s2.b) <= 2e-10
    xo, ro = H.solve(s2.b, tol=1e-10)
    assert abs(rep.iters - ro["iters"]) <= 1


def _exports(G):
    out = []
    for l, inf in enumerate(G.info()):
        out.append(G.export_csr(l, 0))
        if not inf["coarsest"]:
            out += [G.export_csr(l, 1), G.export_csr(l, 2), G.export_cf(l)]
    return out


@pytest.mark.parametrize("case", ["fd2d_reaction_laip_d2", "dg_p2_16_dt", "fd2d_lump0_pmis", "fd2d_laip_mixed_d3"])
def test_refresh_with_setup_values_is_bit_identical(lair, case):
    make1, make2, kw = CASES[case]
    s1, s2 = make1(), make2()
    G = lair.Hierarchy.from_system(s1, device=True, **kw)
    F = lair.Hierarchy.from_system(s1, device=True, **kw)
    G.refresh(np.ascontiguousarray(s2.val))      # host buffer
    G.refresh(np.ascontiguousarray(s1.val))
    for a, b in zip(_exports(G), _exports(F)):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    v = _dev(np.random.default_rng(1).uniform(-1, 1, s1.n))
    assert np.array_equal(G.precond(v).cpu().numpy(), F.precond(v).cpu().numpy())


def test_refresh_full_size_dg(lair):
    """786,432 unknowns: refresh to half the time step, solve, check the defining equation of R,
    (R A)_{c,j} = 0 on the neighbourhood (Eq. (3.1)), on sampled rows of level 0, and the true residual."""
    s1 = W.dg_p2_advection(256)
    s2 = W.dg_p2_advection(256, dt=0.5 / 256)
    kw = dict(distance=2, interp=1, strength_abs=1, block_size=6, precision=1)
    G = lair.Hierarchy.from_system(s1, device=True, **kw)
    G.refresh(_dev(s2.val))
    x, rep = G.solve(_dev(s2.b), tol=1e-8)
    assert rep.status == 0
    xh = x.cpu().numpy()
    assert np.linalg.norm(s2.b - s2.to_scipy() @ xh) / np.linalg.norm(s2.b) <= 1.5e-8
    rp, col, val = G.export_csr(0, 0)            # the block-scaled level-0 operator
    A = sp.csr_matrix((val, col.astype(np.int64), rp), shape=(s2.n, s2.n))
    rrp, rcol, rval = G.export_csr(0, 1)
    cf, _, _, _ = G.export_cf(0)
    Cpts = np.nonzero(cf == 1)[0]
    R = sp.csr_matrix((rval, rcol.astype(np.int64), rrp), shape=(len(Cpts), s2.n))
    rows = np.random.default_rng(4).choice(len(Cpts), 300, replace=False)
    RA = (R[rows] @ A).tocsr()
    scale = (abs(R[rows]) @ abs(A)).tocsr()         # the size of the terms that cancel
    for q, c in enumerate(rows):
        for j in rcol[rrp[c]:rrp[c + 1]]:
            if j != Cpts[c]:
                # the local systems are solved in FP32 in mixed precision
                assert abs(RA[q, j]) <= 1e-5 * scale[q, j]


def test_refresh_adjoint(lair):
    s1, s2 = _fd2d(50.0), _fd2d(0.5)
    G = lair.Hierarchy.from_system(s1)
    g = np.random.default_rng(2).uniform(-1, 1, s1.n)
    G.adjoint(g, tol=1e-10)                      # builds the adjoint hierarchy
    G.refresh(np.ascontiguousarray(s2.val))
    lam, rep = G.adjoint(g, tol=1e-10)
    assert rep.status == 0
    AT = s2.to_scipy().T.tocsr()
    assert np.linalg.norm(g - AT @ lam) / np.linalg.norm(g) <= 2e-10
    t1, t2 = O.transpose(s1), O.transpose(s2)
    H = O.Hierarchy(W.CsrSystem(s1.n, *t1, g))
    assert H.refresh(W.CsrSystem(s2.n, *t2, g)) == 0
    lo, ro = H.solve(g, tol=1e-10)
    assert abs(rep.iters - ro["iters"]) <= 1
    assert np.linalg.norm(lam - lo) <= 1e-8 * np.linalg.norm(lo)


def test_refresh_batched(lair):
    systems1 = [W.fd_adr_2d(n, a, 1e-3, 20.0, b_seed=q) for q, (n, a) in enumerate([(24, 0.3), (40, 1.2), (31, 2.5)])]
    systems2 = [W.fd_adr_2d(n, a, 1e-3, 0.2, b_seed=q) for q, (n, a) in enumerate([(24, 0.3), (40, 1.2), (31, 2.5)])]
    (B1, offs), (B2, _) = W.block_diagonal(systems1), W.block_diagonal(systems2)
    G = lair.Hierarchy.batched(_dev(B1.row_ptr), _dev(B1.col), _dev(B1.val), offs, distance=2)
    G.refresh(_dev(B2.val))
    H = O.Hierarchy(B1, seg=offs, distance=2)
    assert H.refresh(B2) == 0
    compare_hierarchies(G, H, TOL64)
    x, its, rel, st = G.solve_batched(_dev(B2.b), tol=1e-10, cycle=lair.FGMRES)
    assert st == 0 and (rel <= 1e-10).all()


def test_refresh_zero_diagonal_then_recover(lair):
    s1, s2 = _fd2d(50.0), _fd2d(0.5)
    G = lair.Hierarchy.from_system(s1, device=True, distance=2)
    bad = s2.val.copy()
    rows = np.repeat(np.arange(s2.n), np.diff(s2.row_ptr))
    bad[np.nonzero((rows == s2.col) & (rows == 100))[0]] = 0.0
    with pytest.raises(lair.LairError) as e:
        G.refresh(_dev(bad))
    assert e.value.status == 5
    G.refresh(_dev(s2.val))
    H = O.Hierarchy(s1, distance=2)
    assert H.refresh(s2) == 0
    compare_hierarchies(G, H, TOL64)


def test_refresh_rejects_wrong_length(lair):
    s = _fd2d(1.0)
    G = lair.Hierarchy.from_system(s)
    with pytest.raises(ValueError):
        G.refresh(np.zeros(s.nnz - 1))
