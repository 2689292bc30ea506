"""The nodal (block) hierarchy on the GPU (Sec. 3.1 with k x k blocks, Sec. 4.2.1 approach (iii)), through
the C ABI, against the oracle.

Integer structure (block strength expanded to the entries of A, splittings, patterns of R, P and every coarse
operator) must be identical; FP64 values within 1e-12 and FP32 (mixed precision) values within 1e-5 of the
row's largest entry. The GPU applies block Jacobi as point Jacobi on D^{-1}A with right-hand side D^{-1}b, the
oracle as x + D^{-1}(b - A x): the cycles agree to rounding (1e-10 in FP64, 1e-5 mixed).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import oracle as O
from tests.helpers import compare_hierarchies, entrywise_rel

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
    m = dict(cf_mode="cf_mode", distance="distance", theta="theta", interp="interp", lump_tol="lump_tol",
             lump_level0="lump_level0", coarse_max="coarse_max", max_levels="max_levels", precision="prec",
             nodal="nodal")
    return {m[k]: v for k, v in kw.items()}


def _kron(k):
    s = W.fd_adr_2d(24, 3 * math.pi / 16, 1e-2, 0.5)
    A = sp.kron(s.to_scipy(), sp.identity(k), format="csr")
    A.sort_indices()
    n = A.shape[0]
    return W.CsrSystem(n, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.copy(),
                       np.random.default_rng(k).uniform(-1, 1, n))


CASES = {
    "dg12_onepoint_d2": (lambda: W.dg_p2_advection(12), dict(nodal=6, distance=2, interp=1)),
    "dg16_onepoint_d2_mixed": (lambda: W.dg_p2_advection(16), dict(nodal=6, distance=2, interp=1, precision=1)),
    "dg12_laip_d1": (lambda: W.dg_p2_advection(12), dict(nodal=6, distance=1, interp=0)),
    "dg16_pmis_d2_lump0": (lambda: W.dg_p2_advection(16),
                           dict(nodal=6, distance=2, interp=1, cf_mode=1, lump_tol=0.01, lump_level0=1)),
    "dg12_rs_d3": (lambda: W.dg_p2_advection(12), dict(nodal=6, distance=3, interp=1, cf_mode=0)),
    "kron2_laip_d2": (lambda: _kron(2), dict(nodal=2, distance=2, interp=0, lump_tol=0.01)),
    "kron3_onepoint_mixed": (lambda: _kron(3), dict(nodal=3, distance=2, interp=1, precision=1)),
}


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("case", sorted(CASES))
def test_nodal_hierarchy_matches_oracle(lair, case):
    make, kw = CASES[case]
    s = make()
    G = lair.Hierarchy.from_system(s, device=True, **kw)
    H = O.Hierarchy(s, **okw(kw))
    assert H.status == 0
    mixed = kw.get("precision") == 1
    compare_hierarchies(G, H, TOL32 if mixed else TOL64)
    v = np.random.default_rng(5).uniform(-1, 1, s.n)
    z = G.precond(_dev(v)).cpu().numpy()
    zo = H.precond(v)
    assert entrywise_rel(z, zo) <= (TOL32 if mixed else 1e-10)
    x, rep = G.solve(_dev(s.b), tol=1e-9, max_iter=200)
    xo, ro = H.solve(s.b, tol=1e-9, max_iter=200)
    assert rep.status == 0 and ro["status"] == 0
    assert abs(rep.iters - ro["iters"]) <= 1
    xh = x.cpu().numpy()
    assert np.linalg.norm(s.b - s.to_scipy() @ xh) <= 2e-9 * np.linalg.norm(s.b)


def test_nodal_refresh_matches_oracle(lair):
    s1, s2 = W.dg_p2_advection(12), W.dg_p2_advection(12, dt=0.5 / 12)
    kw = dict(nodal=6, distance=2, interp=1, lump_tol=0.01)
    G = lair.Hierarchy.from_system(s1, device=True, **kw)
    G.refresh(_dev(s2.val))
    H = O.Hierarchy(s1, **okw(kw))
    assert H.refresh(s2) == 0
    compare_hierarchies(G, H, TOL64)
    v = np.random.default_rng(6).uniform(-1, 1, s2.n)
    z = G.precond(_dev(v)).cpu().numpy()
    zo = H.precond(v)
    assert entrywise_rel(z, zo) <= 1e-10


def test_nodal_full_size_dg(lair):
    """786,432 unknowns, nodes of 6: the hierarchy solves to 1e-8 in mixed precision."""
    s = W.dg_p2_advection(256)
    G = lair.Hierarchy.from_system(s, device=True, nodal=6, distance=2, interp=1, precision=1)
    x, rep = G.solve(_dev(s.b), tol=1e-8)
    assert rep.status == 0 and rep.iters <= 15
    xh = x.cpu().numpy()
    assert np.linalg.norm(s.b - s.to_scipy() @ xh) <= 1.5e-8 * np.linalg.norm(s.b)


@pytest.mark.parametrize("kw,code", [(dict(nodal=6, block_size=6), 1), (dict(nodal=9), 13), (dict(nodal=5), 1),
                                     (dict(nodal=6, restriction=1), 13)])
def test_nodal_rejected_combinations(lair, kw, code):
    s = W.dg_p2_advection(4)
    with pytest.raises(lair.LairError) as e:
        lair.Hierarchy.from_system(s, **kw)
    assert e.value.status == code


def test_nodal_adjoint_matches_oracle_on_the_transpose(lair):
    s = W.dg_p2_advection(10)
    kw = dict(nodal=6, distance=2, interp=1)
    G = lair.Hierarchy.from_system(s, **kw)
    g = np.random.default_rng(3).uniform(-1, 1, s.n)
    lam, rep = G.adjoint(g, tol=1e-10)
    assert rep.status == 0
    AT = s.to_scipy().T.tocsr()
    assert np.linalg.norm(g - AT @ lam) <= 2e-10 * np.linalg.norm(g)
    H = O.Hierarchy(W.CsrSystem(s.n, *O.transpose(s), g), **okw(kw))
    lo, ro = H.solve(g, tol=1e-10)
    assert abs(rep.iters - ro["iters"]) <= 1
    assert np.linalg.norm(lam - lo) <= 1e-8 * np.linalg.norm(lo)


def test_nodal_user_splitting_matches_oracle(lair):
    s = W.dg_p2_advection(10)
    N = s.n // 6
    cfB = (np.random.default_rng(8).uniform(size=N) < 0.4).astype(np.int8)
    cf = np.repeat(cfB, 6)
    kw = dict(nodal=6, distance=2, interp=1)
    G = lair.Hierarchy.from_system(s, device=True, cf_user=cf, **kw)
    H = O.Hierarchy(s, cf_user=cf, **okw(kw))
    assert H.status == 0
    compare_hierarchies(G, H, TOL64)
