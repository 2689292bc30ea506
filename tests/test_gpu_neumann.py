"""The Neumann restriction nAIR (Sec. 3.2) on the GPU, through the C ABI, against the oracle.

Integer structure (splittings, the sets of the series, the patterns of R, P and every coarse operator)
must be identical; FP64 values within 1e-12 and FP32 (mixed precision) values within 1e-5 of the row's
largest entry; the cycle and the solve agree with the oracle's.
"""
import math

import numpy as np
import pytest

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
    m = dict(cf_mode="cf_mode", distance="distance", theta="theta", strength_abs="strength_abs", interp="interp",
             lump_tol="lump_tol", coarse_max="coarse_max", max_levels="max_levels", block_size="block_size",
             precision="prec", restriction="restriction")
    return {m[k]: v for k, v in kw.items()}


CASES = {
    "fd2d64_d1": (lambda: W.config("fd2d_64"), dict(distance=1)),
    "fd2d64_d2": (lambda: W.config("fd2d_64"), dict(distance=2)),
    "fd2d64_d3_mixed": (lambda: W.config("fd2d_64"), dict(distance=3, precision=1)),
    "fd2d64_pmis_d2_onepoint": (lambda: W.config("fd2d_64"), dict(distance=2, cf_mode=1, interp=1)),
    "fd3d_20_d2": (lambda: W.config("fd3d_192", scale=20), dict(distance=2)),
    "dg_p2_16_d2_mixed": (lambda: W.dg_p2_advection(16),
                          dict(distance=2, interp=1, strength_abs=1, block_size=6, precision=1)),
    "random_d2": (lambda: W.random_sparse(1500, 6, seed=5), dict(distance=2, lump_tol=0.01)),
    "diffusive_d4": (lambda: W.fd_adr_2d(40, 1.1, 0.5, 0.3), dict(distance=4)),
}


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("case", sorted(CASES))
def test_neumann_hierarchy_matches_oracle(lair, case):
    make, kw = CASES[case]
    s = make()
    kw = dict(kw, restriction=lair.R_NEUMANN)
    G = lair.Hierarchy.from_system(s, device=True, **kw)
    H = O.Hierarchy(s, **okw(kw))
    assert H.status == 0
    tol = TOL32 if kw.get("precision") == 1 else TOL64
    compare_hierarchies(G, H, tol)
    v = np.random.default_rng(11).uniform(-1, 1, s.n)
    z = G.precond(_dev(v)).cpu().numpy()
    zo = H.precond(v)
    assert entrywise_rel(z, zo) <= tol
    x, rep = G.solve(_dev(s.b), tol=1e-9, max_iter=300)
    xo, ro = H.solve(s.b, tol=1e-9, max_iter=300)
    assert rep.status == ro["status"]
    if rep.status == 0:
        assert abs(rep.iters - ro["iters"]) <= 1


def test_neumann_refresh_matches_oracle(lair):
    s1, s2 = W.fd_adr_2d(64, 3 * math.pi / 16, 1e-3, 20.0), W.fd_adr_2d(64, 3 * math.pi / 16, 1e-3, 0.5)
    kw = dict(distance=2, restriction=lair.R_NEUMANN)
    G = lair.Hierarchy.from_system(s1, device=True, **kw)
    G.refresh(_dev(s2.val))
    H = O.Hierarchy(s1, **okw(kw))
    assert H.refresh(s2) == 0
    compare_hierarchies(G, H, TOL64)


def test_neumann_rejects_unknown_restriction(lair):
    s = W.config("fd2d_64", scale=16)
    with pytest.raises(lair.LairError) as e:
        lair.Hierarchy.from_system(s, restriction=2)
    assert e.value.status == 1
