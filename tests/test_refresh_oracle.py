"""Pins of the oracle's hierarchy refresh: new values on the set-up matrix's pattern.

The refresh keeps the splittings, the neighbourhoods of the local systems and the patterns of R, P
and of every coarse operator, and recomputes every value. What fixes the result independently of the
refresh code:

* the backward Euler matrix I + dt S of Sec. 4.1.1: dt scales every off-diagonal of a row by the same
  factor, so the strength of connection (Sec. 4) and with it the whole level-0 structure do not depend
  on dt; a two-level refresh must then reproduce a fresh set-up on the new matrix bit for bit;
* row scaling by powers of two (Sec. 3.1): R~ = D_c R D_f^{-1}, one-point P unchanged, coarse
  operators D_c K, all exact in floating point;
* the defining equations of the transfer operators on the new matrix: (R A)_{c,j} = 0 for j in the
  neighbourhood of c (Eq. (3.1)) and (A P)_{j,c} = 0 for j in Q_c (Eq. (2.6));
* scipy's sparse triple product R A P for the coarse operators, and the lumping rule of Sec. 3.3
  (row sums kept, kept entries unchanged);
* scipy's sparse direct solve for the solution.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import oracle as O
from tests.helpers import backward_euler, with_values


def csr_to_scipy(t, shape):
    rp, col, val = t
    return sp.csr_matrix((val, col.astype(np.int64), rp), shape=shape)


def assert_same_hierarchy(H1, H2):
    assert len(H1.levels) == len(H2.levels)
    for L1, L2 in zip(H1.levels, H2.levels):
        for a, b in zip(L1.A, L2.A):
            assert np.array_equal(a, b)
        for name in ("cf", "strong", "ls_R", "ls_P"):
            a, b = getattr(L1, name), getattr(L2, name)
            assert (a is None) == (b is None)
            if a is not None:
                assert np.array_equal(a, b), name
        for name in ("R", "P"):
            a, b = getattr(L1, name), getattr(L2, name)
            assert (a is None) == (b is None)
            if a is not None:
                for x, y in zip(a, b):
                    assert np.array_equal(x, y), name


OPTION_SETS = [
    dict(distance=2, interp=O.P_LAIP, lump_tol=1e-3),
    dict(distance=1, interp=O.P_ONEPOINT, lump_tol=1e-3, cf_mode=O.CF_PMIS),
    dict(distance=2, interp=O.P_LAIP, lump_tol=1e-2, lump_level0=1, prec=1),
    dict(distance=3, interp=O.P_ONEPOINT, lump_tol=0.0),
]


@pytest.mark.parametrize("kw", OPTION_SETS)
def test_refresh_with_the_same_values_changes_nothing(kw):
    s = W.config("fd2d_64", scale=32)
    H = O.Hierarchy(s, **kw)
    G = O.Hierarchy(s, **kw)
    assert H.status == 0 and H.refresh(s) == 0
    assert_same_hierarchy(H, G)
    x1, r1 = H.solve(s.b, tol=1e-10)
    x2, r2 = G.solve(s.b, tol=1e-10)
    assert r1["iters"] == r2["iters"] and np.array_equal(x1, x2)


def test_refresh_block_scaled_dg_same_values():
    s = W.dg_p2_advection(8)
    kw = dict(block_size=6, distance=2, interp=O.P_ONEPOINT, lump_tol=1e-3)
    H = O.Hierarchy(s, **kw)
    assert H.status == 0 and H.refresh(s) == 0
    assert_same_hierarchy(H, O.Hierarchy(s, **kw))


@pytest.mark.parametrize("interp,distance", [(O.P_LAIP, 2), (O.P_ONEPOINT, 2), (O.P_LAIP, 1)])
def test_two_level_refresh_of_backward_euler_equals_fresh_setup(interp, distance):
    """Sec. 4.1.1: I + dt S for a new dt has the level-0 structure of the old one, so with two levels
    (no coarse-level strength in play) the refreshed hierarchy is the set-up of the new matrix."""
    S = W.fd_adr_2d(40, 3 * math.pi / 16, 1e-2, 0.0)
    kw = dict(distance=distance, interp=interp, lump_tol=0.0, max_levels=2, coarse_max=10)
    A1, A2 = backward_euler(S, 0.05), backward_euler(S, 0.4)
    H = O.Hierarchy(A1, **kw)
    F = O.Hierarchy(A2, **kw)
    assert H.status == 0 and F.status == 0
    assert not np.array_equal(H.levels[1].A[2], F.levels[1].A[2])
    assert H.refresh(A2) == 0
    assert_same_hierarchy(H, F)


def test_refresh_row_scaling_by_powers_of_two_is_exact():
    """Sec. 3.1: with A~ = D A (D powers of two), R~ = D_c R D_f^{-1}, one-point P is unchanged and
    the coarse operator is D_c K -- exactly, on every level, lumping included."""
    s = W.config("fd2d_64", scale=24)
    rng = np.random.default_rng(5)
    d = 2.0 ** rng.integers(-4, 5, s.n)
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    s2 = with_values(s, s.val * d[rows], s.b * d)
    kw = dict(distance=2, cf_mode=O.CF_RS, lump_tol=1e-3, interp=O.P_ONEPOINT)
    H0 = O.Hierarchy(s, **kw)
    H = O.Hierarchy(s, **kw)
    assert H.refresh(s2) == 0
    dl = d
    for L0, L in zip(H0.levels, H.levels):
        r = np.repeat(np.arange(L0.n), np.diff(L0.A[0]))
        assert np.array_equal(L0.A[2] * dl[r], L.A[2])
        if L0.R is None:
            break
        Cpts = np.nonzero(L0.cf == 1)[0]
        rr = np.repeat(np.arange(L0.nc), np.diff(L0.R[0]))
        assert np.array_equal(L0.R[2] * dl[Cpts][rr] / dl[L0.R[1]], L.R[2])
        assert np.array_equal(L0.P[2], L.P[2])
        dl = dl[Cpts]


@pytest.mark.parametrize("kw", [
    dict(distance=2, interp=O.P_LAIP, lump_tol=1e-2),
    dict(distance=2, interp=O.P_ONEPOINT, lump_tol=1e-3, cf_mode=O.CF_PMIS),
])
def test_refreshed_operators_satisfy_their_defining_equations(kw):
    """Multilevel refresh from a reaction-dominated matrix to an advection-dominated one on the same
    pattern: every level's R, P and coarse operator are checked against the new matrix."""
    s1 = W.fd_adr_2d(48, 3 * math.pi / 16, 1e-3, 50.0)
    s2 = W.fd_adr_2d(48, 3 * math.pi / 16, 1e-3, 0.5)
    assert np.array_equal(s1.col, s2.col)
    H = O.Hierarchy(s1, **kw)
    old = [None if L.R is None else L.R[2].copy() for L in H.levels]
    assert H.status == 0 and H.refresh(s2) == 0
    lvl = H.levels
    assert np.array_equal(lvl[0].A[2], s2.val)
    changed = 0
    for l in range(len(lvl) - 1):
        L, Ln = lvl[l], lvl[l + 1]
        A = csr_to_scipy(L.A, (L.n, L.n))
        R = csr_to_scipy(L.R, (L.nc, L.n))
        P = csr_to_scipy(L.P, (L.n, L.nc))
        changed += not np.array_equal(old[l], L.R[2])
        scale = abs(A).max()
        Cpts = np.nonzero(L.cf == 1)[0]
        RA = (R @ A).tocsr()
        for c in range(L.nc):
            cols = L.R[1][L.R[0][c]:L.R[0][c + 1]]
            zs = np.abs(L.R[2][L.R[0][c]:L.R[0][c + 1]]).sum()
            for j in cols:
                if j != Cpts[c]:
                    assert abs(RA[c, int(j)]) <= 1e-12 * scale * max(1.0, zs)
        if kw["interp"] == O.P_LAIP:
            AP = (A @ P).tocsc()
            PT = P.T.tocsr()
            for c in range(L.nc):
                for j in PT.indices[PT.indptr[c]:PT.indptr[c + 1]]:
                    if j != Cpts[c]:
                        assert abs(AP[int(j), c]) <= 1e-11 * scale * max(1.0, abs(PT[c]).sum())
        # lumping (Sec. 3.3) of the exact triple product onto the kept pattern
        K = (R @ A @ P).toarray()
        Kl = csr_to_scipy(Ln.A, (L.nc, L.nc)).toarray()
        tol = 1e-13 * np.abs(K).max()
        np.testing.assert_allclose(Kl.sum(1), K.sum(1), rtol=0, atol=tol * 10)
        mask = Kl != 0
        np.fill_diagonal(mask, False)
        np.testing.assert_allclose(Kl[mask], K[mask], rtol=0, atol=tol)
    assert changed == len(lvl) - 1
    x, rep = H.solve(s2.b, tol=1e-10)
    assert rep["status"] == 0
    xd = spla.spsolve(s2.to_scipy().tocsc(), s2.b)
    assert np.abs(x - xd).max() <= 1e-7 * np.abs(xd).max()


def test_refresh_rejects_another_size():
    s = W.config("fd2d_64", scale=16)
    H = O.Hierarchy(s)
    t = W.config("fd2d_64", scale=20)
    assert H.refresh(t) != 0


def test_refresh_rejects_another_pattern():
    """Same size, different pattern: the kept structure does not apply, the refresh says so."""
    s = W.fd_adr_2d(16, 3 * math.pi / 16, 1e-3, 0.5)
    t = W.fd_adr_2d(16, 3 * math.pi / 16, 1e-3, 0.5)
    A = t.to_scipy().tolil()
    A[0, 17] = -0.01                  # one more entry in row 0
    t2 = W.CsrSystem(s.n, *(lambda M: (M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data))(
        A.tocsr()), s.b)
    H = O.Hierarchy(s)
    assert H.status == 0
    assert H.refresh(t2) != 0
