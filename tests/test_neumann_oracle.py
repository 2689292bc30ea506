"""Pins of the oracle's Neumann restriction (nAIR, Sec. 3.2) against what the paper and the mathematics fix.

nAIR of distance d (degree k = d - 1): Z = -A_cf sum_{m=0}^{k} (D_ff^{-1} E_ff)^m D_ff^{-1}, E_ff = D_ff - A_ff,
the paper's -A_cf sum L_ff^m for a unit-diagonal matrix. Expected values come from dense numpy products of
that formula, from the exact inverse where the series is finite (triangular A_ff), from exact power-of-two row
scaling, from ℓAIR on a chain (where the paper states the two coincide), and from the paper's Table 1 finding
that Neumann barely improves on Z = 0 for a recirculating flow while ℓAIR does.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import oracle as O


def csr_to_scipy(t, shape):
    rp, col, val = t
    return sp.csr_matrix((val, col.astype(np.int64), rp), shape=shape)


def system(M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    n = M.shape[0]
    return W.CsrSystem(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64),
                       np.ones(n))


def two_level(s, cf, d, **kw):
    H = O.Hierarchy(s, cf_user=cf, distance=d, restriction=O.R_NEUMANN, max_levels=2, coarse_max=2, lump_tol=0.0,
                    **kw)
    assert H.status == 0
    return H.levels[0]


def dense_neumann(A, cf, k):
    F, Cp = np.nonzero(cf == 0)[0], np.nonzero(cf == 1)[0]
    Aff = A[np.ix_(F, F)]
    D = np.diag(np.diag(Aff))
    Dinv = np.diag(1.0 / np.diag(Aff))
    T = Dinv @ (D - Aff)
    S = np.zeros_like(Aff)
    P = np.eye(len(F))
    for _ in range(k + 1):
        S += P
        P = P @ T
    return -A[np.ix_(Cp, F)] @ S @ Dinv, F, Cp


def random_cf(n, seed, frac=0.35):
    rng = np.random.default_rng(seed)
    cf = (rng.uniform(size=n) < frac).astype(np.int8)
    cf[0] = 1
    return cf


@pytest.mark.parametrize("d", [1, 2, 3])
def test_neumann_matches_the_dense_series(d):
    s = W.random_sparse(160, 5, seed=3)
    A = s.to_scipy().toarray()
    cf = random_cf(s.n, 1)
    L = two_level(s, cf, d)
    Z, F, Cp = dense_neumann(A, cf, d - 1)
    R = csr_to_scipy(L.R, (len(Cp), s.n)).toarray()
    assert np.array_equal(R[np.arange(len(Cp)), Cp], np.ones(len(Cp)))
    np.testing.assert_allclose(R[:, F], Z, rtol=0, atol=1e-13 * np.abs(Z).max())
    # the pattern is every F point within d edges of the C point through F points (graph of all nonzeros)
    G = (A != 0) & ~np.eye(s.n, dtype=bool)
    for c, i in enumerate(Cp):
        reach, front = set(), {int(i)}
        for _ in range(d):
            front = {int(j) for f in front for j in np.nonzero(G[f])[0] if cf[j] == 0} - reach
            reach |= front
        got = set(int(j) for j in L.R[1][L.R[0][c]:L.R[0][c + 1]]) - {int(i)}
        assert got == reach


def test_unit_lower_triangular_is_the_papers_formula_and_finite():
    """Sec. 3.2 as printed: A = I - L (L strictly lower), Z = -A_cf sum_{m<=k} L_ff^m; once k reaches the
    longest F path the series is the exact inverse and Z is ideal restriction."""
    rng = np.random.default_rng(7)
    n = 60
    Lm = np.tril(rng.uniform(-0.6, 0.6, (n, n)) * (rng.uniform(size=(n, n)) < 0.08), -1)
    A = np.eye(n) - Lm
    s = system(A)
    cf = random_cf(n, 2, 0.6)
    F, Cp = np.nonzero(cf == 0)[0], np.nonzero(cf == 1)[0]
    Lff = Lm[np.ix_(F, F)]
    for d in (1, 2, 3):
        L = two_level(s, cf, d)
        S = sum(np.linalg.matrix_power(Lff, m) for m in range(d))
        Z = -A[np.ix_(Cp, F)] @ S
        R = csr_to_scipy(L.R, (len(Cp), n)).toarray()
        np.testing.assert_allclose(R[:, F], Z, rtol=0, atol=1e-14 * max(1.0, np.abs(Z).max()))
    # longest path in the F graph: nilpotency index of L_ff
    depth = next(m for m in range(1, len(F) + 1) if not np.linalg.matrix_power(Lff, m).any())
    assert 2 <= depth <= 4
    for d in range(depth, 5):
        L = two_level(s, cf, d)
        Zi = -A[np.ix_(Cp, F)] @ np.linalg.inv(A[np.ix_(F, F)])
        R = csr_to_scipy(L.R, (len(Cp), n)).toarray()
        np.testing.assert_allclose(R[:, F], Zi, rtol=0, atol=1e-13 * max(1.0, np.abs(Zi).max()))


def test_neumann_row_scaling_by_powers_of_two_is_exact():
    """Z~ = D_c Z D_f^{-1} for A~ = D A (the unit-diagonal form is scaling-free), exactly."""
    s = W.random_sparse(200, 6, seed=9)
    d = 2.0 ** np.random.default_rng(4).integers(-3, 4, s.n)
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    s2 = W.CsrSystem(s.n, s.row_ptr.copy(), s.col.copy(), s.val * d[rows], s.b * d)
    cf = random_cf(s.n, 5)
    for dist in (1, 2):
        L1, L2 = two_level(s, cf, dist), two_level(s2, cf, dist)
        assert np.array_equal(L1.R[1], L2.R[1])
        Cp = np.nonzero(cf == 1)[0]
        rr = np.repeat(np.arange(len(Cp)), np.diff(L1.R[0]))
        assert np.array_equal(L1.R[2] * d[Cp][rr] / d[L1.R[1]], L2.R[2])


@pytest.mark.parametrize("d", [1, 2, 3])
def test_neumann_equals_lair_on_an_upwind_chain(d):
    """Sec. 3.2: for triangular (transport) matrices the two approximations coincide -- on a 1D upwind chain
    with two F points between C points, both eliminate every F point within distance d exactly."""
    s = W.upwind_chain(90)
    cf = np.zeros(s.n, np.int8)
    cf[::3] = 1
    Ln = two_level(s, cf, d)
    Hl = O.Hierarchy(s, cf_user=cf, distance=d, theta=0.0, max_levels=2, coarse_max=2, lump_tol=0.0)
    Ll = Hl.levels[0]
    assert np.array_equal(Ln.R[0], Ll.R[0]) and np.array_equal(Ln.R[1], Ll.R[1])
    np.testing.assert_allclose(Ln.R[2], Ll.R[2], rtol=1e-14, atol=1e-15)


def _ideal_error(s, d, restriction, **kw):
    H = O.Hierarchy(s, distance=d, restriction=restriction, max_levels=2, coarse_max=4, lump_tol=0.0, **kw)
    L = H.levels[0]
    A = s.to_scipy().toarray()
    F, Cp = np.nonzero(L.cf == 0)[0], np.nonzero(L.cf == 1)[0]
    Zi = -A[np.ix_(Cp, F)] @ np.linalg.inv(A[np.ix_(F, F)])
    Z = csr_to_scipy(L.R, (len(Cp), s.n)).toarray()[:, F]
    return np.linalg.norm(Z - Zi) / np.linalg.norm(Zi)


def test_recirculating_flow_neumann_is_no_better_than_zero():
    """Table 1 (Sec. 3.2): on a recirculating flow the Neumann approximation is hardly closer to ideal
    restriction than Z = 0 (relative error about 1), while ℓAIR is, and improves with distance."""
    s = W.dg_p2_advection(10)
    kw = dict(strength_abs=1)
    en = [_ideal_error(s, d, O.R_NEUMANN, **kw) for d in (1, 2)]
    el = [_ideal_error(s, d, O.R_LAIR, **kw) for d in (1, 2)]
    assert min(en) > 0.95
    assert el[1] < el[0] < 0.8


def test_neumann_hierarchy_solves_and_refreshes():
    s = W.config("fd2d_64", scale=40)
    kw = dict(distance=2, restriction=O.R_NEUMANN)
    H = O.Hierarchy(s, **kw)
    assert H.status == 0
    x, rep = H.solve(s.b, tol=1e-10)
    assert rep["status"] == 0
    assert np.linalg.norm(s.b - s.to_scipy() @ x) <= 1.5e-10 * np.linalg.norm(s.b)
    G = O.Hierarchy(s, **kw)
    assert G.refresh(s) == 0
    for L1, L2 in zip(H.levels, G.levels):
        for a, b in zip(L1.A, L2.A):
            assert np.array_equal(a, b)
        if L1.R is not None:
            for a, b in zip(L1.R, L2.R):
                assert np.array_equal(a, b)
