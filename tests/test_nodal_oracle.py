"""Pins of the oracle's nodal (block) hierarchy: Sec. 3.1 (k x k blocks) and Sec. 4.2.1 approach (iii).

Expected values come from the Kronecker structure A_s (x) I_k (every block a multiple of the identity, so the
nodal method must reproduce the scalar method on A_s in abs mode, tensored with I_k), from the exact block
ideal restriction when the neighbourhoods cover every F node, from scipy's triple product with the block
lumping rule, from a two-grid cycle written out in numpy with block Jacobi, and from the paper's finding that
treating DG nodally converges like block-diagonal scaling while ignoring the blocks does not.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import oracle as O


def csr_to_scipy(t, shape):
    rp, col, val = t
    return sp.csr_matrix((val, col.astype(np.int64), rp), shape=shape)


def system(M, b=None):
    M = sp.csr_matrix(M)
    M.sort_indices()
    n = M.shape[0]
    return W.CsrSystem(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64),
                       np.ones(n) if b is None else b)


@pytest.mark.parametrize("k,interp", [(2, O.P_ONEPOINT), (3, O.P_ONEPOINT), (2, O.P_LAIP)])
def test_kronecker_identity_blocks_reproduce_the_scalar_method(k, interp):
    """A = A_s (x) I_k: block norms are sqrt(k)|a|, every local block system splits into k copies of the
    scalar one, so every operator of the nodal hierarchy is the scalar (abs-mode) one tensored with I_k."""
    s = W.fd_adr_2d(20, 3 * math.pi / 16, 1e-2, 0.5)
    As = s.to_scipy()
    A = sp.kron(As, sp.identity(k), format="csr")
    big = system(A)
    kw = dict(distance=2, interp=interp, cf_mode=O.CF_RS, lump_tol=1e-2)
    Hs = O.Hierarchy(s, strength_abs=1, coarse_max=20, **kw)
    Hn = O.Hierarchy(big, nodal=k, coarse_max=20 * k, **kw)
    assert Hs.status == 0 and Hn.status == 0
    assert len(Hs.levels) == len(Hn.levels)
    for Ls, Ln in zip(Hs.levels, Hn.levels):
        ref = sp.kron(csr_to_scipy(Ls.A, (Ls.n, Ls.n)), sp.identity(k), format="csr")
        ref.sort_indices()
        got = csr_to_scipy(Ln.A, (Ln.n, Ln.n))
        assert abs(got - ref).max() <= 1e-14 * abs(ref).max()
        if Ls.R is None:
            break
        assert np.array_equal(np.repeat(Ls.cf, k), Ln.cf)
        for name, shape_s in (("R", (Ls.nc, Ls.n)), ("P", (Ls.n, Ls.nc))):
            ref = sp.kron(csr_to_scipy(getattr(Ls, name), shape_s), sp.identity(k), format="csr")
            got = csr_to_scipy(getattr(Ln, name), (shape_s[0] * k, shape_s[1] * k))
            assert abs(got - ref).max() <= 1e-14 * max(1.0, abs(ref).max()), name


def test_full_block_neighbourhoods_give_block_ideal_restriction():
    """Sec. 3.1 with blocks: when each C node's neighbourhood holds every F node, R_F = -A_cf A_ff^{-1}."""
    rng = np.random.default_rng(4)
    k, N = 3, 12
    A = rng.uniform(-1, 0, (N * k, N * k))
    for I in range(N):
        A[I * k:(I + 1) * k, I * k:(I + 1) * k] = rng.uniform(-1, 1, (k, k)) + 4 * k * N * np.eye(k)
    s = system(A)
    cfB = np.zeros(N, np.int8)
    cfB[[0, 4, 9]] = 1
    cf = np.repeat(cfB, k)
    H = O.Hierarchy(s, nodal=k, cf_user=cf, distance=1, theta=0.0, max_levels=2, coarse_max=2, lump_tol=0.0)
    assert H.status == 0
    L = H.levels[0]
    F, C = np.nonzero(cf == 0)[0], np.nonzero(cf == 1)[0]
    Zi = -A[np.ix_(C, F)] @ np.linalg.inv(A[np.ix_(F, F)])
    R = csr_to_scipy(L.R, (len(C), s.n)).toarray()
    np.testing.assert_allclose(R[:, F], Zi, rtol=0, atol=1e-13 * np.abs(Zi).max())
    np.testing.assert_array_equal(R[:, C], np.eye(len(C)))


def test_block_lumping_keeps_row_sums_and_kept_blocks():
    s = W.dg_p2_advection(8)
    k = 6
    H0 = O.Hierarchy(s, nodal=k, distance=2, interp=O.P_ONEPOINT, lump_tol=0.0, max_levels=2, coarse_max=10)
    H1 = O.Hierarchy(s, nodal=k, distance=2, interp=O.P_ONEPOINT, lump_tol=0.05, max_levels=2, coarse_max=10)
    L0 = H0.levels[0]
    A = csr_to_scipy(L0.A, (L0.n, L0.n))
    K = (csr_to_scipy(L0.R, (L0.nc, L0.n)) @ A @ csr_to_scipy(L0.P, (L0.n, L0.nc))).toarray()
    K1 = csr_to_scipy(H1.levels[1].A, (L0.nc, L0.nc)).toarray()
    n = K.shape[0]
    np.testing.assert_allclose(K1.sum(1), K.sum(1), rtol=0, atol=1e-13 * np.abs(K).max())
    N = n // k
    norms = np.array([[np.linalg.norm(K[I * k:(I + 1) * k, J * k:(J + 1) * k]) for J in range(N)] for I in range(N)])
    dropped = 0
    for I in range(N):
        thr = 0.05 * norms[I].max()
        for J in range(N):
            blk = slice(J * k, (J + 1) * k)
            rows = slice(I * k, (I + 1) * k)
            if J == I:
                continue
            if norms[I, J] < thr:
                assert not K1[rows, blk].any()
                dropped += norms[I, J] > 0
            else:
                np.testing.assert_allclose(K1[rows, blk], K[rows, blk], rtol=0, atol=1e-13 * np.abs(K).max())
    assert dropped > 0
    # the diagonal blocks took the dropped blocks entrywise
    for I in range(N):
        rows = slice(I * k, (I + 1) * k)
        add = sum(K[rows, J * k:(J + 1) * k] for J in range(N) if J != I and norms[I, J] < 0.05 * norms[I].max())
        np.testing.assert_allclose(K1[rows, rows], K[rows, rows] + add, rtol=0, atol=1e-13 * np.abs(K).max())


@pytest.mark.parametrize("prec", [0, 1])
def test_two_grid_cycle_with_block_jacobi(prec):
    """Sec. 4 cycle on a nodal hierarchy: x = P K^{-1} R b, then block Jacobi over F, F, C nodes:
    x_I += D_I^{-1} (b - A x)_I with every update of a sweep reading the old x."""
    s = W.dg_p2_advection(6)
    k = 6
    H = O.Hierarchy(s, nodal=k, distance=2, interp=O.P_ONEPOINT, max_levels=2, coarse_max=10, prec=prec)
    assert H.status == 0
    L0, L1 = H.levels
    A = csr_to_scipy(L0.A, (L0.n, L0.n)).toarray()
    R = csr_to_scipy(L0.R, (L0.nc, L0.n)).toarray()
    P = csr_to_scipy(L0.P, (L0.n, L0.nc)).toarray()
    K = csr_to_scipy(L1.A, (L1.n, L1.n)).toarray()
    b = np.random.default_rng(1).uniform(-1, 1, s.n)
    x = P @ np.linalg.solve(K, R @ b)
    N = s.n // k
    for tgt in (0, 0, 1):
        r = b - A @ x
        xn = x.copy()
        for I in range(N):
            if L0.cf[I * k] != tgt:
                continue
            sl = slice(I * k, (I + 1) * k)
            xn[sl] = x[sl] + np.linalg.solve(A[sl, sl], r[sl])
        x = xn
    z = H.precond(b)
    tol = 1e-5 if prec else 1e-11
    assert np.linalg.norm(z - x) <= tol * np.linalg.norm(x)


def test_nodal_dg_converges_like_block_scaling_and_scalar_does_not():
    """Sec. 4.2.1: for advection-dominated DG, the nodal hierarchy converges about as well as one built
    on the block-diagonally scaled matrix, while ignoring the block structure does not."""
    s = W.dg_p2_advection(12)
    _, rn = O.Hierarchy(s, nodal=6, distance=2, interp=O.P_ONEPOINT).solve(s.b, tol=1e-8, max_iter=300)
    _, rb = O.Hierarchy(s, block_size=6, distance=2, interp=O.P_ONEPOINT, strength_abs=1).solve(s.b, tol=1e-8,
                                                                                                max_iter=300)
    _, rs = O.Hierarchy(s, distance=2, interp=O.P_ONEPOINT, strength_abs=1).solve(s.b, tol=1e-8, max_iter=300)
    assert rn["status"] == 0 and rb["status"] == 0
    assert rn["iters"] <= rb["iters"] + 1
    assert rs["status"] != 0 or rs["iters"] >= 5 * rn["iters"]


def test_nodal_refresh_and_defining_equation():
    s1 = W.dg_p2_advection(10)
    s2 = W.dg_p2_advection(10, dt=0.5 / 10)
    kw = dict(nodal=6, distance=2, interp=O.P_ONEPOINT)
    H = O.Hierarchy(s1, **kw)
    G = O.Hierarchy(s1, **kw)
    assert G.refresh(s1) == 0
    for L1, L2 in zip(H.levels, G.levels):
        for a, b in zip(L1.A, L2.A):
            assert np.array_equal(a, b)
    assert G.refresh(s2) == 0
    L = G.levels[0]
    A = csr_to_scipy(L.A, (L.n, L.n))
    R = csr_to_scipy(L.R, (L.nc, L.n))
    RA = (R @ A).toarray()
    Cp = np.nonzero(L.cf == 1)[0]
    for c in range(0, L.nc, 7):
        for j in L.R[1][L.R[0][c]:L.R[0][c + 1]]:
            if j != Cp[c]:
                assert abs(RA[c, j]) <= 1e-12 * abs(A).max() * max(1.0, np.abs(L.R[2][L.R[0][c]:L.R[0][c + 1]]).sum())
    x, rep = G.solve(s2.b, tol=1e-10)
    assert rep["status"] == 0
    assert np.linalg.norm(s2.b - s2.to_scipy() @ x) <= 1.5e-10 * np.linalg.norm(s2.b)


def test_nodal_rejects_what_it_does_not_combine_with():
    s = W.dg_p2_advection(4)
    assert O.Hierarchy(s, nodal=6, block_size=6).status == 1
    assert O.Hierarchy(s, nodal=6, restriction=O.R_NEUMANN).status == 1
    assert O.Hierarchy(s, nodal=7).status == 1
