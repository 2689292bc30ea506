"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks. None of them re-derives an expected value
by calling the oracle a second way: the expected values come from closed forms
(ideal restriction/interpolation, Schur complements, the two-grid spectrum),
from hand derivations (tests/golden), from numpy/scipy dense linear algebra, or
from exact invariants (row scaling by powers of two).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_to_scipy(t, shape):
    rp, col, val = t
    return sp.csr_matrix((val, col.astype(np.int64), rp), shape=shape)


def dense_system(n, seed, dominance=2.0):
    """Dense, diagonally dominant, nonsymmetric matrix (every pair connected)."""
    rng = np.random.default_rng(seed)
    A = -rng.uniform(0.1, 1.0, (n, n))
    np.fill_diagonal(A, 0.0)
    np.fill_diagonal(A, dominance * np.abs(A).sum(1))
    S = sp.csr_matrix(A)
    S.sort_indices()
    return W.CsrSystem(n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.copy(),
                       rng.uniform(-1, 1, n))


def system_from_scipy(M, b=None):
    M = sp.csr_matrix(M)
    M.sort_indices()
    n = M.shape[0]
    return W.CsrSystem(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64),
                       np.zeros(n) if b is None else b)


# --------------------------------------------------------------------------------------
# strength of connection (Sec. 4, hard-minimum definition of N_i)
# --------------------------------------------------------------------------------------

def test_strength_fd_stencil_hand_derived():
    # 64x64 FD, angle 3pi/16, eps 1e-4: h = 1/65, eps/h^2 = 0.4225,
    # west = -0.4225 - cos(3pi/16)*65, south = -0.4225 - sin(3pi/16)*65, east = north = -0.4225.
    s = W.config("fd2d_64")
    A = s.to_scipy()
    i = 64 * 10 + 10
    row = A[i].toarray()[0]
    west = -0.4225 - math.cos(3 * math.pi / 16) * 65
    south = -0.4225 - math.sin(3 * math.pi / 16) * 65
    assert row[i - 1] == pytest.approx(west, rel=1e-14)
    assert row[i - 64] == pytest.approx(south, rel=1e-14)
    assert row[i + 1] == pytest.approx(-0.4225, rel=1e-12)
    mask = O.strength(s, 0.25)
    cols = s.col[s.row_ptr[i]:s.row_ptr[i + 1]]
    strong = set(cols[mask[s.row_ptr[i]:s.row_ptr[i + 1]] == 1].tolist())
    # theta * max = 0.25 * 54.468 = 13.6 -> only the two upstream neighbours are strong
    assert strong == {i - 1, i - 64}


def test_strength_rules():
    # row 0: diag 4, off-diagonals -2 (strong), -0.4 (weak at theta .25), +3 (positive: not strong signed),
    # explicit zero (never strong)
    M = sp.csr_matrix(np.array([[4.0, -2.0, -0.4, 3.0, 0.0],
                                [0, 1, 0, 0, 0], [0, 0, 1, 0, 0], [0, 0, 0, 1, 0], [0, 0, 0, 0, 1]]))
    M = sp.csr_matrix((np.array([4.0, -2.0, -0.4, 3.0, 0.0, 1, 1, 1, 1]),
                       np.array([0, 1, 2, 3, 4, 1, 2, 3, 4]), np.array([0, 5, 6, 7, 8, 9])), shape=(5, 5))
    s = system_from_scipy(M)
    s = W.CsrSystem(5, np.array([0, 5, 6, 7, 8, 9], np.int64), np.array([0, 1, 2, 3, 4, 1, 2, 3, 4], np.int32),
                    np.array([4.0, -2.0, -0.4, 3.0, 0.0, 1, 1, 1, 1]), np.zeros(5))
    m = O.strength(s, 0.25)
    assert m[:5].tolist() == [0, 1, 0, 0, 0]          # max |a_ik| = 3 -> threshold .75
    m = O.strength(s, 0.25, absmode=True)
    assert m[:5].tolist() == [0, 1, 0, 1, 0]
    m = O.strength(s, 0.0, absmode=True)               # theta 0: every stored nonzero off-diagonal
    assert m[:5].tolist() == [0, 1, 1, 1, 0]
    assert m[5:].tolist() == [0, 0, 0, 0]              # rows without off-diagonals


# --------------------------------------------------------------------------------------
# C/F splitting (Sec. 4: classical first pass, no second pass) and PMIS
# --------------------------------------------------------------------------------------

def read_golden_chain():
    d = {}
    for line in open(os.path.join(GOLDEN, "chain8.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        d[k] = v
    return d


def test_rs_chain_golden():
    g = read_golden_chain()
    s = W.upwind_chain(8)
    cf = O.cf_split(s, O.strength(s, 0.25), O.CF_RS)
    assert cf.tolist() == [int(v) for v in g["cf"]]


def test_chain_hierarchy_golden_is_ideal():
    """Sec. 3.2: for triangular A with A_ff diagonal, distance-one lAIR is exact ideal restriction."""
    g = read_golden_chain()
    s = W.upwind_chain(8)
    H = O.Hierarchy(s, cf_mode=O.CF_RS, coarse_max=2, max_levels=2, lump_tol=0.0)
    L = H.levels[0]
    assert L.cf.tolist() == [int(v) for v in g["cf"]]
    R = csr_to_scipy(L.R, (4, 8)).toarray()
    P = csr_to_scipy(L.P, (8, 4)).toarray()
    for r in range(4):
        v = g[f"R{r}"]
        exp = np.zeros(8)
        for k in range(0, len(v), 2):
            exp[int(v[k])] = float(v[k + 1])
        assert np.array_equal(R[r], exp)
    for r in range(8):
        v = g[f"P{r}"]
        exp = np.zeros(4)
        exp[int(v[0])] = float(v[1])
        assert np.array_equal(P[r], exp)


def _graph(s, mask):
    S = [set() for _ in range(s.n)]
    for i in range(s.n):
        for k in range(s.row_ptr[i], s.row_ptr[i + 1]):
            if mask[k]:
                S[i].add(int(s.col[k]))
    ST = [set() for _ in range(s.n)]
    for i in range(s.n):
        for j in S[i]:
            ST[j].add(i)
    return S, ST


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rs_invariants_and_greedy_order(seed):
    """Every F point has a strong C dependency (or no connections at all), and the
    C points were taken greedily: replaying the splitting with a plain O(n^2) scan
    of lambda gives the same result (a second, independent implementation)."""
    s = W.fd_adr_2d(12, seed * 1.3 + 0.2, 10.0 ** (-seed - 1), 0.1)
    mask = O.strength(s, 0.25)
    cf = O.cf_split(s, mask, O.CF_RS)
    S, ST = _graph(s, mask)
    for i in range(s.n):
        if cf[i] == O.CF_F and (S[i] or ST[i]):
            assert any(cf[j] == O.CF_C for j in S[i])
    # brute-force replay
    lam = [len(ST[i]) for i in range(s.n)]
    st = ["U"] * s.n
    for i in range(s.n):
        if not S[i] and not ST[i]:
            st[i] = "F"
    while "U" in st:
        best = max((lam[i], -i) for i in range(s.n) if st[i] == "U")
        i = -best[1]
        st[i] = "C"
        for j in sorted(ST[i]):
            if st[j] == "U":
                st[j] = "F"
                for k in S[j]:
                    if st[k] == "U":
                        lam[k] += 1
        for k in S[i]:
            if st[k] == "U":
                lam[k] -= 1
    assert [1 if v == "C" else 0 for v in st] == cf.tolist()


@pytest.mark.parametrize("B", [7, 40, 1000])
def test_blocked_first_pass_replay(B):
    """The first pass run independently on index blocks: lambda and updates count only
    in-block strong connections; one block covering every point is the classical pass."""
    s = W.fd_adr_2d(14, 0.9, 1e-3, 0.1)
    mask = O.strength(s, 0.25)
    cf = O.cf_split(s, mask, O.CF_AUTO, seed=B)
    if B >= s.n:
        assert np.array_equal(cf, O.cf_split(s, mask, O.CF_RS))
    S, ST = _graph(s, mask)
    out = []
    for b0 in range(0, s.n, B):
        blk = range(b0, min(s.n, b0 + B))
        inb = lambda j: b0 <= j < b0 + B
        lam = {i: sum(1 for j in ST[i] if inb(j)) for i in blk}
        st = {i: ("F" if not S[i] and not ST[i] else "U") for i in blk}
        while "U" in st.values():
            i = -max((lam[i], -i) for i in blk if st[i] == "U")[1]
            st[i] = "C"
            for j in sorted(ST[i]):
                if inb(j) and st[j] == "U":
                    st[j] = "F"
                    for k in S[j]:
                        if inb(k) and st[k] == "U":
                            lam[k] += 1
            for k in S[i]:
                if inb(k) and st[k] == "U":
                    lam[k] -= 1
        out += [1 if st[i] == "C" else 0 for i in blk]
    assert out == cf.tolist()
    # every F point with connections depends on a C point
    for i in range(s.n):
        if cf[i] == 0 and (S[i] or ST[i]):
            assert any(cf[j] == 1 for j in S[i])


def test_pmis_weight_splitmix64_vector():
    # splitmix64 (Vigna): the first output of the generator seeded with 0 is 0xE220A8397B1DCDAF
    u = O.pmis_weight(0, 0, 0)
    assert u == (0xE220A8397B1DCDAF >> 11) * 2.0 ** -53
    assert O.pmis_weight(7, 123, 5) >= 7.0 and O.pmis_weight(7, 123, 5) < 8.0


def _splitmix64(x):
    m = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


@pytest.mark.parametrize("seed", [0, 3])
def test_pmis_replay_and_maximal(seed):
    """PMIS rounds replayed in plain Python from the definition (hashed weights, synchronous
    rounds); F points either influence nobody or depend on a C point."""
    s = W.fd_adr_2d(20, 0.7 + seed, 1e-3, 0.1)
    mask = O.strength(s, 0.25)
    cf = O.cf_split(s, mask, O.CF_PMIS, seed=seed)
    S, ST = _graph(s, mask)
    w = [len(ST[i]) + (_splitmix64(((seed << 32) ^ i) & ((1 << 64) - 1)) >> 11) * 2.0 ** -53 for i in range(s.n)]
    st = ["F" if len(ST[i]) == 0 else "U" for i in range(s.n)]
    while "U" in st:
        new_c = [i for i in range(s.n) if st[i] == "U" and
                 all(st[j] != "U" or (w[i], -i) > (w[j], -j) for j in S[i] | ST[i])]
        assert new_c
        for i in new_c:
            st[i] = "C"
        for i in new_c:
            for j in ST[i]:
                if st[j] == "U":
                    st[j] = "F"
    assert [1 if v == "C" else 0 for v in st] == cf.tolist()
    for i in range(s.n):
        if cf[i] == O.CF_F:
            assert len(ST[i]) == 0 or any(cf[j] == O.CF_C for j in S[i])


# --------------------------------------------------------------------------------------
# local systems (Sec. 3.1, Eq. (3.2)) and the least-squares branch (Sec. 3.1 footnote)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("s", [1, 2, 5, 17, 40, 64])
def test_local_solve_matches_dense_solve(s):
    rng = np.random.default_rng(s)
    M = rng.standard_normal((s, s)) + s * np.eye(s) * 0.3
    rhs = rng.standard_normal(s)
    z, ls = O.local_solve(M, rhs)
    assert not ls
    ref = np.linalg.solve(M, rhs)
    assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref) * np.linalg.cond(M)


def test_local_solve_pivoting_needed():
    M = np.array([[0.0, 1.0, 2.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    rhs = np.array([1.0, 2.0, 3.0])
    z, ls = O.local_solve(M, rhs)
    assert not ls
    np.testing.assert_allclose(z, np.linalg.solve(M, rhs), rtol=1e-14)


@pytest.mark.parametrize("s", [2, 6, 33])
def test_local_solve_singular_is_min_norm_least_squares(s):
    rng = np.random.default_rng(10 + s)
    M = rng.standard_normal((s, s))
    M[:, -1] = M[:, 0]                    # duplicate column -> rank s-1
    rhs = rng.standard_normal(s)
    z, ls = O.local_solve(M, rhs)
    assert ls
    ref = np.linalg.lstsq(M, rhs, rcond=None)[0]
    assert np.linalg.norm(z - ref) <= 1e-11 * max(1.0, np.linalg.norm(ref))


def test_local_solve_zero_matrix():
    z, ls = O.local_solve(np.zeros((3, 3)), np.ones(3))
    assert ls and np.all(z == 0)


def test_local_solve_f32():
    rng = np.random.default_rng(4)
    s = 12
    M = (rng.standard_normal((s, s)) + 3 * np.eye(s)).astype(np.float32)
    rhs = rng.standard_normal(s).astype(np.float32)
    z, ls = O.local_solve(M, rhs, f32=True)
    assert z.dtype == np.float32 and not ls
    ref = np.linalg.solve(M.astype(np.float64), rhs.astype(np.float64))
    assert np.linalg.norm(z - ref) <= 1e-5 * np.linalg.norm(ref) * np.linalg.cond(M)


# --------------------------------------------------------------------------------------
# lAIR on the full pattern is ideal restriction (Eq. (2.8)); lAIP is ideal interpolation
# (Eq. (2.6)); Galerkin products reduce to the Schur complement (Sec. 2.2, Sec. 3.1)
# --------------------------------------------------------------------------------------

def _split(n, seed):
    rng = np.random.default_rng(seed)
    cf = np.zeros(n, np.int8)
    cf[rng.choice(n, n // 3, replace=False)] = 1
    return cf


@pytest.mark.parametrize("n,seed", [(30, 0), (48, 1)])
def test_full_pattern_gives_ideal_operators(n, seed):
    s = dense_system(n, seed)
    cf = _split(n, seed)
    H = O.Hierarchy(s, cf_user=cf, theta=0.0, theta_cf=0.0, strength_abs=1, distance=1,
                    lump_tol=0.0, coarse_max=n - 1, max_levels=2, interp=O.P_LAIP)
    assert H.status == 0
    L = H.levels[0]
    A = s.to_scipy().toarray()
    Fi = np.nonzero(cf == 0)[0]
    Ci = np.nonzero(cf == 1)[0]
    nc = len(Ci)
    Aff, Afc, Acf, Acc = A[np.ix_(Fi, Fi)], A[np.ix_(Fi, Ci)], A[np.ix_(Ci, Fi)], A[np.ix_(Ci, Ci)]
    R = csr_to_scipy(L.R, (nc, n)).toarray()
    P = csr_to_scipy(L.P, (n, nc)).toarray()
    Zideal = -Acf @ np.linalg.inv(Aff)
    Wideal = -np.linalg.inv(Aff) @ Afc
    np.testing.assert_allclose(R[:, Fi], Zideal, rtol=0, atol=1e-12 * np.abs(Zideal).max())
    np.testing.assert_array_equal(R[:, Ci], np.eye(nc))
    np.testing.assert_allclose(P[Fi, :], Wideal, rtol=0, atol=1e-12 * np.abs(Wideal).max())
    np.testing.assert_array_equal(P[Ci, :], np.eye(nc))
    K = csr_to_scipy(H.levels[1].A, (nc, nc)).toarray()
    Schur = Acc - Acf @ np.linalg.inv(Aff) @ Afc
    np.testing.assert_allclose(K, Schur, rtol=0, atol=1e-11 * np.abs(Schur).max())


def test_ideal_R_gives_schur_for_any_P():
    """R_ideal A = (0, S_A) (Sec. 3.1) so R_ideal A P = S_A for any W: one-point P here."""
    n = 36
    s = dense_system(n, 7)
    cf = _split(n, 7)
    H = O.Hierarchy(s, cf_user=cf, theta=0.0, theta_cf=0.0, strength_abs=1, lump_tol=0.0,
                    coarse_max=n - 1, max_levels=2, interp=O.P_ONEPOINT)
    A = s.to_scipy().toarray()
    Fi, Ci = np.nonzero(cf == 0)[0], np.nonzero(cf == 1)[0]
    Schur = A[np.ix_(Ci, Ci)] - A[np.ix_(Ci, Fi)] @ np.linalg.inv(A[np.ix_(Fi, Fi)]) @ A[np.ix_(Fi, Ci)]
    K = csr_to_scipy(H.levels[1].A, Schur.shape).toarray()
    np.testing.assert_allclose(K, Schur, rtol=0, atol=1e-11 * np.abs(Schur).max())


def test_one_point_interpolation_strongest_c():
    """Sec. 4: each F point takes the value of its strongest C neighbour."""
    s = W.config("fd2d_64", scale=16)
    H = O.Hierarchy(s, cf_mode=O.CF_RS, interp=O.P_ONEPOINT, max_levels=2, coarse_max=10)
    L = H.levels[0]
    A = s.to_scipy()
    mask = O.strength(s, 0.25)
    cidx = np.cumsum(L.cf == 1) - 1
    P = csr_to_scipy(L.P, (s.n, L.nc)).toarray()
    for j in range(s.n):
        if L.cf[j] == 1:
            assert P[j].tolist() == np.eye(L.nc)[cidx[j]].tolist()
            continue
        cand = [(-A[j, c], -c) for k in range(s.row_ptr[j], s.row_ptr[j + 1])
                if mask[k] and L.cf[(c := int(s.col[k]))] == 1]
        if not cand:
            assert not P[j].any()
        else:
            c = -max(cand)[1]
            assert P[j].tolist() == np.eye(L.nc)[cidx[c]].tolist()


# --------------------------------------------------------------------------------------
# defining invariant (RA)_{i,j} = 0 on the pattern of R (Sec. 3.1, Eq. (3.1))
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("cfg,kw", [
    ("fd2d_64", dict(distance=1)),
    ("fd2d_64", dict(distance=2)),
    ("fd2d_64", dict(distance=2, cf_mode=O.CF_PMIS)),
    ("fd2d_64", dict(distance=3)),
    ("fd2d_64", dict(distance=4, cf_mode=O.CF_PMIS)),
])
def test_RA_zero_on_pattern_every_level(cfg, kw):
    s = W.config(cfg, scale=32)
    H = O.Hierarchy(s, **kw)
    assert H.status == 0
    for L in H.levels[:-1]:
        A = csr_to_scipy(L.A, (L.n, L.n))
        R = csr_to_scipy(L.R, (L.nc, L.n))
        RA = (R @ A).tocsr()
        scale = abs(A).max()
        Cpts = np.nonzero(L.cf == 1)[0]
        for c in range(L.nc):
            for k in range(L.R[0][c], L.R[0][c + 1]):
                j = int(L.R[1][k])
                if j == Cpts[c]:
                    continue
                assert abs(RA[c, j]) <= 1e-12 * scale * max(1.0, np.abs(L.R[2][L.R[0][c]:L.R[0][c + 1]]).sum())


def test_larger_neighbourhood_is_more_accurate():
    """Sec. 3.1: a larger neighbourhood approximates ideal restriction better (Table 1 metric)."""
    # diffusive stencil and a PMIS splitting, so that A_ff is not diagonal and distance two adds F points
    s = W.fd_adr_2d(12, 3 * math.pi / 16, 1.0, 0.1)
    errs = []
    A = s.to_scipy().toarray()
    cf = None
    for k in (1, 2, 3, 4):
        H = O.Hierarchy(s, distance=k, cf_mode=O.CF_PMIS, max_levels=2, coarse_max=4, lump_tol=0.0)
        L = H.levels[0]
        cf = L.cf if cf is None else cf
        assert (L.cf == cf).all()
        Fi, Ci = np.nonzero(cf == 0)[0], np.nonzero(cf == 1)[0]
        Zi = -A[np.ix_(Ci, Fi)] @ np.linalg.inv(A[np.ix_(Fi, Fi)])
        Z = csr_to_scipy(L.R, (len(Ci), s.n)).toarray()[:, Fi]
        errs.append(np.linalg.norm(Z - Zi) / np.linalg.norm(Zi))
    assert errs[3] < errs[2] < errs[1] < errs[0] < 1.0


@pytest.mark.parametrize("distance", [1, 2, 3, 4])
def test_neighbourhoods_are_strong_F_paths(distance):
    """Sec. 3.1 / Sec. 4: the neighbourhood of C point i is every F point reachable from i by a path
    of at most `distance` strong edges whose points after i are all F -- checked by enumerating the
    paths directly on a small random graph (R's pattern is the neighbourhood plus i itself)."""
    s = W.random_sparse(300, 5, seed=11)
    H = O.Hierarchy(s, distance=distance, cf_mode=O.CF_PMIS, max_levels=2, coarse_max=4, lump_tol=0.0)
    L = H.levels[0]
    rp, col, _ = L.A
    strong = np.asarray(L.strong).astype(bool)
    nbrs = [col[rp[i]:rp[i + 1]][strong[rp[i]:rp[i + 1]]] for i in range(L.n)]
    Cpts = np.nonzero(L.cf == 1)[0]
    for c, i in enumerate(Cpts):
        reach, frontier = set(), [i]
        for _ in range(distance):
            nxt = []
            for j in frontier:
                for k in nbrs[j]:
                    k = int(k)
                    if L.cf[k] == 0 and k not in reach:
                        reach.add(k)
                        nxt.append(k)
            frontier = nxt
        got = set(int(j) for j in L.R[1][L.R[0][c]:L.R[0][c + 1]]) - {int(i)}
        assert got == reach


# --------------------------------------------------------------------------------------
# row-scaling invariance (Sec. 3.1, Remark): Z~ = D_c Z D_f^{-1}, R~ A~ P = D_c R A P
# --------------------------------------------------------------------------------------

def test_row_scaling_invariance_exact():
    s = W.config("fd2d_64", scale=24)
    rng = np.random.default_rng(3)
    d = 2.0 ** rng.integers(-4, 5, s.n)          # powers of two: scaling is exact in floating point
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    s2 = W.CsrSystem(s.n, s.row_ptr.copy(), s.col.copy(), s.val * d[rows], s.b * d)
    # one-point P is exactly invariant, so the whole hierarchy scales bit for bit
    kw = dict(distance=2, cf_mode=O.CF_RS, lump_tol=1e-3, interp=O.P_ONEPOINT)
    H1 = O.Hierarchy(s, **kw)
    H2 = O.Hierarchy(s2, **kw)
    assert len(H1.levels) == len(H2.levels)
    dl = d
    for L1, L2 in zip(H1.levels, H2.levels):
        assert np.array_equal(L1.A[0], L2.A[0]) and np.array_equal(L1.A[1], L2.A[1])
        r = np.repeat(np.arange(L1.n), np.diff(L1.A[0]))
        assert np.array_equal(L1.A[2] * dl[r], L2.A[2])
        if L1.R is None:
            break
        assert np.array_equal(L1.cf, L2.cf)
        assert np.array_equal(L1.R[1], L2.R[1]) and np.array_equal(L1.P[1], L2.P[1])
        Cpts = np.nonzero(L1.cf == 1)[0]
        rr = np.repeat(np.arange(L1.nc), np.diff(L1.R[0]))
        assert np.array_equal(L1.R[2] * dl[Cpts][rr] / dl[L1.R[1]], L2.R[2])
        assert np.array_equal(L1.P[2], L2.P[2])
        dl = dl[Cpts]
    # lAIP: W solves A_QQ w = -A_Qc, invariant under row scaling up to rounding (pivot order may change)
    kw = dict(distance=2, cf_mode=O.CF_RS, lump_tol=0.0, interp=O.P_LAIP, max_levels=2, coarse_max=10)
    P1 = O.Hierarchy(s, **kw).levels[0].P
    P2 = O.Hierarchy(s2, **kw).levels[0].P
    assert np.array_equal(P1[1], P2[1])
    np.testing.assert_allclose(P2[2], P1[2], rtol=1e-12)


# --------------------------------------------------------------------------------------
# Galerkin product and lumping (Sec. 2.1, Sec. 3.3)
# --------------------------------------------------------------------------------------

def test_rap_matches_sparse_triple_product():
    s = W.config("fd2d_64", scale=40)
    H = O.Hierarchy(s, distance=2, lump_tol=0.0)
    for l in range(len(H.levels) - 1):
        L = H.levels[l]
        A = csr_to_scipy(L.A, (L.n, L.n))
        K = (csr_to_scipy(L.R, (L.nc, L.n)) @ A @ csr_to_scipy(L.P, (L.n, L.nc))).toarray()
        Ko = csr_to_scipy(H.levels[l + 1].A, (L.nc, L.nc)).toarray()
        np.testing.assert_allclose(Ko, K, rtol=0, atol=1e-13 * np.abs(K).max())


def test_lumping_keeps_row_sums_and_large_entries():
    s = W.config("fd2d_64", scale=40)
    H0 = O.Hierarchy(s, distance=2, lump_tol=0.0, max_levels=2, coarse_max=10)
    H1 = O.Hierarchy(s, distance=2, lump_tol=0.05, max_levels=2, coarse_max=10)
    K0 = csr_to_scipy(H0.levels[1].A, (H0.levels[1].n,) * 2).toarray()
    K1 = csr_to_scipy(H1.levels[1].A, (H1.levels[1].n,) * 2).toarray()
    np.testing.assert_allclose(K1.sum(1), K0.sum(1), rtol=1e-14, atol=1e-14 * np.abs(K0).max())
    thr = 0.05 * np.abs(K0).max(1)
    n = K0.shape[0]
    off = ~np.eye(n, dtype=bool)
    big = (np.abs(K0) >= thr[:, None]) & off
    assert np.array_equal(K1[big], K0[big])
    assert not ((np.abs(K0) < thr[:, None]) & off & (K1 != 0)).any()
    assert len(H1.levels[1].A[1]) < len(H0.levels[1].A[1])


# --------------------------------------------------------------------------------------
# two-grid spectrum (Sec. 2.4, Eq. (2.9)) and exactness
# --------------------------------------------------------------------------------------

def _precond_matrix(H, n):
    return np.stack([H.precond(np.eye(n)[:, j]) for j in range(n)], 1)


def test_two_grid_eigenvalues_equal_eig_G():
    s = W.config("fd2d_64", scale=10)
    n = s.n
    H = O.Hierarchy(s, relax=O.RELAX_FF, cf_mode=O.CF_RS, coarse_max=n - 1, max_levels=2, lump_tol=0.0)
    L = H.levels[0]
    A = s.to_scipy().toarray()
    E = np.eye(n) - _precond_matrix(H, n) @ A
    Fi, Ci = np.nonzero(L.cf == 0)[0], np.nonzero(L.cf == 1)[0]
    R = csr_to_scipy(L.R, (len(Ci), n)).toarray()
    P = csr_to_scipy(L.P, (n, len(Ci))).toarray()
    Z, Wm = R[:, Fi], P[Fi, :]
    Aff, Afc, Acf = A[np.ix_(Fi, Fi)], A[np.ix_(Fi, Ci)], A[np.ix_(Ci, Fi)]
    K = R @ A @ P
    Dinv = np.diag(1 / np.diag(Aff))
    T = np.eye(len(Fi)) - Dinv @ Aff
    Delta = (np.eye(len(Fi)) - T @ T) @ np.linalg.inv(Aff)       # two Jacobi F-sweeps
    G = (np.eye(len(Fi)) - Delta @ Aff) + Delta @ (Aff @ Wm + Afc) @ np.linalg.inv(K) @ (Z @ Aff + Acf)
    eG = np.sort_complex(np.linalg.eigvals(G))
    eE = np.linalg.eigvals(E)
    # E has n_c zero eigenvalues (range of P) plus the eigenvalues of G
    eE = eE[np.argsort(np.abs(eE))][len(Ci):]
    eE = np.sort_complex(eE)
    for lam in eG:
        assert np.min(np.abs(eE - lam)) <= 1e-8 * max(1.0, abs(lam))


def test_exact_F_solve_with_ideal_R_converges_in_one_cycle():
    """Sec. 2.4: exact F-solve and ideal restriction give rho(E_TG) = 0 (triangular chain:
    A_ff diagonal, so one Jacobi F-sweep is exact and distance-one lAIR is ideal)."""
    s = W.upwind_chain(33, a=-0.7)
    H = O.Hierarchy(s, cf_mode=O.CF_RS, relax=O.RELAX_FF, coarse_max=17, max_levels=2, lump_tol=0.0)
    assert len(H.levels) == 2
    A = s.to_scipy().toarray()
    x = H.precond(s.b)
    np.testing.assert_allclose(x, np.linalg.solve(A, s.b), rtol=1e-13, atol=1e-13)


def test_vcycle_factor_matches_spectral_radius():
    """Measured asymptotic V-cycle factor (power iteration on the error) vs rho(E) of the
    dense error propagator; the average factor of the stationary solve is below rho + 0.05."""
    s = W.config("fd2d_64", scale=24)
    n = s.n
    H = O.Hierarchy(s, cf_mode=O.CF_RS)
    A = s.to_scipy().toarray()
    E = np.eye(n) - _precond_matrix(H, n) @ A
    rho = np.abs(np.linalg.eigvals(E)).max()
    e = np.random.default_rng(0).standard_normal(n)
    ratios = []
    for k in range(300):
        e2 = E @ e
        ratios.append(np.linalg.norm(e2) / np.linalg.norm(e))
        e = e2 / np.linalg.norm(e2)
    measured = math.exp(np.mean(np.log(ratios[-50:])))
    assert abs(measured - rho) <= 0.02 * rho + 1e-3
    x, rep = H.solve(s.b, tol=1e-10, cycle=0)
    assert rep["status"] == 0
    cf = (rep["rel"] / rep["hist"][0]) ** (1.0 / rep["iters"])
    assert cf <= rho + 0.05


# --------------------------------------------------------------------------------------
# outer loops: solution, FGMRES minimal residual (Sec. 4: V-cycles precondition GMRES)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("cycle", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_solution_matches_sparse_direct(cycle, prec):
    s = W.config("fd2d_64")
    H = O.Hierarchy(s, prec=prec)
    x, rep = H.solve(s.b, tol=1e-10, cycle=cycle)
    assert rep["status"] == 0 and rep["rel"] <= 1e-10
    ref = spla.spsolve(s.to_scipy().tocsc(), s.b)
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)


def test_fgmres_minimal_residual_property():
    """With a fixed preconditioner M, FGMRES iterate k minimises ||b - A x|| over
    x0 + span{M v_0 ... } = x0 + M K_k(A M, r0)."""
    s = W.config("fd2d_64", scale=16)
    n = s.n
    H = O.Hierarchy(s, cf_mode=O.CF_PMIS, distance=1)
    A = s.to_scipy().toarray()
    Minv = _precond_matrix(H, n)
    AM = A @ Minv
    r0 = s.b.copy()
    for k in (1, 2, 3, 4):
        x, rep = H.solve(s.b, tol=0.0, cycle=1, max_iter=k, restart=30)
        Kb = [r0]
        for _ in range(k - 1):
            Kb.append(AM @ Kb[-1])
        Q, _ = np.linalg.qr(np.stack(Kb, 1))
        y, *_ = np.linalg.lstsq(AM @ Q, r0, rcond=None)
        best = np.linalg.norm(r0 - AM @ Q @ y)
        got = np.linalg.norm(s.b - A @ x)
        assert got == pytest.approx(best, rel=1e-6, abs=1e-14)


# --------------------------------------------------------------------------------------
# DG block-diagonal scaling (Sec. 4.2.1) and the DG generator
# --------------------------------------------------------------------------------------

def test_block_scale_matches_dense():
    s = W.dg_p2_advection(3)
    st, (rp, col, val), dinv = O.block_scale(s, 6)
    assert st == 0
    A = s.to_scipy().toarray()
    Db = sla.block_diag(*[A[6 * k:6 * k + 6, 6 * k:6 * k + 6] for k in range(s.n // 6)])
    ref = np.linalg.solve(Db, A)
    got = sp.csr_matrix((val, col.astype(np.int64), rp), shape=A.shape).toarray()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    for k in range(s.n // 6):
        assert np.array_equal(got[6 * k:6 * k + 6, 6 * k:6 * k + 6], np.eye(6))


def test_triangle_rule_exactness():
    pts, w = W.triangle_rule(5)
    for p in range(9):
        for q in range(9 - p):
            exact = math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2)
            assert np.dot(w, pts[:, 0] ** p * pts[:, 1] ** q) == pytest.approx(exact, rel=1e-13)


def test_dg_generator_consistency():
    s = W.dg_p2_advection(4)
    A = s.to_scipy()
    # divergence-free velocity with no boundary inflow: S 1 = 0 up to quadrature error, so
    # A 1 = Mass 1 and the entries of Mass 1 sum to the domain area
    assert (A @ np.ones(s.n)).sum() == pytest.approx(1.0, rel=1e-12)
    # the neighbour blocks couple only elements sharing an edge
    assert s.n == 6 * 2 * 16


def test_batched_splitting_is_per_system():
    """Batched systems (block diagonal): the splitting of every system equals the one it gets alone."""
    systems = W.batched_fd(count=5, side_lo=8, side_hi=20)
    A, offs = W.block_diagonal(systems)
    for mode in (O.CF_RS, O.CF_AUTO):
        H = O.Hierarchy(A, seg=offs, cf_mode=mode, rs_block=150, max_levels=2, coarse_max=4)
        cf = H.levels[0].cf
        for k, s in enumerate(systems):
            seg_cf = cf[offs[k]:offs[k + 1]]
            if mode == O.CF_RS:
                alone = O.cf_split(s, O.strength(s, 0.25), O.CF_RS)
            else:
                alone = O.cf_split(s, O.strength(s, 0.25), O.CF_AUTO, seed=150)
            assert np.array_equal(seg_cf, alone)
        # coarse offsets count the C points of the systems before
        c = np.concatenate([[0], np.cumsum([int((cf[offs[k]:offs[k + 1]] == 1).sum()) for k in range(len(systems))])])
        assert np.array_equal(H.seg(1), c)


# --------------------------------------------------------------------------------------
# batched outer loops (independent systems in one block-diagonal hierarchy)
# --------------------------------------------------------------------------------------

def _batch(count=4, lo=8, hi=14, seed=3):
    systems = W.batched_fd(count=count, side_lo=lo, side_hi=hi, seed=seed)
    A, offs = W.block_diagonal(systems)
    return systems, A, offs


def _system_precond(H, n, a, b):
    """Dense matrix of the preconditioner restricted to the rows/columns [a, b) of one system;
    also checks that the block-diagonal hierarchy leaves every other system untouched."""
    cols = []
    for j in range(a, b):
        e = np.zeros(n)
        e[j] = 1.0
        z = H.precond(e)
        assert not np.any(z[:a]) and not np.any(z[b:])
        cols.append(z[a:b])
    return np.stack(cols, 1)


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_stationary_is_per_system_refinement(prec):
    """Stationary refinement on a batch: each system follows x <- x + M_q^{-1} (b_q - A_q x) on its own
    and stops once its own relative residual is <= tol; the result solves each system (sparse LU)."""
    systems, A, offs = _batch()
    H = O.Hierarchy(A, seg=offs, prec=prec)
    tol = 1e-10
    x, rep = H.solve_batched(A.b, tol=tol, cycle=0)
    assert rep["status"] == 0
    for q, s in enumerate(systems):
        a, b = offs[q], offs[q + 1]
        Aq = s.to_scipy().toarray()
        Mq = _system_precond(H, A.n, a, b)
        xr = np.zeros(s.n)
        k = 0
        while np.linalg.norm(s.b - Aq @ xr) / np.linalg.norm(s.b) > tol:
            xr = xr + Mq @ (s.b - Aq @ xr)
            k += 1
            assert k <= 500
        assert rep["iters"][q] == k
        np.testing.assert_allclose(x[a:b], xr, rtol=0, atol=1e-9 * np.abs(xr).max())
        ref = spla.spsolve(s.to_scipy().tocsc(), s.b)
        assert np.linalg.norm(x[a:b] - ref) <= 1e-7 * np.linalg.norm(ref)
        relq = np.linalg.norm(s.b - Aq @ x[a:b]) / np.linalg.norm(s.b)
        assert relq <= tol and rep["rel"][q] == pytest.approx(relq, rel=1e-6)


def test_batched_fgmres_minimal_residual_per_system():
    """FGMRES on a batch with a fixed preconditioner: iterate k of system q minimises
    ||b_q - A_q x|| over M_q K_k(A_q M_q, b_q) (zero initial guess), whatever the other systems do."""
    systems, A, offs = _batch(count=3, seed=4)
    H = O.Hierarchy(A, seg=offs, cf_mode=O.CF_PMIS)
    mats = [(s.to_scipy().toarray(), _system_precond(H, A.n, offs[q], offs[q + 1])) for q, s in enumerate(systems)]
    for k in (1, 2, 3):
        x, rep = H.solve_batched(A.b, tol=0.0, cycle=1, max_iter=k)
        for q, s in enumerate(systems):
            Aq, Mq = mats[q]
            AM = Aq @ Mq
            Kb = [s.b]
            for _ in range(k - 1):
                Kb.append(AM @ Kb[-1])
            Q, _ = np.linalg.qr(np.stack(Kb, 1))
            y, *_ = np.linalg.lstsq(AM @ Q, s.b, rcond=None)
            best = np.linalg.norm(s.b - AM @ Q @ y)
            got = np.linalg.norm(s.b - Aq @ x[offs[q]:offs[q + 1]])
            assert rep["iters"][q] == k
            assert got == pytest.approx(best, rel=1e-6, abs=1e-14)
    x, rep = H.solve_batched(A.b, tol=1e-10, cycle=1)
    assert rep["status"] == 0
    for q, s in enumerate(systems):
        ref = spla.spsolve(s.to_scipy().tocsc(), s.b)
        assert np.linalg.norm(x[offs[q]:offs[q + 1]] - ref) <= 1e-7 * np.linalg.norm(ref)


# --------------------------------------------------------------------------------------
# the FP32 cycle of mixed precision (FP32 cycle inside the FP64 outer loop), restated in numpy float32
# --------------------------------------------------------------------------------------

def _f32_two_level_cycle(A, cf, R, P, K, b, seq):
    """One V-cycle (post-relaxation, zero initial guess) of a two-level hierarchy in float32:
    b rounded to float; b_c = R b; the coarse system solved in FP64 and rounded to float;
    x = P x_c; then the Jacobi sweeps of seq (all updates of a sweep read the same old x)."""
    f = np.float32
    A32, R32, P32 = (M.astype(f).toarray() for M in (A, R, P))
    dinv = (1.0 / A.diagonal()).astype(f)
    b32 = b.astype(f)
    bc = R32 @ b32
    xc = np.linalg.solve(K.toarray(), bc.astype(np.float64)).astype(f)
    x = P32 @ xc
    for tgt in seq:
        r = b32 - A32 @ x
        x = np.where(cf == tgt, x + dinv * r, x).astype(f)
    assert x.dtype == f
    return x


@pytest.mark.parametrize("relax,seq", [(O.RELAX_FFC, (0, 0, 1)), (O.RELAX_FCF, (0, 1, 0)), (O.RELAX_FF, (0, 0))])
def test_fp32_cycle_matches_numpy_float32(relax, seq):
    """Mixed precision: the oracle's FP32 two-level cycle against the same cycle in numpy float32,
    entry by entry (a wrong sweep order moves entries by about 5e-4 of the largest here). The cut
    between precisions: R holds FP32 values and the cycle returns FP32 values, which the FP64 cycle
    does not."""
    s = W.config("fd2d_64", scale=13)                     # n = 169
    kw = dict(cf_mode=O.CF_RS, max_levels=2, coarse_max=s.n - 1, relax=relax, lump_tol=0.0)
    H32 = O.Hierarchy(s, prec=1, **kw)
    H64 = O.Hierarchy(s, prec=0, **kw)
    assert len(H32.levels) == 2
    L0, L1 = H32.levels
    n, nc = L0.n, L0.nc
    A = csr_to_scipy(L0.A, (n, n))
    R = csr_to_scipy(L0.R, (nc, n))
    P = csr_to_scipy(L0.P, (n, nc))
    K = csr_to_scipy(L1.A, (nc, nc))
    assert np.array_equal(R.data.astype(np.float32).astype(np.float64), R.data)   # FP32 local solves
    rng = np.random.default_rng(11)
    for _ in range(3):
        v = rng.uniform(-1, 1, n)
        ref = _f32_two_level_cycle(A, L0.cf, R, P, K, v, seq).astype(np.float64)
        z = H32.precond(v)
        scale = np.abs(ref).max()
        assert np.abs(z - ref).max() <= 1e-6 * scale
        assert np.array_equal(z.astype(np.float32).astype(np.float64), z)
        z64 = H64.precond(v)
        assert not np.array_equal(z64.astype(np.float32).astype(np.float64), z64)
        assert np.abs(z64 - ref).max() <= 1e-5 * scale


# --------------------------------------------------------------------------------------
# host threads: the oracle's independent loops give the same bits for any thread count
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,scale,kw", [
    ("fd3d_192", 14, dict(distance=1, prec=1)),
    ("dg_p2_256", 6, dict(distance=2, interp=1, strength_abs=1, block_size=6, cf_mode=O.CF_PMIS)),
    ("fd2d_64", 30, dict(distance=2, cf_mode=O.CF_AUTO, rs_block=100)),
])
def test_oracle_thread_count_does_not_change_results(name, scale, kw):
    s = W.config(name, scale=scale)
    before = O.threads()
    out = []
    try:
        for t in (1, 4):
            O.set_threads(t)
            H = O.Hierarchy(s, **kw)
            x, rep = H.solve(s.b, tol=1e-10, cycle=1)
            out.append((H, x, rep["iters"]))
    finally:
        O.set_threads(before)
    (H1, x1, i1), (H4, x4, i4) = out
    assert i1 == i4 and np.array_equal(x1, x4)
    for L1, L4 in zip(H1.levels, H4.levels):
        for a, b in ((L1.A, L4.A), (L1.R, L4.R), (L1.P, L4.P)):
            if a is not None:
                assert all(np.array_equal(u, v) for u, v in zip(a, b))
