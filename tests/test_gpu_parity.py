"""GPU path (through the C ABI) against the CPU oracle, element by element.

Integer structure (strength masks, C/F splittings, least-squares flags, patterns of
R, P and every coarse operator) must be identical; FP64 values within 1e-12 and FP32
(mixed precision) values within 1e-5 of the row's largest entry. The set-up follows
the same operation order on both sides, so in practice the values agree bit for bit.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import oracle as O
from tests.helpers import compare_hierarchies, entrywise_rel, max_rel

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


def oracle_kw(kw):
    m = dict(cf_mode="cf_mode", distance="distance", theta="theta", theta_cf="theta_cf", strength_abs="strength_abs",
             interp="interp", relax="relax", lump_tol="lump_tol", coarse_max="coarse_max", max_levels="max_levels",
             block_size="block_size", rs_block="rs_block", precision="prec")
    return {m[k]: v for k, v in kw.items()}


CASES = {
    "fd2d64_rs_d1": ("fd2d_64", None, dict(cf_mode=0, distance=1)),
    "fd2d64_rs_d2": ("fd2d_64", None, dict(cf_mode=0, distance=2)),
    "fd2d64_pmis_d1": ("fd2d_64", None, dict(cf_mode=1, distance=1)),
    "fd2d64_auto_onepoint": ("fd2d_64", None, dict(distance=2, interp=1, rs_block=1000)),
    "fd2d64_mixed": ("fd2d_64", None, dict(cf_mode=0, distance=2, precision=1)),
    "fd2d_diffusive_d2": ("diffusive", None, dict(distance=2)),
    "fd3d_20_d1": ("fd3d_192", 20, dict(distance=1)),
    "fd3d_20_mixed": ("fd3d_192", 20, dict(distance=1, precision=1)),
    "dg_p2_16": ("dg_p2_256", 16, dict(distance=2, interp=1, strength_abs=1, block_size=6, precision=1)),
    "dg_p2_16_fp64_laip": ("dg_p2_256", 16, dict(distance=2, interp=0, strength_abs=1, block_size=6)),
    "random_theta_cf": ("random", None, dict(distance=2, theta=0.1, theta_cf=0.3, lump_tol=0.01)),
    "fd2d512_auto_blocks": ("adjoint_fd2d_512", None, dict(distance=1)),
    "fd3d_40_auto_blocks": ("fd3d_192", 40, dict(distance=1, rs_block=2048)),
    # one-point P with dense coarse operators: some R A rows exceed the fused triple-product kernels
    "fd3d_16_onepoint_d2_nolump": ("fd3d_192", 16, dict(distance=2, interp=1, lump_tol=0.0)),
    "diffusive_onepoint_d2": ("diffusive", None, dict(distance=2, interp=1, lump_tol=0.0)),
    # neighbourhoods beyond distance two (Sec. 4, pure advection)
    "fd2d64_d3": ("fd2d_64", None, dict(distance=3)),
    "fd2d64_pmis_d4_mixed": ("fd2d_64", None, dict(distance=4, cf_mode=1, precision=1)),
    "dg_p2_12_d3": ("dg_p2_256", 12, dict(distance=3, interp=1, strength_abs=1, block_size=6, cf_mode=1)),
}


def make(name, scale):
    if name == "diffusive":
        return W.fd_adr_2d(40, 1.1, 0.5, 0.3)
    if name == "random":
        return W.random_sparse(1500, 6, seed=5)
    return W.config(name, scale=scale)


@pytest.mark.parametrize("case", sorted(CASES))
def test_hierarchy_matches_oracle(lair, case):
    name, scale, kw = CASES[case]
    s = make(name, scale)
    G = lair.Hierarchy.from_system(s, device=True, **kw)
    H = O.Hierarchy(s, **oracle_kw(kw))
    assert H.status == 0
    tol = TOL32 if kw.get("precision") == 1 else TOL64
    worst = compare_hierarchies(G, H, tol)
    assert max(worst.values()) <= tol


@pytest.mark.parametrize("M", [24, 32, 40])
def test_vcycle_dg_sizes_match_oracle(lair, M):
    """The cycle on several DG meshes (coarsest levels of different sizes, interpolation rows
    without entries): finite and equal to the oracle's."""
    import torch
    s = W.config("dg_p2_256", scale=M)
    kw = dict(distance=2, interp=1, strength_abs=1, block_size=6, cf_mode=1, precision=1)
    G = lair.Hierarchy.from_system(s, device=True, **kw)
    H = O.Hierarchy(s, **oracle_kw(kw))
    v = np.random.default_rng(M).uniform(-1, 1, s.n)
    z = G.precond(torch.from_numpy(v).cuda()).cpu().numpy()
    zo = H.precond(v)
    assert np.isfinite(z).all()
    assert entrywise_rel(z, zo) <= TOL32


@pytest.mark.parametrize("case", ["fd2d64_rs_d1", "fd2d64_mixed", "fd3d_20_d1", "dg_p2_16", "fd2d_diffusive_d2"])
def test_vcycle_matches_oracle(lair, case):
    import torch
    name, scale, kw = CASES[case]
    s = make(name, scale)
    G = lair.Hierarchy.from_system(s, device=True, **kw)
    H = O.Hierarchy(s, **oracle_kw(kw))
    rng = np.random.default_rng(7)
    for _ in range(2):
        v = rng.uniform(-1, 1, s.n)      # with block scaling the cycle acts on the scaled system on both sides
        z = G.precond(torch.from_numpy(v).cuda()).cpu().numpy()
        zo = H.precond(v)
        tol = TOL32 if kw.get("precision") == 1 else TOL64
        assert entrywise_rel(z, zo) <= tol, entrywise_rel(z, zo)


@pytest.mark.parametrize("cycle", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_fd2d_64(lair, cycle, precision):
    import torch
    s = W.config("fd2d_64")
    G = lair.Hierarchy.from_system(s, device=True, cf_mode=0, precision=precision)
    H = O.Hierarchy(s, cf_mode=O.CF_RS, prec=precision)
    b = torch.from_numpy(s.b).cuda()
    x, rep = G.solve(b, tol=1e-10, cycle=cycle)
    xo, ro = H.solve(s.b, tol=1e-10, cycle=cycle)
    assert rep.status == 0 and rep.final_rel <= 1e-10
    A = s.to_scipy()
    xg = x.cpu().numpy()
    assert np.linalg.norm(s.b - A @ xg) / np.linalg.norm(s.b) <= 1.5e-10
    # same preconditioner, same iteration: counts agree and iterates are close
    assert abs(rep.iters - ro["iters"]) <= 1
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)


def test_host_and_device_buffers_agree(lair):
    import torch
    s = W.config("fd2d_64", scale=40)
    Gd = lair.Hierarchy.from_system(s, device=True)
    Gh = lair.Hierarchy.from_system(s, device=False)
    xd, rd = Gd.solve(torch.from_numpy(s.b).cuda(), tol=1e-10)
    xh, rh = Gh.solve(s.b.copy(), tol=1e-10)
    assert rd.iters == rh.iters
    np.testing.assert_array_equal(xd.cpu().numpy(), xh)


def test_single_level_direct_solve(lair):
    s = W.config("fd2d_64", scale=10)          # n = 100 <= coarse_max: the hierarchy is one dense level
    G = lair.Hierarchy.from_system(s)
    assert len(G.info()) == 1
    x, rep = G.solve(s.b.copy(), tol=1e-12, cycle=0)
    assert rep.iters == 1 and rep.final_rel <= 1e-12


def test_least_squares_branch_matches_oracle(lair):
    """A C point whose two F neighbours have proportional rows on the neighbourhood gives a
    singular local system (Sec. 3.1 footnote): minimum-norm least squares on both sides."""
    n = 9
    A = np.eye(n) * 4.0
    # C point 0 depends strongly on F points 1 and 2; rows 1 and 2 restricted to {1, 2} are equal
    A[0, 1] = A[0, 2] = -1.0
    A[1, 1], A[1, 2] = 2.0, 2.0
    A[2, 1], A[2, 2] = 2.0, 2.0
    A[1, 0], A[2, 0] = -0.5, -0.7          # rows differ outside the neighbourhood: A itself is nonsingular
    for i in range(3, n):
        A[i, i - 1] = -1.0
    M = sp.csr_matrix(A)
    M.sort_indices()
    s = W.CsrSystem(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.copy(), np.ones(n))
    cf = np.array([1, 0, 0, 1, 0, 1, 0, 1, 0], np.int8)
    kw = dict(distance=1, max_levels=2, coarse_max=2, lump_tol=0.0, theta=0.1, theta_cf=0.1)
    G = lair.Hierarchy.from_system(s, cf_user=cf, **kw)
    H = O.Hierarchy(s, cf_user=cf, **oracle_kw(kw))
    assert H.levels[0].ls_R[0] == 1
    compare_hierarchies(G, H, TOL64)


@pytest.mark.parametrize("bad,code", [("unsorted", 3), ("duplicate", 4), ("zero_diag", 5), ("bad_rowptr", 2)])
def test_invalid_input_reports_status(lair, bad, code):
    s = W.config("fd2d_64", scale=8)
    rp, col, val = s.row_ptr.copy(), s.col.copy(), s.val.copy()
    if bad == "unsorted":
        col[rp[5]], col[rp[5] + 1] = col[rp[5] + 1], col[rp[5]]
    elif bad == "duplicate":
        col[rp[5] + 1] = col[rp[5]]
    elif bad == "zero_diag":
        k = rp[5] + list(col[rp[5]:rp[6]]).index(5)
        val[k] = 0.0
    else:
        rp[-1] += 1
    with pytest.raises(lair.LairError) as e:
        lair.Hierarchy(rp, col, val)
    assert e.value.status == code


def test_not_converged_status(lair):
    s = W.config("fd2d_64")
    G = lair.Hierarchy.from_system(s)
    x, rep = G.solve(s.b.copy(), tol=1e-14, cycle=0, max_iter=2)
    assert rep.status == 7 and rep.iters == 2
    with pytest.raises(lair.LairError):
        G.solve(s.b.copy(), tol=1e-14, cycle=0, max_iter=2, raise_on_nc=True)


def test_adjoint_gradients(lair):
    """grad_b = A^{-T} g and grad_A = -lambda x^T on the pattern, against dense FP64 algebra and
    central finite differences of J(x) = 1/2 ||x - x*||^2."""
    import torch
    from paper_1708_06065_gb300 import autograd
    s = W.config("adjoint_fd2d_512", scale=32)
    xs = s.meta["x_star"]
    rp = torch.from_numpy(s.row_ptr).cuda()
    col = torch.from_numpy(s.col).cuda()
    vals = torch.from_numpy(s.val).cuda().requires_grad_(True)
    b = torch.from_numpy(s.b).cuda().requires_grad_(True)
    xstar = torch.from_numpy(xs).cuda()
    x = autograd.solve(rp, col, vals, b, tol=1e-12)
    J = 0.5 * ((x - xstar) ** 2).sum()
    J.backward()
    A = s.to_scipy().toarray()
    xd = np.linalg.solve(A, s.b)
    lam = np.linalg.solve(A.T, xd - xs)
    np.testing.assert_allclose(b.grad.cpu().numpy(), lam, rtol=0, atol=1e-8 * np.abs(lam).max())
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    gA = -lam[rows] * xd[s.col]
    np.testing.assert_allclose(vals.grad.cpu().numpy(), gA, rtol=0, atol=1e-8 * np.abs(gA).max())
    # central differences along random directions of b and of the nonzeros of A
    rng = np.random.default_rng(3)

    def Jf(v, bb):
        Ad = sp.csr_matrix((v, s.col, s.row_ptr), shape=(s.n, s.n)).toarray()
        xx = np.linalg.solve(Ad, bb)
        return 0.5 * np.sum((xx - xs) ** 2)

    for _ in range(4):
        db = rng.standard_normal(s.n)
        dv = rng.standard_normal(len(s.val)) * np.abs(s.val)
        h = 1e-6
        fd_b = (Jf(s.val, s.b + h * db) - Jf(s.val, s.b - h * db)) / (2 * h)
        fd_v = (Jf(s.val + h * dv, s.b) - Jf(s.val - h * dv, s.b)) / (2 * h)
        assert fd_b == pytest.approx(float(b.grad.cpu().numpy() @ db), rel=1e-5)
        assert fd_v == pytest.approx(float(vals.grad.cpu().numpy() @ dv), rel=1e-5)


def test_adjoint_gradients_full_size(lair):
    """The adjoint workload at full size (512 x 512 upwind FD, n = 262,144): grad_b and grad_A
    against an FP64 sparse LU of A, and central finite differences of J along 64 random
    directions of b and 64 random directions of the nonzeros of A."""
    import torch
    import scipy.sparse.linalg as spla
    from paper_1708_06065_gb300 import autograd
    s = W.config("adjoint_fd2d_512")
    assert s.n == 262144
    xs = s.meta["x_star"]
    rp = torch.from_numpy(s.row_ptr).cuda()
    col = torch.from_numpy(s.col).cuda()
    vals = torch.from_numpy(s.val).cuda().requires_grad_(True)
    b = torch.from_numpy(s.b).cuda().requires_grad_(True)
    x = autograd.solve(rp, col, vals, b, tol=1e-12)
    J = 0.5 * ((x - torch.from_numpy(xs).cuda()) ** 2).sum()
    J.backward()
    A = s.to_scipy().tocsc()
    lu = spla.splu(A)
    xd = lu.solve(s.b)
    lam = lu.solve(xd - xs, trans="T")
    gb = b.grad.cpu().numpy()
    gv = vals.grad.cpu().numpy()
    np.testing.assert_allclose(gb, lam, rtol=0, atol=1e-8 * np.abs(lam).max())
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    gA = -lam[rows] * xd[s.col]
    np.testing.assert_allclose(gv, gA, rtol=0, atol=1e-8 * np.abs(gA).max())
    rng = np.random.default_rng(64)
    # J is quadratic in b, so a central difference in b is exact for any step (h_b = 1 keeps the
    # cancellation small); in the nonzeros of A, h_v = 1e-5 balances truncation against rounding
    h_b, h_v = 1.0, 1e-5

    def Jb(bb):
        return 0.5 * np.sum((lu.solve(bb) - xs) ** 2)

    for _ in range(64):
        db = rng.standard_normal(s.n)
        fd = (Jb(s.b + h_b * db) - Jb(s.b - h_b * db)) / (2 * h_b)
        assert fd == pytest.approx(float(gb @ db), rel=1e-5)

    def Jv(v):
        # (A + h dA) x = b by refinement on the LU of A: the perturbation is O(h), so a few steps
        # reach rounding level
        Ad = sp.csr_matrix((v, s.col, s.row_ptr), shape=(s.n, s.n))
        xx = xd.copy()
        for _ in range(6):
            xx += lu.solve(s.b - Ad @ xx)
        assert np.linalg.norm(s.b - Ad @ xx) <= 1e-13 * np.linalg.norm(s.b)
        return 0.5 * np.sum((xx - xs) ** 2)

    for _ in range(64):
        dv = rng.standard_normal(len(s.val)) * np.abs(s.val)
        fd = (Jv(s.val + h_v * dv) - Jv(s.val - h_v * dv)) / (2 * h_v)
        assert fd == pytest.approx(float(gv @ dv), rel=1e-5)


def test_adjoint_hierarchy_matches_oracle_on_transpose(lair):
    s = W.config("fd2d_64", scale=40)
    G = lair.Hierarchy.from_system(s)
    g = np.random.default_rng(2).uniform(-1, 1, s.n)
    lam, rep = G.adjoint(g, tol=1e-10)
    trp, tcol, tval = O.transpose(s)
    st = W.CsrSystem(s.n, trp, tcol, tval, g)
    H = O.Hierarchy(st)
    lo, ro = H.solve(g, tol=1e-10)
    assert rep.status == 0 and abs(rep.iters - ro["iters"]) <= 1
    assert np.linalg.norm(lam - lo) <= 1e-8 * np.linalg.norm(lo)


def _diag_system(n, rng):
    return W.CsrSystem(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), rng.uniform(1, 2, n),
                       rng.uniform(-1, 1, n))


def _dense_system(n, rng):
    A = rng.uniform(-1, 1, (n, n)) + n * np.eye(n)
    return W.CsrSystem(n, np.arange(0, n * n + 1, n, dtype=np.int64), np.tile(np.arange(n, dtype=np.int32), n),
                       A.ravel(), rng.uniform(-1, 1, n))


@pytest.mark.parametrize("kind", ["diagonal_1000", "n_1", "dense_3", "dense_200"])
def test_degenerate_systems(lair, kind):
    """Degenerate inputs: no strong connection at all (every point F, no coarse level: the whole
    matrix goes to the dense solve), a single unknown, and dense systems small enough that the
    finest level is the coarsest or nearly so. Hierarchy as the oracle's, solution as a dense solve."""
    rng = np.random.default_rng(7)
    s = {"diagonal_1000": lambda: _diag_system(1000, rng), "n_1": lambda: _diag_system(1, rng),
         "dense_3": lambda: _dense_system(3, rng), "dense_200": lambda: _dense_system(200, rng)}[kind]()
    G = lair.Hierarchy.from_system(s)
    H = O.Hierarchy(s)
    assert H.status == 0
    assert len(G.info()) == len(H.levels)
    worst = compare_hierarchies(G, H, TOL64)
    assert max(worst.values(), default=0.0) <= TOL64
    x, rep = G.solve(s.b, tol=1e-12)
    xr = np.linalg.solve(s.to_scipy().toarray(), s.b)
    assert rep.status == 0
    assert np.abs(x - xr).max() <= 1e-10 * max(1.0, np.abs(xr).max())


def test_pmis_grid_barrier_wait_gives_up(lair):
    """Every wait of the cooperative PMIS kernel is bounded. With a bound of one poll the first block at
    a grid barrier gives up, every block returns, lair_setup reports LAIR_ERR_DEVICE_TIMEOUT, and the
    context stays usable: the same set-up with the default bound then succeeds and solves."""
    s = W.config("fd2d_64", scale=128)          # 16,384 points: above the thread-block-cluster PMIS size
    with pytest.raises(lair.LairError) as e:
        lair.Hierarchy.from_system(s, device=True, cf_mode=1, wait_polls=1)
    assert e.value.status == 11
    G = lair.Hierarchy.from_system(s, device=True, cf_mode=1)
    H = O.Hierarchy(s, cf_mode=O.CF_PMIS)
    compare_hierarchies(G, H, TOL64)
    x, rep = G.solve(s.b.copy(), tol=1e-10)
    assert rep.status == 0
