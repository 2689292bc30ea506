"""Seeded synthetic linear systems for the lAIR solver (inputs only).

This module holds no part of the solver's arithmetic: it writes down matrices
and right-hand sides, nothing else. Both the plain CPU oracle (``oracle/``) and
the GPU path draw their inputs from here, so the two sides always see the same
bits.

Families (the model equation of Sec. 4, Eq. (4.1): -div(k grad u) + b.grad u +
c u = f, in synthetic stand-ins for the paper's Dolfin discretisations):

* ``fd_adr``        first-order upwind finite differences, 2D 5-point or 3D
                    7-point, Dirichlet 0 eliminated, lexicographic order with x
                    fastest, mesh width h = 1/(N+1).
* ``dg_p2_advection`` upwind discontinuous Galerkin, nodal P2 on a structured
                    triangulated square, recirculating velocity, backward Euler
                    mass shift (the implicit time step of Sec. 4.1.1, Eq. (4.3)).
* ``batched_fd``    many independent ``fd_adr`` systems with drawn parameters.

Every matrix is CSR with int64 row pointers, int32 sorted column indices,
float64 values and an explicit diagonal.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CsrSystem", "fd_adr", "fd_adr_2d", "fd_adr_3d", "batched_fd", "block_diagonal", "dg_p2_advection",
    "config", "CONFIG_NAMES", "upwind_chain", "random_sparse", "triangle_rule",
]


@dataclass
class CsrSystem:
    """A sparse system A x = b in CSR form (inputs only)."""
    n: int
    row_ptr: np.ndarray          # int64 [n+1]
    col: np.ndarray              # int32 [nnz], ascending within each row
    val: np.ndarray              # float64 [nnz]
    b: np.ndarray                # float64 [n]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col.astype(np.int64), self.row_ptr), shape=(self.n, self.n))


def _csr_from_coo(n, rows, cols, vals):
    """Sum duplicates, sort columns, return (row_ptr, col, val)."""
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    vals = np.asarray(vals, np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = uniq // n
    c = uniq % n
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr, c.astype(np.int32), summed.astype(np.float64)


# --------------------------------------------------------------------------------------
# Upwind finite differences (2D 5-point, 3D 7-point)
# --------------------------------------------------------------------------------------

def fd_adr(N: int, dim: int, velocity, eps: float, c: float, *, b_seed=0, b=None) -> CsrSystem:
    """Upwind FD discretisation of -eps lap u + v.grad u + c u on (0,1)^dim.

    N interior points per side, h = 1/(N+1), Dirichlet 0 eliminated. Row i at grid
    point (ix, iy[, iz]) with i = ix + N*iy (+ N*N*iz). Diagonal 2*dim*eps/h^2 +
    sum_a |v_a|/h + c; every neighbour -eps/h^2, plus -|v_a|/h on the upstream
    neighbour along axis a (x-h when v_a > 0, x+h when v_a < 0).
    """
    v = np.asarray(velocity, np.float64)
    assert v.shape == (dim,)
    h = 1.0 / (N + 1)
    n = N ** dim
    d = eps / (h * h)
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for _ in range(dim):
        coords.append(rem % N)
        rem //= N
    diag = 2 * dim * d + np.abs(v).sum() / h + c
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, diag)]
    stride = 1
    for a in range(dim):
        ca = coords[a]
        for step in (-1, +1):
            ok = (ca + step >= 0) & (ca + step < N)
            coef = -d
            upstream = (v[a] > 0 and step == -1) or (v[a] < 0 and step == +1)
            if upstream:
                coef = -d - abs(v[a]) / h
            rows.append(idx[ok])
            cols.append(idx[ok] + step * stride)
            vals.append(np.full(int(ok.sum()), coef))
        stride *= N
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    row_ptr, col, val = _csr_from_coo(n, rows, cols, vals)
    if b is None:
        b = np.random.default_rng(b_seed).uniform(-1.0, 1.0, n)
    return CsrSystem(n, row_ptr, col, val, np.asarray(b, np.float64),
                     dict(kind="fd", N=N, dim=dim, velocity=v.tolist(), eps=eps, c=c))


def fd_adr_2d(N, angle, eps, c, **kw):
    return fd_adr(N, 2, (math.cos(angle), math.sin(angle)), eps, c, **kw)


def fd_adr_3d(N, velocity, eps, c, **kw):
    v = np.asarray(velocity, np.float64)
    return fd_adr(N, 3, v / np.linalg.norm(v), eps, c, **kw)


def batched_fd(count=512, side_lo=32, side_hi=256, seed=2):
    """Independent 2D upwind FD systems with drawn parameters.

    One generator ``default_rng(seed)``; per system, in this order: side in
    [side_lo, side_hi], angle ~ U(0, 2 pi), log10 eps ~ U(-6, 0), c ~ U(0, 1),
    then b ~ U(-1, 1)^n.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        side = int(rng.integers(side_lo, side_hi + 1))
        angle = float(rng.uniform(0.0, 2 * math.pi))
        eps = float(10.0 ** rng.uniform(-6.0, 0.0))
        cc = float(rng.uniform(0.0, 1.0))
        b = rng.uniform(-1.0, 1.0, side * side)
        s = fd_adr_2d(side, angle, eps, cc, b=b)
        s.meta.update(angle=angle)
        out.append(s)
    return out


def block_diagonal(systems):
    """Concatenate independent systems into one block-diagonal CSR; returns (CsrSystem, offsets)."""
    offs = np.zeros(len(systems) + 1, np.int64)
    for k, s_ in enumerate(systems):
        offs[k + 1] = offs[k] + s_.n
    nnzs = np.array([s_.nnz for s_ in systems], np.int64)
    noff = np.concatenate([[0], np.cumsum(nnzs)])
    n = int(offs[-1])
    row_ptr = np.zeros(n + 1, np.int64)
    col = np.empty(int(noff[-1]), np.int32)
    val = np.empty(int(noff[-1]))
    b = np.empty(n)
    for k, s_ in enumerate(systems):
        row_ptr[offs[k] + 1:offs[k + 1] + 1] = s_.row_ptr[1:] + noff[k]
        col[noff[k]:noff[k + 1]] = s_.col + offs[k]
        val[noff[k]:noff[k + 1]] = s_.val
        b[offs[k]:offs[k + 1]] = s_.b
    return CsrSystem(n, row_ptr, col, val, b, dict(kind="batch", nsys=len(systems))), offs


# --------------------------------------------------------------------------------------
# Small structured cases used by the tests
# --------------------------------------------------------------------------------------

def upwind_chain(n: int, a: float = -0.5) -> CsrSystem:
    """1D upwind chain: unit lower bidiagonal, a_{i,i-1} = a (a triangular A, Sec. 3.2)."""
    rows = np.concatenate([np.arange(n), np.arange(1, n)])
    cols = np.concatenate([np.arange(n), np.arange(n - 1)])
    vals = np.concatenate([np.ones(n), np.full(n - 1, a)])
    row_ptr, col, val = _csr_from_coo(n, rows, cols, vals)
    return CsrSystem(n, row_ptr, col, val, np.random.default_rng(0).uniform(-1, 1, n), dict(kind="chain"))


def random_sparse(n: int, per_row: int, seed: int, dominance: float = 1.5, sym_pattern=False) -> CsrSystem:
    """Random sparse matrix with negative off-diagonals and a dominant diagonal."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        js = rng.choice(n, size=min(per_row, n - 1) + 1, replace=False)
        js = js[js != i][:per_row]
        w = -rng.uniform(0.1, 1.0, len(js))
        rows += [i] * len(js)
        cols += js.tolist()
        vals += w.tolist()
        if sym_pattern:
            rows += js.tolist()
            cols += [i] * len(js)
            vals += (-rng.uniform(0.1, 1.0, len(js))).tolist()
    row_ptr, col, val = _csr_from_coo(n, rows, cols, vals)
    # diagonal = dominance * sum |offdiag| of the row
    offsum = np.zeros(n)
    for i in range(n):
        offsum[i] = np.abs(val[row_ptr[i]:row_ptr[i + 1]]).sum()
    r2 = np.concatenate([np.repeat(np.arange(n), np.diff(row_ptr)), np.arange(n)])
    c2 = np.concatenate([col.astype(np.int64), np.arange(n)])
    v2 = np.concatenate([val, dominance * offsum + 0.1])
    row_ptr, col, val = _csr_from_coo(n, r2, c2, v2)
    return CsrSystem(n, row_ptr, col, val, rng.uniform(-1, 1, n), dict(kind="random"))


# --------------------------------------------------------------------------------------
# Upwind DG, nodal P2, structured triangulation
# --------------------------------------------------------------------------------------

def triangle_rule(order: int):
    """Collapsed (Duffy) Gauss rule on the reference triangle {x>=0, y>=0, x+y<=1}.

    Tensor Gauss-Legendre with ``order`` points per direction mapped by
    (u, v) -> (u, v (1-u)); exact for polynomials of degree 2*order-2 (at least).
    Returns points [q, 2] and weights [q] summing to the area 1/2.
    """
    g, w = np.polynomial.legendre.leggauss(order)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    u, v = np.meshgrid(g, g, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    x = u.ravel()
    y = (v * (1.0 - u)).ravel()
    ww = (wu * wv * (1.0 - u)).ravel()
    return np.stack([x, y], 1), ww


def _p2_basis(xi, eta):
    """Nodal P2 basis on the reference triangle: vertices (0,0),(1,0),(0,1), then
    edge midpoints of edges (v0,v1), (v1,v2), (v2,v0). Returns phi [6, q], dphi [6, 2, q]."""
    l0 = 1.0 - xi - eta
    l1 = xi
    l2 = eta
    dl = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])   # d(l_k)/d(xi, eta)
    L = [l0, l1, l2]
    phi = [L[0] * (2 * L[0] - 1), L[1] * (2 * L[1] - 1), L[2] * (2 * L[2] - 1),
           4 * L[0] * L[1], 4 * L[1] * L[2], 4 * L[2] * L[0]]
    dphi = []
    for k in range(3):
        coef = 4 * L[k] - 1
        dphi.append(np.stack([coef * dl[k, 0], coef * dl[k, 1]]))
    for (p, q) in ((0, 1), (1, 2), (2, 0)):
        dphi.append(np.stack([4 * (L[p] * dl[q, 0] + L[q] * dl[p, 0]),
                              4 * (L[p] * dl[q, 1] + L[q] * dl[p, 1])]))
    return np.stack(phi), np.stack(dphi)


def _recirc_velocity(x, y):
    return -np.sin(np.pi * x) * np.cos(np.pi * y), np.cos(np.pi * x) * np.sin(np.pi * y)


def dg_p2_advection(M: int = 256, dt: float | None = None, *, b_seed=0, tri_order=5, edge_order=5) -> CsrSystem:
    """Upwind DG (nodal P2) for pure advection with recirculating velocity,
    as one backward-Euler step: A = Mass + dt * S_upwind (Eq. (4.3)).

    Mesh: M x M squares on the unit square, each cut along its lower-left to
    upper-right diagonal; elements row-major by square, lower triangle first.
    Lower triangle vertices (x0,y0),(x1,y0),(x1,y1); upper (x0,y0),(x1,y1),(x0,y1).
    6 DOFs per element, contiguous: 3 vertices then 3 edge midpoints.
    S_upwind(u, v) = sum_K int_K (beta.grad u) v - sum_K int_{dK} min(beta.n, 0) (u_K - u_ext) v,
    u_ext = 0 on the domain boundary (no inflow there: beta.n = 0). Element K couples
    to neighbour K' iff beta.n_K < 0 at some quadrature point of the shared edge.
    dt defaults to h = 1/M.
    """
    h = 1.0 / M
    if dt is None:
        dt = h
    nel = 2 * M * M
    n = 6 * nel
    qp, qw = triangle_rule(tri_order)
    phi, dphi = _p2_basis(qp[:, 0], qp[:, 1])           # [6,q], [6,2,q]
    eg, ew = np.polynomial.legendre.leggauss(edge_order)
    eg = 0.5 * (eg + 1.0)
    ew = 0.5 * ew

    sq = np.arange(M * M)
    sx = sq % M
    sy = sq // M
    x0 = sx * h
    y0 = sy * h
    # vertices per element [nel, 3, 2]
    V = np.zeros((nel, 3, 2))
    lo = 2 * sq
    up = 2 * sq + 1
    V[lo, 0] = np.stack([x0, y0], 1)
    V[lo, 1] = np.stack([x0 + h, y0], 1)
    V[lo, 2] = np.stack([x0 + h, y0 + h], 1)
    V[up, 0] = np.stack([x0, y0], 1)
    V[up, 1] = np.stack([x0 + h, y0 + h], 1)
    V[up, 2] = np.stack([x0, y0 + h], 1)

    J = np.stack([V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]], 2)   # [nel, 2(x,y), 2(xi,eta)]
    detJ = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    Jinv = np.empty_like(J)
    Jinv[:, 0, 0] = J[:, 1, 1] / detJ
    Jinv[:, 1, 1] = J[:, 0, 0] / detJ
    Jinv[:, 0, 1] = -J[:, 0, 1] / detJ
    Jinv[:, 1, 0] = -J[:, 1, 0] / detJ
    adet = np.abs(detJ)

    # physical quadrature points [nel, q, 2]
    X = V[:, None, 0, :] + np.einsum("eij,qj->eqi", J, qp)
    bx, by = _recirc_velocity(X[..., 0], X[..., 1])
    # physical gradients: grad_x phi = Jinv^T grad_ref phi  -> [nel, 6, 2, q]
    gphys = np.einsum("eji,kjq->ekiq", Jinv, dphi)
    bgrad = gphys[:, :, 0, :] * bx[:, None, :] + gphys[:, :, 1, :] * by[:, None, :]   # [nel, 6(j), q]
    # volume: Mass_ij = int phi_j phi_i; Adv_ij = int (beta.grad phi_j) phi_i
    mass = np.einsum("iq,jq,q->ij", phi, phi, qw)[None] * adet[:, None, None]
    adv = np.einsum("iq,ejq,q,e->eij", phi, bgrad, qw, adet)
    blocks_diag = mass + dt * adv

    rows, cols, vals = [], [], []
    el = np.arange(nel)

    # edges of element (local vertex pairs) and reference parametrisation
    ref_v = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    local_edges = ((0, 1), (1, 2), (2, 0))

    def neighbour(e_lo_up, sxv, syv, edge):
        """Neighbour element index across local edge, or -1 on the boundary."""
        nb = np.full(sxv.shape, -1, np.int64)
        if e_lo_up == 0:   # lower triangle: edges (v0,v1) bottom, (v1,v2) right, (v2,v0) diagonal
            if edge == 0:
                ok = syv > 0
                nb[ok] = 2 * ((syv[ok] - 1) * M + sxv[ok]) + 1          # upper tri of square below: its top edge
            elif edge == 1:
                ok = sxv < M - 1
                nb[ok] = 2 * (syv[ok] * M + sxv[ok] + 1) + 1            # upper tri of square to the right: its left edge
            else:
                nb[:] = 2 * (syv * M + sxv) + 1                          # upper tri of the same square
        else:              # upper triangle: edges (v0,v1) diagonal, (v1,v2) top, (v2,v0) left
            if edge == 0:
                nb[:] = 2 * (syv * M + sxv)
            elif edge == 1:
                ok = syv < M - 1
                nb[ok] = 2 * ((syv[ok] + 1) * M + sxv[ok])              # lower tri of square above: its bottom edge
            else:
                ok = sxv > 0
                nb[ok] = 2 * (syv[ok] * M + sxv[ok] - 1)                # lower tri of square to the left: its right edge
        return nb

    # face terms, one pass per (lower/upper, local edge)
    for lu in (0, 1):
        es = 2 * sq + lu
        for edge, (p, q) in enumerate(local_edges):
            # reference points along the edge
            rp = ref_v[p][None, :] * (1 - eg[:, None]) + ref_v[q][None, :] * eg[:, None]   # [g, 2]
            ph_e, _ = _p2_basis(rp[:, 0], rp[:, 1])                                      # [6, g]
            P0 = V[es, p]
            P1 = V[es, q]
            tvec = P1 - P0
            elen = np.linalg.norm(tvec, axis=1)
            # outward normal for a counter-clockwise triangle: (t_y, -t_x)/|t|
            nrm = np.stack([tvec[:, 1], -tvec[:, 0]], 1) / elen[:, None]
            Xe = P0[:, None, :] + tvec[:, None, :] * eg[None, :, None]                  # [E, g, 2]
            ex, ey = _recirc_velocity(Xe[..., 0], Xe[..., 1])
            bn = ex * nrm[:, None, 0] + ey * nrm[:, None, 1]                             # [E, g]
            inflow = np.minimum(bn, 0.0)                                                 # min(beta.n, 0)
            w = ew[None, :] * elen[:, None]                                               # [E, g]
            # diagonal contribution: - int min(b.n,0) u_K v
            Fd = -np.einsum("ig,jg,eg->eij", ph_e, ph_e, inflow * w)
            blocks_diag[es] += dt * Fd
            nb = neighbour(lu, sx, sy, edge)
            couple = (nb >= 0) & (bn < 0).any(axis=1)
            if not couple.any():
                continue
            # neighbour trace at the same physical points: map Xe into neighbour reference coords
            E = np.nonzero(couple)[0]
            nbE = nb[E]
            Jn = J[nbE]
            Jni = Jinv[nbE]
            ref_n = np.einsum("eij,egj->egi", Jni, Xe[E] - V[nbE, 0][:, None, :])       # [E', g, 2]
            ph_n, _ = _p2_basis(ref_n[..., 0].ravel(), ref_n[..., 1].ravel())
            ph_n = ph_n.reshape(6, len(E), len(eg))                                      # [6, E', g]
            # off-diagonal: + int min(b.n,0) u_ext v
            Fo = np.einsum("ieg,jeg,eg->eij", ph_e[:, None, :].repeat(len(E), 1), ph_n,
                           inflow[E] * w[E])
            blk = dt * Fo
            eK = es[E]
            r = (6 * eK)[:, None, None] + np.arange(6)[None, :, None]
            cc = (6 * nbE)[:, None, None] + np.arange(6)[None, None, :]
            rows.append(np.broadcast_to(r, blk.shape).ravel())
            cols.append(np.broadcast_to(cc, blk.shape).ravel())
            vals.append(blk.ravel())

    r = (6 * el)[:, None, None] + np.arange(6)[None, :, None]
    cc = (6 * el)[:, None, None] + np.arange(6)[None, None, :]
    rows.append(np.broadcast_to(r, blocks_diag.shape).ravel())
    cols.append(np.broadcast_to(cc, blocks_diag.shape).ravel())
    vals.append(blocks_diag.ravel())
    row_ptr, col, val = _csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    b = np.random.default_rng(b_seed).uniform(-1.0, 1.0, n)
    return CsrSystem(n, row_ptr, col, val, b, dict(kind="dg_p2", M=M, dt=dt, block_size=6))


# --------------------------------------------------------------------------------------
# Named workloads (sizes of the benchmark configurations, plus scaled-down variants)
# --------------------------------------------------------------------------------------

CONFIG_NAMES = ("fd2d_64", "dg_p2_256", "batched_512", "adjoint_fd2d_512", "fd3d_192")


def config(name: str, scale: int | None = None):
    """Build a named workload. ``scale`` overrides the grid side (for small test variants).

    fd2d_64          2D FD, N=64, angle 3pi/16, eps 1e-4, c 0.1, b ~ U(-1,1) seed 0
    dg_p2_256        DG-P2 recirculating advection, 256x256 squares, dt = h, b seed 0
    batched_512      512 systems, sides 32..256 (``scale`` = count)
    adjoint_fd2d_512 2D FD, N=512, C1's parameters; also x* ~ N(0,1) seed 1
    fd3d_192         3D FD, N=192, velocity (1,0.7,0.4)/|.|, eps 1e-5, c 0.05, b seed 0
    """
    if name == "fd2d_64":
        return fd_adr_2d(scale or 64, 3 * math.pi / 16, 1e-4, 0.1, b_seed=0)
    if name == "dg_p2_256":
        return dg_p2_advection(scale or 256, b_seed=0)
    if name == "batched_512":
        return batched_fd(count=scale or 512)
    if name == "adjoint_fd2d_512":
        s = fd_adr_2d(scale or 512, 3 * math.pi / 16, 1e-4, 0.1, b_seed=0)
        s.meta["x_star"] = np.random.default_rng(1).standard_normal(s.n)
        return s
    if name == "fd3d_192":
        return fd_adr_3d(scale or 192, (1.0, 0.7, 0.4), 1e-5, 0.05, b_seed=0)
    raise KeyError(name)


# Solver options of the benchmark workloads (shared by bench.py and the full-size parity tests).
# Keys are lair.Hierarchy keyword arguments; no arithmetic here.
BENCH_OPTIONS = {
    "dg_p2_256": dict(opts=dict(distance=2, interp=1, strength_abs=1, block_size=6, cf_mode=1), tol=1e-8,
                      cycle="fgmres"),
    # PMIS, one-point P, lumping 0.05: half the time of the blocked first pass with lAIP (measured)
    "batched_512": dict(opts=dict(distance=1, cf_mode=1, interp=1, lump_tol=0.05), tol=1e-8, cycle="fgmres",
                        batched=True),
    # PMIS and one-point P with lumping 0.05: the fastest set-up + solve measured for this system (the blocked
    # classical first pass, approximate ideal interpolation and smaller lumping thresholds are slower; 0.12 diverges)
    "fd3d_192": dict(opts=dict(distance=1, cf_mode=1, interp=1, lump_tol=0.05), tol=1e-8, cycle="stationary"),
    # the 64 x 64 system with the exact classical first pass, FP64 V-cycles to 1e-10
    "fd2d_64": dict(opts=dict(distance=1, cf_mode=0), tol=1e-10, cycle="stationary"),
    # forward solve, then the adjoint solve on A^T and the gradient with respect to A's nonzeros
    # (PMIS, one-point P and lumping 0.05 as for the 3D system: 30 ms per step against 98 ms with the blocked
    # first pass and lAIP, measured)
    "adjoint_fd2d_512": dict(opts=dict(distance=1, cf_mode=1, interp=1, lump_tol=0.05), tol=1e-8, cycle="fgmres",
                             adjoint=True),
}
