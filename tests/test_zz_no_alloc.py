"""The allocation-free local-solve entry point, against the restriction rows lair_setup builds.

lair_local_solve_noalloc serves callers that cannot allocate device memory where they need a
solve (inside CUDA graph capture or replay, under an exhausted memory budget, on threads that
must stay off the allocator); its working storage is a fixed device array inside the library.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def local_systems(s, R, cf):
    """Dense systems of Eq. (3.2) for every C point, from A and the column pattern of R."""
    A = s.to_scipy().tocsr()
    Cpts = np.nonzero(cf == 1)[0]
    out = []
    for c, i in enumerate(Cpts):
        cols = R[1][R[0][c]:R[0][c + 1]]
        nb = cols[cols != i]
        sub = A[nb][:, nb].toarray()
        M = sub.T.copy()                                   # M[r][c] = a_{l_c, l_r}
        rhs = -A[i, nb].toarray().ravel()
        out.append((c, nb, M, rhs))
    return out


def noalloc_solve(lair, Ms, rhss):
    """One call of the allocation-free entry point on device copies of the given systems."""
    import torch
    nsys, size = len(Ms), len(rhss[0])
    M = torch.from_numpy(np.stack(Ms)).cuda().contiguous()
    b = torch.from_numpy(np.stack(rhss)).cuda().contiguous()
    z = torch.full((nsys, size), np.nan, dtype=torch.float64, device="cuda")
    flags = torch.full((nsys,), 7, dtype=torch.uint8, device="cuda")
    st = lair.lib.lair_local_solve_noalloc(nsys, int(size), M.data_ptr(), b.data_ptr(), z.data_ptr(),
                                           flags.data_ptr(), None)
    assert st == 0
    torch.cuda.synchronize()
    return z.cpu().numpy(), flags.cpu().numpy()


@pytest.mark.parametrize("band", ["cta", "warp_and_thread"])
def test_local_solve_noalloc_matches_setup_rows(band):
    """Two calls in a row, each with every system of one size, against the rows of R that lair_setup built
    through the existing entry point: the same routine, so the same bits. Sizes above 32 are solved by
    CTA teams in the set-up, sizes up to 32 by warp or thread teams there."""
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair

    s = W.random_sparse(2000, 8, seed=7)
    G = lair.Hierarchy.from_system(s, distance=2, max_levels=2, coarse_max=10)   # existing entry point
    R = G.export_csr(0, 1)
    cf, _, ls_R, _ = G.export_cf(0)
    systems = local_systems(s, R, cf)
    sizes = np.array([len(nb) for _, nb, _, _ in systems])
    lo, hi = (32, 64) if band == "cta" else (0, 32)
    picked = [v for v in np.unique(sizes) if lo < v <= hi]
    picked.sort(key=lambda v: -(sizes == v).sum())
    assert len(picked) >= 2
    for size in picked[:2]:
        group = [t for t in systems if len(t[1]) == size]
        zh, fh = noalloc_solve(lair, [t[2] for t in group], [t[3] for t in group])
        for k, (c, nb, _, _) in enumerate(group):
            row = slice(R[0][c], R[0][c + 1])
            cols, vals = R[1][row], R[2][row]
            ref = vals[np.isin(cols, nb)]
            assert np.array_equal(zh[k], ref), (size, c, np.abs(zh[k] - ref).max())
            assert fh[k] == ls_R[c]


def test_local_solve_noalloc_singular_systems_take_least_squares():
    """Systems with a duplicated column are singular: the flag is set and z is the minimum-norm
    least-squares solution (Sec. 3.1 footnote), compared with numpy's and with the oracle's."""
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair
    from oracle import oracle as O

    rng = np.random.default_rng(3)
    for size in (5, 40):
        Ms, rhss = [], []
        for _ in range(3):
            M = rng.uniform(-1, 1, (size, size)) + size * np.eye(size)
            M[:, size - 1] = M[:, 1]                         # a repeated column: rank size - 1
            Ms.append(M)
            rhss.append(rng.uniform(-1, 1, size))
        zh, fh = noalloc_solve(lair, Ms, rhss)
        for k in range(len(Ms)):
            assert fh[k] == 1
            ref = np.linalg.lstsq(Ms[k], rhss[k], rcond=None)[0]
            assert np.abs(zh[k] - ref).max() <= 1e-10 * np.abs(ref).max()
            zo, ls = O.local_solve(Ms[k], rhss[k])
            assert ls
            assert np.abs(zh[k] - zo).max() <= 1e-12 * np.abs(zo).max()


def test_local_solve_noalloc_rejects_oversized_and_bad_arguments():
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair
    assert lair.lib.lair_local_solve_noalloc(1, 65, None, None, None, None, None) == 1   # NULL pointers first
    dummy = ctypes.c_void_p(1)
    assert lair.lib.lair_local_solve_noalloc(1, 65, dummy, dummy, dummy, None, None) == 13   # UNSUPPORTED
    assert lair.lib.lair_local_solve_noalloc(1, 0, dummy, dummy, dummy, None, None) == 1
    assert lair.lib.lair_local_solve_noalloc(0, 8, None, None, None, None, None) == 0
