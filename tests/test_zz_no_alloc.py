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


def test_local_solve_noalloc_matches_setup_rows():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair

    s = W.random_sparse(2000, 8, seed=7)
    G = lair.Hierarchy.from_system(s, distance=2, max_levels=2, coarse_max=10)   # existing entry point
    R = G.export_csr(0, 1)
    cf, _, ls_R, _ = G.export_cf(0)
    systems = local_systems(s, R, cf)
    sizes = np.array([len(nb) for _, nb, _, _ in systems])
    # two calls in a row, with the two most frequent sizes above 32 (the CTA-team range)
    big = [v for v in np.unique(sizes) if 32 < v <= 64]
    big.sort(key=lambda v: -(sizes == v).sum())
    assert len(big) >= 2
    for size in big[:2]:
        group = [t for t in systems if len(t[1]) == size]
        M = torch.from_numpy(np.stack([t[2] for t in group])).cuda().contiguous()
        b = torch.from_numpy(np.stack([t[3] for t in group])).cuda().contiguous()
        z = torch.full((len(group), size), np.nan, dtype=torch.float64, device="cuda")
        flags = torch.full((len(group),), 7, dtype=torch.uint8, device="cuda")
        st = lair.lib.lair_local_solve_noalloc(len(group), int(size), M.data_ptr(), b.data_ptr(), z.data_ptr(),
                                               flags.data_ptr(), None)
        assert st == 0
        torch.cuda.synchronize()
        zh = z.cpu().numpy()
        fh = flags.cpu().numpy()
        for k, (c, nb, _, _) in enumerate(group):
            row = slice(R[0][c], R[0][c + 1])
            cols, vals = R[1][row], R[2][row]
            ref = vals[np.isin(cols, nb)]
            scale = np.abs(ref).max()
            assert np.abs(zh[k] - ref).max() <= 1e-12 * scale, (size, c)
            assert fh[k] == ls_R[c]


def test_local_solve_noalloc_rejects_oversized_and_bad_arguments():
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair
    assert lair.lib.lair_local_solve_noalloc(1, 65, None, None, None, None, None) == 1   # NULL pointers first
    dummy = ctypes.c_void_p(1)
    assert lair.lib.lair_local_solve_noalloc(1, 65, dummy, dummy, dummy, None, None) == 13   # UNSUPPORTED
    assert lair.lib.lair_local_solve_noalloc(1, 0, dummy, dummy, dummy, None, None) == 1
    assert lair.lib.lair_local_solve_noalloc(0, 8, None, None, None, None, None) == 0
