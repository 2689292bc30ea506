"""The launch-schedule autotuner of the cycle kernels changes timing only: with and without it, the
preconditioner and the solve give the same bits (each row of a sliced-ELL view is one thread's)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lair():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair as L
    torch.cuda.init()
    return L


# levels of at least 65,536 rows are tuned: 2D FD 512^2 and DG-P2 on a 128^2 mesh have several
@pytest.mark.parametrize("name,scale,kw", [("adjoint_fd2d_512", None, dict(precision=1)),
                                           ("adjoint_fd2d_512", None, dict(precision=0)),
                                           ("dg_p2_256", 128, dict(distance=2, interp=1, strength_abs=1,
                                                                   block_size=6, precision=1))])
def test_autotune_does_not_change_results(lair, name, scale, kw):
    import torch
    s = W.config(name, scale=scale)
    G0 = lair.Hierarchy.from_system(s, device=True, autotune=0, **kw)
    G1 = lair.Hierarchy.from_system(s, device=True, autotune=1, **kw)
    v = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, s.n)).cuda()
    assert torch.equal(G0.precond(v), G1.precond(v))
    b = torch.from_numpy(s.b).cuda()
    x0, r0 = G0.solve(b, tol=1e-10)
    x1, r1 = G1.solve(b, tol=1e-10)
    assert r0.status == 0 and r0.iters == r1.iters and torch.equal(x0, x1)
