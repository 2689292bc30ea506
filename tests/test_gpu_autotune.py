"""The launch-schedule autotuners change timing only. Cycle kernels: with and without tuning, the
preconditioner and the solve give the same bits (each row of a sliced-ELL view is one thread's). Local
solves: every system is solved by the same operations whichever team (thread, warp, CTA) takes it, so the
hierarchy is the same bits under the tuned schedule."""
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


@pytest.mark.parametrize("name,scale,kw", [
    ("fd3d_192", 64, dict(precision=1)),                                     # lAIP: R and P solves tuned
    ("fd3d_192", 64, dict(precision=0, interp=1, cf_mode=1)),
    ("dg_p2_256", 128, dict(distance=2, interp=1, strength_abs=1, block_size=6, precision=1, cf_mode=1)),
])
def test_local_solve_tuning_keeps_every_bit(lair, name, scale, kw):
    """Batches of at least 65,536 local systems are tuned over their launch schedules; R, P and every
    coarse operator come out the same bits as without tuning, and the choice is reported."""
    s = W.config(name, scale=scale)
    G0 = lair.Hierarchy.from_system(s, device=True, autotune=0, **kw)
    G1 = lair.Hierarchy.from_system(s, device=True, autotune=1, timing=1, **kw)
    info = G0.info()
    assert len(info) == len(G1.info())
    for l in range(len(info)):
        for which in (0, 1, 2) if not info[l]["coarsest"] else (0,):
            for a, b in zip(G0.export_csr(l, which), G1.export_csr(l, which)):
                assert np.array_equal(a, b), (l, which)
    assert any(k.startswith("tune_local_L") for k in G1.timers())
