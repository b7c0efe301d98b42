"""The kernel timer (amg_timer_enable) only observes: with a kernel family
timed or not, a solve gives the same bits and the same iteration counts, and
the solve without the timer takes no longer, within noise, than with it.
The benchmark times its steps with the timer off and reads kernel times in
separate solves."""
import numpy as np
import pytest

from paper_1907_04417_gb300.hostsetup import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


def test_timer_changes_nothing_but_time(amg):
    import torch

    import bench
    P = inputs.anisotropic(256, nrhs=1)
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    B = bench.rhs_block(P, 32, 0)
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.zeros_like(Bd)
    o = amg.opts(cycle_precision=32, maxit=2000)

    def solve():
        Xd.zero_()
        _, inf, st = H.solve(Bd, Xd, o)
        assert st == amg.AMG_OK
        return Xd.clone(), [i["iters"] for i in inf]

    def timed(reps=5):
        out = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            solve()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.median(out))

    X0, it0 = solve()
    t_off = timed()
    for kid in (amg.KERNEL_SPMV_CG, amg.KERNEL_CG_UPDATE, amg.KERNEL_COARSE_LEVELS):
        H.timer_enable(kid)
        X1, it1 = solve()
        ms, n = H.timer_read()
        assert n > 0 and ms > 0, kid
        assert it1 == it0, kid
        assert torch.equal(X0, X1), kid
        H.timer_enable(0, False)
    H.timer_enable(amg.KERNEL_SPMV_CG)
    solve()
    t_on = timed()
    H.timer_enable(0, False)
    X2, it2 = solve()
    assert torch.equal(X0, X2) and it2 == it0
    assert t_off <= 1.10 * t_on + 1.0, (t_off, t_on)
    H.close()
