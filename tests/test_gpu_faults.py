"""Failure detection on the GPU without a fault: every device wait of the
library is bounded, and a wait that gives up turns into AMG_ERR_TIMEOUT on
the host while the context stays usable.

The test hook AMG_TEST_FIRST_WAIT=1 (read when a solve workspace is
created) limits the first wait for each staged shared-memory copy to one
non-blocking poll, which a copy issued a moment earlier cannot meet.  The
wait after it keeps its full bound, so no copy is left in flight; the solve
then finishes and reports the timeout.  A hierarchy made without the hook
afterwards solves normally in the same process.
"""
import numpy as np
import pytest

from paper_1907_04417_gb300.hostsetup import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


def test_staged_copy_wait_gives_up_with_timeout(amg, monkeypatch):
    import torch
    P = inputs.anisotropic(128, nrhs=1, levels=4)
    B = np.random.default_rng(3).uniform(-1, 1, (P.n, 32))
    Bd = torch.from_numpy(B).cuda()
    o = amg.opts(cycle_precision=32, maxit=500)
    monkeypatch.setenv("AMG_TEST_FIRST_WAIT", "1")
    monkeypatch.setenv("AMG_COARSE_KERNELS", "grouped")   # the grouped levels always stage
    monkeypatch.setenv("AMG_RESTRICT_RFORM", "0")         # ... and restrict through P^T
    monkeypatch.setenv("AMG_FUSED_COARSE", "0")           # ... when they run as kernels of their own
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    with pytest.raises(amg.AMGError) as e:
        H.solve(Bd, torch.zeros_like(Bd), o)
    assert e.value.status == amg.AMG_ERR_TIMEOUT
    assert "bounded wait" in amg.last_error()
    H.close()
    monkeypatch.delenv("AMG_TEST_FIRST_WAIT")
    monkeypatch.delenv("AMG_COARSE_KERNELS")
    monkeypatch.delenv("AMG_FUSED_COARSE")
    monkeypatch.delenv("AMG_RESTRICT_RFORM")
    H2 = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    X, infos, st = H2.solve(Bd, torch.zeros_like(Bd), o)
    assert st == amg.AMG_OK
    Xc = X.cpu().numpy()
    rel = np.linalg.norm(B - P.A @ Xc, axis=0) / np.linalg.norm(B, axis=0)
    assert rel.max() <= 1.1e-8
    H2.close()


def test_grid_barrier_gives_up_with_timeout(amg, monkeypatch):
    """AMG_TEST_BARRIER_HANG=1 makes the first grid barrier of the fused
    small-level cycle wait for one CTA more than the grid has: every CTA's
    bounded wait gives up (about a millisecond), the launch ends, and the
    solve reports AMG_ERR_TIMEOUT.  A hierarchy made afterwards without the
    hook solves normally."""
    import torch
    P = inputs.anisotropic(128, nrhs=1, levels=4)
    B = np.random.default_rng(4).uniform(-1, 1, (P.n, 8))
    Bd = torch.from_numpy(B).cuda()
    o = amg.opts(cycle_precision=64, maxit=20)
    monkeypatch.setenv("AMG_TEST_BARRIER_HANG", "1")
    monkeypatch.setenv("AMG_FUSED_COARSE", "1")
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    with pytest.raises(amg.AMGError) as e:
        H.solve(Bd, torch.zeros_like(Bd), o)
    assert e.value.status == amg.AMG_ERR_TIMEOUT
    assert "grid barrier" in amg.last_error()
    H.close()
    monkeypatch.delenv("AMG_TEST_BARRIER_HANG")
    H2 = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    X, infos, st = H2.solve(Bd, torch.zeros_like(Bd), amg.opts(cycle_precision=64, maxit=500))
    assert st == amg.AMG_OK
    rel = np.linalg.norm(B - P.A @ X.cpu().numpy(), axis=0) / np.linalg.norm(B, axis=0)
    assert rel.max() <= 1.1e-8
    H2.close()


def test_check_mode_passes_valid_plans(amg, monkeypatch):
    """AMG_CHECK=1: the device check of every index array passes on a real
    hierarchy and on a batch plan, and the solves are unchanged."""
    monkeypatch.setenv("AMG_CHECK", "1")
    probs = [inputs.anisotropic(N, nrhs=1, levels=4) for N in (48, 64)]
    Hs = [amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W) for P in probs]
    X, infos, st = amg.solve_batched(Hs, [P.B for P in probs], options=amg.opts(maxit=500))
    assert st == amg.AMG_OK
    for h in Hs:
        h.close()


def test_check_mode_refuses_a_corrupt_column_index(amg, monkeypatch):
    """A column index planted out of range in level 1 (test hook, after the
    level is built and before any kernel gathers through it) is found by the
    check, and setup is refused with the array, level and position named."""
    P = inputs.anisotropic(48, nrhs=1, levels=4)
    monkeypatch.setenv("AMG_CHECK", "1")
    monkeypatch.setenv("AMG_TEST_CORRUPT_COL", "1")
    with pytest.raises(amg.AMGError) as e:
        amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    msg = amg.last_error()
    assert "internal index check" in msg and "level 1" in msg and "col[0]" in msg, msg
    monkeypatch.delenv("AMG_TEST_CORRUPT_COL")
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)       # the same input without the hook
    x, info, st = H.solve(P.B[:, :1])
    assert st == amg.AMG_OK
    H.close()
