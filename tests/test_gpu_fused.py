"""The small levels of the V-cycle in one cooperative launch (the fused
small-level cycle) against the oracle, and against the launch-per-step
cycle (AMG_FUSED_COARSE=0): one V-cycle element by element, PCG iteration
counts, and fewer launches per cycle when the fused path runs."""
import numpy as np
import pytest

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


@pytest.fixture(scope="module")
def case():
    P = inputs.anisotropic(256, nrhs=1)
    return P, O.setup(P.A, P.aggs, P.n_nodes, P.W)


def _cycle(amg, P, R, prec, fused, monkeypatch):
    if fused:
        monkeypatch.delenv("AMG_FUSED_COARSE", raising=False)
    else:
        monkeypatch.setenv("AMG_FUSED_COARSE", "0")
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    o = amg.opts(cycle_precision=prec)
    H.vcycle(R, o)                       # workspace
    l0 = amg.kernel_launches()
    Z = H.vcycle(R, o)
    launches = amg.kernel_launches() - l0
    x, info, st = H.solve(P.B[:, :1], options=amg.opts(cycle_precision=prec, maxit=2000))
    H.close()
    return Z, launches, info[0]["iters"], st


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 2e-5)])
@pytest.mark.parametrize("ncol", [1, 5, 32])
def test_fused_small_levels_match_oracle(amg, case, monkeypatch, prec, tol, ncol):
    P, Ho = case
    R = np.random.default_rng(ncol).standard_normal((P.n, ncol))
    Zo = O.vcycle(Ho, R)
    Zf, nf, itf, stf = _cycle(amg, P, R, prec, True, monkeypatch)
    Zu, nu, itu, stu = _cycle(amg, P, R, prec, False, monkeypatch)
    for Z in (Zf, Zu):
        assert np.linalg.norm(Z - Zo) / np.linalg.norm(Zo) <= tol
    assert stf == stu == amg.AMG_OK
    assert abs(itf - itu) <= (0 if prec == 64 else 1)
    assert nf < nu, (nf, nu)           # the fused path ran: fewer launches per cycle


def test_fused_batch_of_uneven_systems(amg, monkeypatch):
    """The batched plan (block-diagonal levels and coarsest inverse) through
    the fused cycle (forced, AMG_FUSED_COARSE=1): every column reaches the
    true residual."""
    monkeypatch.setenv("AMG_FUSED_COARSE", "1")   # the fused path, not the tuner's choice
    probs = [inputs.anisotropic(N, nrhs=1, levels=4, cfg=2) for N in (64, 96)]
    Hs = [amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W) for P in probs]
    Bs = [np.random.default_rng(s).uniform(-1, 1, (P.n, 3)) for s, P in enumerate(probs)]
    for prec in (64, 32):
        X, infos, st = amg.solve_batched(Hs, Bs, options=amg.opts(cycle_precision=prec, maxit=2000))
        assert st == amg.AMG_OK
        for P, B, Xs in zip(probs, Bs, X):
            rel = np.linalg.norm(B - P.A @ Xs, axis=0) / np.linalg.norm(B, axis=0)
            assert rel.max() <= 1.1e-8
    for h in Hs:
        h.close()
