"""GPU parity with more than one l1-Jacobi sweep per side.

With one pre-sweep the float32 cycle folds the first pre-sweep from zero into
a column-scaled level-0 matrix (u0 = D^{-1} r is never stored); with more
pre-sweeps it stores u0 and smooths from it.  Both paths, and the float64
cycle, are checked against the oracle's V-cycle and PCG with the same sweep
counts: the V-cycle element by element, the float64 PCG iteration count
within one and its iterate at that count within 1e-10, the float32-cycle
batch by its true residual and at most three extra iterations.
"""
import numpy as np
import pytest

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import inputs

pytestmark = pytest.mark.gpu

SWEEPS = [(2, 2), (1, 2), (3, 1)]


@pytest.fixture(scope="module")
def amg():
    import torch  # noqa: F401
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


@pytest.fixture(scope="module")
def built(amg):
    out = {}
    for name, mk in {"aniso64": lambda: inputs.anisotropic(64, nrhs=1, levels=4),
                     "jump16": lambda: inputs.jumping3d(16, nrhs=1, max_coarse=256)}.items():
        P = mk()
        out[name] = (P, O.setup(P.A, P.aggs, P.n_nodes, P.W), amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W))
    return out


@pytest.mark.parametrize("name", ["aniso64", "jump16"])
@pytest.mark.parametrize("pre,post", SWEEPS)
@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 2e-5)])
def test_vcycle_sweeps(amg, built, name, pre, post, prec, tol):
    P, Ho, Hg = built[name]
    R = np.random.default_rng(pre * 10 + post).standard_normal((P.n, 3))
    Zg = Hg.vcycle(R, amg.opts(cycle_precision=prec, pre=pre, post=post))
    Zo = O.vcycle(Ho, R, pre=pre, post=post)
    assert np.linalg.norm(Zg - Zo) / np.linalg.norm(Zo) <= tol


@pytest.mark.parametrize("name", ["aniso64", "jump16"])
@pytest.mark.parametrize("pre,post", SWEEPS)
def test_pcg_sweeps(amg, built, name, pre, post):
    P, Ho, Hg = built[name]
    B = np.random.default_rng(pre + 7 * post).uniform(-1.0, 1.0, (P.n, 8))
    X64, i64, st64 = Hg.solve(B, options=amg.opts(pre=pre, post=post))
    X32, i32, st32 = Hg.solve(B, options=amg.opts(cycle_precision=32, pre=pre, post=post))
    assert st64 == amg.AMG_OK and st32 == amg.AMG_OK
    prec = lambda r: O.vcycle(Ho, r, pre=pre, post=post)
    for c in (0, 5):
        ro = O.pcg(P.A, B[:, c], prec)
        assert abs(i64[c]["iters"] - ro.iters) <= 1, (i64[c]["iters"], ro.iters)
        rf = O.pcg(P.A, B[:, c], prec, fixed_iters=i64[c]["iters"])
        assert np.linalg.norm(X64[:, c] - rf.x) / np.linalg.norm(rf.x) <= 1e-10
    tr = np.linalg.norm(B - P.A @ X32, axis=0) / np.linalg.norm(B, axis=0)
    assert tr.max() <= 1.1e-8, tr.max()
    for c in range(8):
        assert i32[c]["iters"] <= i64[c]["iters"] + 3
