"""GPU parity of the bootstrap testing phase (Algorithm 1, Section 2).

amg_bootstrap_test applies the composite error operator of several
single-vector hierarchies (symmetrized as in Section 5 (i), or the plain
product of Eq. (comp_AMG)) nu times on the device.  It is checked against
the oracle's bootstrap_test on the same hierarchies and start vectors,
column by column, in float64 (1e-10) and with the float32 cycle (1e-5), and
the GPU driver of Algorithm 1 against the oracle's driver.  Bad arguments
are refused before any launch.
"""
import numpy as np
import pytest

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import aggregation, problems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import torch  # noqa: F401
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


def _stages(N, seeds=(21,)):
    """Single-vector hierarchies on aniso9(N): w = 1 (two pairwise steps per
    level, three levels) and seeded random vectors (four steps per level)."""
    A = problems.aniso9(N)
    n = A.shape[0]
    ws = [(np.ones(n), [2, 2])] + [(np.random.default_rng(s).standard_normal(n), [2, 2, 2]) for s in seeds]
    out = []
    for w, steps in ws:
        aggs, nn = aggregation.aggregate_hierarchy(A, w, steps)
        out.append((aggs, nn, (w / np.linalg.norm(w))[:, None]))
    return A, out


def _rel(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


@pytest.mark.parametrize("symmetric", [True, False])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_bootstrap_test_matches_oracle_fp64(amg, symmetric, nrhs):
    A, st = _stages(32, seeds=(21, 22))
    Hg = [amg.Hierarchy(A, a, nn, w) for a, nn, w in st]
    Ho = [O.setup(A, a, nn, w) for a, nn, w in st]
    x0 = np.random.default_rng(7).standard_normal((A.shape[0], nrhs))
    xg, rg, ng = amg.bootstrap_test(Hg, x0, 4, symmetric)
    xo, ro = O.bootstrap_test(Ho, A, x0, 4, symmetric)
    assert _rel(xg, xo).max() <= 1e-10
    np.testing.assert_allclose(rg, ro, rtol=1e-10)
    np.testing.assert_allclose(ng, O.a_norm(A, xo), rtol=1e-10)
    assert np.all(ro < 1.0)
    for h in Hg:
        h.close()


def test_bootstrap_test_fp32_cycle(amg):
    A, st = _stages(32)
    Hg = [amg.Hierarchy(A, a, nn, w) for a, nn, w in st]
    Ho = [O.setup(A, a, nn, w) for a, nn, w in st]
    x0 = np.random.default_rng(8).standard_normal((A.shape[0], 2))
    xg, rg, _ = amg.bootstrap_test(Hg, x0, 3, True, amg.opts(cycle_precision=32))
    xo, ro = O.bootstrap_test(Ho, A, x0, 3, True)
    assert _rel(xg, xo).max() <= 1e-5
    np.testing.assert_allclose(rg, ro, rtol=1e-5)


def test_bootstrap_driver_matches_oracle(amg):
    """Algorithm 1 with m = 3 at 64^2: the first stage (B_1 from w_0 = 1) is
    compared element by element; the second stage matches on w_1, so it is
    compared where both sides chose the same aggregates."""
    from paper_1907_04417_gb300 import bootstrap as B
    A = problems.aniso9(64)
    n = A.shape[0]
    agg = lambda w: aggregation.aggregate_hierarchy(A, w, [4, 4])
    starts = [np.random.default_rng(40 + r).standard_normal(n) for r in range(2)]
    Wg, rg, Hs = B.bootstrap(A, np.ones(n), 3, 15, agg, starts)
    Wo, ro = O.bootstrap(A, np.ones(n), 3, 15, agg, starts)
    assert _rel(Wg[:, 1:2], Wo[:, 1:2]).max() <= 1e-10
    assert rg[0] == pytest.approx(ro[0], rel=1e-10)
    a_g, a_o = agg(Wg[:, 1]), agg(Wo[:, 1])
    if all(np.array_equal(x, y) for x, y in zip(a_g[0], a_o[0])):
        assert _rel(Wg[:, 2:3], Wo[:, 2:3]).max() <= 1e-8
        assert rg[1] == pytest.approx(ro[1], rel=1e-8)
    assert 0.0 < rg[1] < 1.0
    for h in Hs:
        h.close()


def test_bootstrap_test_rejects_mismatched_hierarchies(amg):
    A1, st1 = _stages(16, seeds=())
    A2, st2 = _stages(20, seeds=())
    H1 = amg.Hierarchy(A1, *st1[0])
    H2 = amg.Hierarchy(A2, *st2[0])
    with pytest.raises(amg.AMGError) as e:
        amg.bootstrap_test([H1, H2], np.ones(A1.shape[0]), 1)
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    with pytest.raises(amg.AMGError):
        amg.bootstrap_test([H1], np.ones(A1.shape[0]), 0)
    H1.close()
    H2.close()


def test_bootstrap_workload_iterations_match_oracle(amg):
    """The benchmark's smooth vectors at 256^2: the device bootstrap on the
    seeded starts, then the float64 PCG, against the iteration count of the
    oracle's own bootstrap and solve (stored in tests/golden)."""
    import json
    import os
    from paper_1907_04417_gb300 import bootstrap as B
    from paper_1907_04417_gb300.hostsetup import inputs
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_iterations.json")))
    P = inputs.anisotropic(256, nrhs=1)
    W, rhos, Hs = B.bootstrap(P.A, np.ones(P.n), P.m, 15, inputs.stage_aggregator(P.A, [4] * (P.levels - 1)),
                              inputs.bootstrap_starts(P.n, P.m))
    for h in Hs:
        h.close()
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, W / np.linalg.norm(W, axis=0))
    x, info, st = H.solve(P.B[:, 0], options=amg.opts(maxit=5000))
    assert st == amg.AMG_OK
    g = gold["aniso9_256x256_bootstrap"]
    assert abs(info[0]["iters"] - g["iters"]) <= 1, (info[0]["iters"], g["iters"])
    assert H.info()["n_level"] == g["levels"]
    tr = np.linalg.norm(P.B[:, 0] - P.A @ x) / np.linalg.norm(P.B[:, 0])
    assert tr <= 1.1e-8
