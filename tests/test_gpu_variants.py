"""GPU parity of the cycle variants (Section 5): multicolour forward/backward
Gauss-Seidel smoothing and the K-cycle with two inner flexible-CG
iterations, in float64.

* the colouring of every smoothed level, bit-exact against the oracle's
  greedy colouring (and at the full 1024^2 anisotropic size on level 0);
* one cycle, element by element, for GS/V, l1-Jacobi/K and GS/K with
  several sweep counts, on several tiles and a ragged column count;
* PCG: iteration counts within one of the oracle's, true residuals, and the
  iterate after a fixed number of iterations;
* padded columns (nrhs not a power of two) and an all-zero column;
* the options the variants reject.
"""
import numpy as np
import pytest

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import inputs

pytestmark = pytest.mark.gpu

VARIANTS = [("gs", "V"), ("l1jacobi", "K"), ("gs", "K")]
SM = {"l1jacobi": 0, "gs": 1}
CY = {"V": 0, "K": 1}


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
                     "poisson48": lambda: inputs.poisson(48, nrhs=1),
                     "jump16": lambda: inputs.jumping3d(16, nrhs=1, max_coarse=256)}.items():
        P = mk()
        out[name] = (P, O.setup(P.A, P.aggs, P.n_nodes, P.W), amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W))
    return out


def _opts(amg, sm, kind, **kw):
    return amg.opts(smoother=SM[sm], cycle=CY[kind], **kw)


def _true_relres(A, B, X):
    B = B.reshape(B.shape[0], -1)
    X = X.reshape(B.shape)
    return np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)


@pytest.mark.parametrize("name", ["aniso64", "poisson48", "jump16"])
def test_colours_bit_exact(amg, built, name):
    P, Ho, Hg = built[name]
    for k in range(Ho.L - 1):
        cg, nc = Hg.level_colours(k)
        co = O.greedy_colouring(Ho.levels[k].A)
        np.testing.assert_array_equal(cg, co)
        assert nc == co.max() + 1


@pytest.mark.parametrize("name", ["aniso64", "jump16"])
@pytest.mark.parametrize("sm,kind", VARIANTS)
@pytest.mark.parametrize("pre,post", [(1, 1), (2, 1), (1, 3)])
def test_cycle_parity(amg, built, name, sm, kind, pre, post):
    P, Ho, Hg = built[name]
    R = np.random.default_rng(3 * pre + post).standard_normal((P.n, 3))
    Zg = Hg.vcycle(R, _opts(amg, sm, kind, pre=pre, post=post))
    Zo = O.cycle(Ho, R, pre=pre, post=post, smoother=sm, kind=kind)
    err = np.linalg.norm(Zg - Zo, axis=0) / np.linalg.norm(Zo, axis=0)
    assert err.max() <= 1e-11, err


@pytest.mark.parametrize("name", ["aniso64", "poisson48", "jump16"])
@pytest.mark.parametrize("sm,kind", VARIANTS)
def test_pcg_parity(amg, built, name, sm, kind):
    P, Ho, Hg = built[name]
    b = P.B[:, 0].copy()
    x, info, st = Hg.solve(b, options=_opts(amg, sm, kind, maxit=3000))
    assert st == amg.AMG_OK and info[0]["converged"]
    _, res = O.solve_variant(Ho, b, maxit=3000, smoother=sm, kind=kind)
    assert abs(info[0]["iters"] - res[0].iters) <= 1, (info[0]["iters"], res[0].iters)
    assert _true_relres(P.A, b, x)[0] <= 1.1e-8
    k = min(8, res[0].iters)
    xk, infk, stk = Hg.solve(b, options=_opts(amg, sm, kind, maxit=k))
    assert infk[0]["iters"] == k
    xo, _ = O.solve_variant(Ho, b, fixed_iters=k, smoother=sm, kind=kind)
    assert np.linalg.norm(xk - xo) / np.linalg.norm(xo) <= 1e-9


@pytest.mark.parametrize("sm,kind", VARIANTS)
def test_padded_and_zero_columns(amg, built, sm, kind):
    """Five columns (padded to eight inside), one of them zero: every other
    column converges with the same count as when solved alone, the zero
    column stays zero, and one cycle matches the oracle column by column."""
    P, Ho, Hg = built["aniso64"]
    B = np.random.default_rng(21).uniform(-1.0, 1.0, (P.n, 5))
    B[:, 3] = 0.0
    Z = Hg.vcycle(B, _opts(amg, sm, kind))
    Zo = O.cycle(Ho, B, smoother=sm, kind=kind)
    assert np.all(Z[:, 3] == 0.0)
    for c in (0, 1, 2, 4):
        assert np.linalg.norm(Z[:, c] - Zo[:, c]) <= 1e-11 * np.linalg.norm(Zo[:, c])
    X, infos, st = Hg.solve(B, options=_opts(amg, sm, kind))
    assert st == amg.AMG_OK
    assert np.all(X[:, 3] == 0.0)
    for c in (0, 2):
        _, i1, _ = Hg.solve(B[:, c].copy(), options=_opts(amg, sm, kind))
        assert abs(infos[c]["iters"] - i1[0]["iters"]) <= 1
    assert _true_relres(P.A, B[:, [0, 1, 2, 4]], X[:, [0, 1, 2, 4]]).max() <= 1.1e-8


def test_variants_rejected_where_unsupported(amg, built):
    P, Ho, Hg = built["poisson48"]
    b = P.B[:, 0].copy()
    for kw in ({"smoother": 1, "cycle_precision": 32}, {"cycle": 1, "cycle_precision": 32},
               {"smoother": 2}, {"cycle": -1}):
        with pytest.raises(amg.AMGError) as ei:
            Hg.solve(b, options=amg.opts(**kw))
        assert ei.value.status == amg.AMG_ERR_INVALID_ARG
    H2 = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    with pytest.raises(amg.AMGError):
        amg.solve_batched([Hg, H2], [P.B, P.B], options=amg.opts(smoother=1))
    with pytest.raises(amg.AMGError):
        Hg.level_colours(Ho.L - 1)


def test_full_size_colouring_and_solve(amg):
    """1024^2 anisotropic workload: level-0 colours bit-exact, GS/K PCG
    converges to the true residual in far fewer iterations than the
    l1-Jacobi V-cycle."""
    P = inputs.anisotropic(1024, nrhs=1)
    Hg = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    cg, nc = Hg.level_colours(0)
    co = O.greedy_colouring(P.A)
    np.testing.assert_array_equal(cg, co)
    b = P.B[:, 0].copy()
    x, info, st = Hg.solve(b, options=amg.opts(smoother=1, cycle=1, maxit=3000))
    assert st == amg.AMG_OK
    assert _true_relres(P.A, b, x)[0] <= 1.1e-8
    _, iv, _ = Hg.solve(b, options=amg.opts(maxit=3000))
    assert info[0]["iters"] < iv[0]["iters"] / 2, (info[0]["iters"], iv[0]["iters"])
