"""GPU parity of the restriction by R = P^T (I - A D^{-1}).

With one pre-sweep of l1-Jacobi from zero the iterate that enters the
restriction of Section 5's V-cycle is u = D^{-1} f, so the restricted
residual P^T (f - A u) equals R f.  The library keeps R by aggregate (every
coarse dof of an aggregate has the same column pattern, the rows that the
aggregate's rows of A reach) and applies it as a grouped product that
gathers each of those rows once, either with a warp per aggregate or with a
slot of lanes per aggregate (patterns padded to multiples of 8 entries).
AMG_RESTRICT_RFORM=1 (warp) or =2 (slot) makes every transfer take it, =0
none.  These tests force each choice and check, against the FP64
oracle: one V-cycle element by element; PCG iteration counts within one and
the iterate at the GPU's count within 1e-10; the float32 cycle (both CG
forms) to the same true residual within three extra iterations; a batch of
uneven systems; and that more than one pre-sweep never takes R.
"""
import numpy as np
import pytest

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import inputs

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "aniso64": lambda: inputs.anisotropic(64, nrhs=1, levels=4),     # r = 4 per aggregate
    "jump16": lambda: inputs.jumping3d(16, nrhs=1, max_coarse=256),  # r <= 3
    "elast6": lambda: inputs.elasticity_grid(6, nrhs=1, levels=3),   # r <= 6 (8 values per entry)
    "cc32": lambda: inputs.diffusion_cc(32, nrhs=1, max_coarse=256),
}


@pytest.fixture(scope="module")
def amg():
    import torch  # noqa: F401
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


@pytest.fixture(scope="module")
def problems():
    out = {}
    for name, mk in PROBLEMS.items():
        P = mk()
        out[name] = (P, O.setup(P.A, P.aggs, P.n_nodes, P.W))
    return out


def _hier(amg, monkeypatch, P, force):
    monkeypatch.setenv("AMG_RESTRICT_RFORM", force)
    # every restriction in its own launch (the fused small-level cycle
    # restricts inside one cooperative kernel, without R)
    monkeypatch.setenv("AMG_FUSED_COARSE", "0")
    monkeypatch.delenv("AMG_TUNE_CACHE", raising=False)
    return amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)


def _by_r(H):
    L = H.info()["levels"]
    return [H.restriction_info(k) for k in range(L - 1)]


@pytest.mark.parametrize("form", ["1", "2"])
@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("k", [1, 8, 32])
def test_rform_vcycle_fp64_matches_oracle(amg, problems, monkeypatch, name, k, form):
    P, Ho = problems[name]
    R = np.random.default_rng(100 + k).uniform(-1.0, 1.0, (P.n, k))
    H = _hier(amg, monkeypatch, P, form)
    Z = H.vcycle(R if k > 1 else R[:, 0])
    info = _by_r(H)
    H.close()
    assert all(i["by_r"] for i in info), info
    assert all(i["entries"] > 0 and i["values_per_entry"] in (4, 8) for i in info), info
    Zo = O.vcycle(Ho, R if k > 1 else R[:, 0])
    Z = np.asarray(Z).reshape(Zo.shape)
    scale = np.abs(Zo).max()
    assert np.abs(Z - Zo).max() <= 1e-12 * scale, np.abs(Z - Zo).max() / scale


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_rform_off_takes_csr(amg, problems, monkeypatch, name):
    P, Ho = problems[name]
    R = np.random.default_rng(7).uniform(-1.0, 1.0, (P.n, 8))
    H = _hier(amg, monkeypatch, P, "0")
    Z = H.vcycle(R)
    info = _by_r(H)
    H.close()
    assert not any(i["by_r"] for i in info), info
    Zo = O.vcycle(Ho, R)
    assert np.abs(Z - Zo).max() <= 1e-12 * np.abs(Zo).max()


@pytest.mark.parametrize("form", ["1", "2"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_rform_pcg_fp64_matches_oracle(amg, problems, monkeypatch, name, form):
    P, Ho = problems[name]
    k = 8
    B = np.random.default_rng(11).uniform(-1.0, 1.0, (P.n, k))
    H = _hier(amg, monkeypatch, P, form)
    X, inf, st = H.solve(B)
    info = _by_r(H)
    H.close()
    assert st == amg.AMG_OK
    assert all(i["by_r"] for i in info), info
    for c in (0, 3, k - 1):
        _, res = O.solve(Ho, B[:, c])
        assert abs(inf[c]["iters"] - res[0].iters) <= 1, (c, inf[c]["iters"], res[0].iters)
        xf, _ = O.solve(Ho, B[:, c], fixed_iters=inf[c]["iters"])
        assert np.linalg.norm(X[:, c] - xf) / np.linalg.norm(xf) <= 1e-10


@pytest.mark.parametrize("form", ["1", "2"])
@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("outer", [0, 1])
def test_rform_fp32_cycle(amg, problems, monkeypatch, name, outer, form):
    P, Ho = problems[name]
    k = 32
    B = np.random.default_rng(5).uniform(-1.0, 1.0, (P.n, k))
    H = _hier(amg, monkeypatch, P, form)
    X64, i64, st64 = H.solve(B)
    X32, i32, st32 = H.solve(B, options=amg.opts(cycle_precision=32, outer_fp64=outer))
    info = _by_r(H)
    H.close()
    assert st64 == amg.AMG_OK and st32 == amg.AMG_OK
    assert all(i["by_r"] for i in info), info
    tr = np.linalg.norm(B - P.A @ X32, axis=0) / np.linalg.norm(B, axis=0)
    assert tr.max() <= 1.1e-8, tr.max()
    for c in range(k):
        assert i32[c]["iters"] <= i64[c]["iters"] + 3, (c, i32[c]["iters"], i64[c]["iters"])


@pytest.mark.parametrize("form", ["1", "2"])
def test_rform_uneven_batch(amg, monkeypatch, form):
    """Two elasticity grids of different sizes in one launch sequence: each
    system's float64 iterate matches the oracle at the GPU's count."""
    Ps = [inputs.elasticity_grid(n, nrhs=1, levels=3) for n in (5, 7)]
    monkeypatch.setenv("AMG_RESTRICT_RFORM", form)
    monkeypatch.setenv("AMG_FUSED_COARSE", "0")
    monkeypatch.delenv("AMG_TUNE_CACHE", raising=False)
    Hs = [amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W) for P in Ps]
    Bs = [np.random.default_rng(20 + s).uniform(-1.0, 1.0, (P.n, 4)) for s, P in enumerate(Ps)]
    Xs, infos, st = amg.solve_batched(Hs, Bs)
    for H in Hs:
        H.close()
    assert st == amg.AMG_OK
    for s, P in enumerate(Ps):
        Ho = O.setup(P.A, P.aggs, P.n_nodes, P.W)
        for c in (0, 3):
            it = infos[s][c]["iters"]
            _, res = O.solve(Ho, Bs[s][:, c])
            assert abs(it - res[0].iters) <= 1
            xf, _ = O.solve(Ho, Bs[s][:, c], fixed_iters=it)
            assert np.linalg.norm(np.asarray(Xs[s])[:, c] - xf) / np.linalg.norm(xf) <= 1e-10


def test_rform_needs_one_presweep(amg, problems, monkeypatch):
    P, Ho = problems["aniso64"]
    R = np.random.default_rng(3).uniform(-1.0, 1.0, (P.n, 8))
    H = _hier(amg, monkeypatch, P, "1")
    Z = H.vcycle(R, options=amg.opts(pre=2, post=2))
    info = _by_r(H)
    H.close()
    assert not any(i["by_r"] for i in info), info
    Zo = O.vcycle(Ho, R, pre=2, post=2)
    assert np.abs(Z - Zo).max() <= 1e-12 * np.abs(Zo).max()


def test_rform_with_fused_small_levels(amg, problems, monkeypatch):
    """With the fused small-level cycle forced on, the restrictions above its
    start level take R and the V-cycle still matches the oracle."""
    P, Ho = problems["aniso64"]
    R = np.random.default_rng(9).uniform(-1.0, 1.0, (P.n, 8))
    monkeypatch.setenv("AMG_RESTRICT_RFORM", "1")
    monkeypatch.setenv("AMG_FUSED_COARSE", "1")
    monkeypatch.delenv("AMG_TUNE_CACHE", raising=False)
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    Z = H.vcycle(R)
    info = _by_r(H)
    H.close()
    assert info[0]["by_r"], info
    Zo = O.vcycle(Ho, R)
    assert np.abs(Z - Zo).max() <= 1e-12 * np.abs(Zo).max()
