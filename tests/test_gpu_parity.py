"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Setup: prolongator blocks and coarse matrices element by element (up to the
column signs, which the preconditioner does not depend on).  Solve: one
V-cycle, PCG iteration counts within one and the iterate at the GPU's
iteration count within 1e-10 (FP64 path); the FP32-cycle path reaches the
same 1e-8 true residual within three extra iterations.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import aggregation, inputs, problems

from .gpu_helpers import compare_coarse_matrices, compare_prolongators

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import torch  # noqa: F401
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


def _problems():
    return {
        "poisson64": lambda: inputs.poisson(64),
        "aniso64": lambda: inputs.anisotropic(64, nrhs=2, levels=4),
        "jump16": lambda: inputs.jumping3d(16, nrhs=2, max_coarse=256),
        "elast6": lambda: inputs.elasticity_grid(6, nrhs=2, levels=3),
        "cc32": lambda: inputs.diffusion_cc(32, nrhs=2, max_coarse=256),
    }


CASES = list(_problems())


@pytest.fixture(scope="module")
def built(amg):
    out = {}
    for name, mk in _problems().items():
        P = mk()
        Ho = O.setup(P.A, P.aggs, P.n_nodes, P.W)
        Hg = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
        out[name] = (P, Ho, Hg)
    return out


@pytest.mark.parametrize("name", CASES)
def test_setup_matches_oracle(built, name):
    P, Ho, Hg = built[name]
    info = Hg.info()
    assert info["levels"] == Ho.L
    assert info["n_level"] == [l.A.shape[0] for l in Ho.levels]
    assert info["nnz_level"] == [l.A.nnz for l in Ho.levels]
    assert info["opc"] == pytest.approx(O.operator_complexity(Ho), rel=1e-12)
    worst, ex, sig, sgn = compare_prolongators(Hg, Ho, atol=1e-10)
    compare_coarse_matrices(Ho, ex, sig, sgn, rtol=1e-10)
    # orthonormal columns of every GPU block (Section 4)
    for k in range(1, Ho.L):
        e = ex[k]
        off = 0
        for t in range(e["naggs"]):
            na = e["row_start"][t + 1] - e["row_start"][t]
            r = e["r"][t]
            B = e["pval"][off:off + na * r].reshape(na, r)
            np.testing.assert_allclose(B.T @ B, np.eye(r), atol=1e-13)
            off += na * r


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", [64, 32])
def test_vcycle_matches_oracle(built, amg, name, prec):
    P, Ho, Hg = built[name]
    rng = np.random.default_rng(7)
    R = rng.standard_normal((P.n, 3))
    Zg = Hg.vcycle(R, amg.opts(cycle_precision=prec))
    Zo = O.vcycle(Ho, R)
    err = np.linalg.norm(Zg - Zo) / np.linalg.norm(Zo)
    assert err <= (1e-12 if prec == 64 else 2e-5), err


@pytest.mark.parametrize("name", CASES)
def test_pcg_fp64_matches_oracle(built, amg, name):
    P, Ho, Hg = built[name]
    b = P.B[:, 0].copy()
    x, info, st = Hg.solve(b)
    assert st == amg.AMG_OK and info[0]["converged"]
    _, res = O.solve(Ho, b)
    assert abs(info[0]["iters"] - res[0].iters) <= 1, (info[0]["iters"], res[0].iters)
    xf, _ = O.solve(Ho, b, fixed_iters=info[0]["iters"])
    err = np.linalg.norm(x - xf) / np.linalg.norm(xf)
    assert err <= 1e-10, err
    tr = np.linalg.norm(b - P.A @ x) / np.linalg.norm(b)
    assert tr <= 1.1e-8


@pytest.mark.parametrize("name", CASES)
def test_pcg_fp32_cycle(built, amg, name):
    P, Ho, Hg = built[name]
    b = P.B[:, 0].copy()
    _, i64, _ = Hg.solve(b)
    x, info, st = Hg.solve(b, options=amg.opts(cycle_precision=32))
    assert st == amg.AMG_OK
    assert info[0]["iters"] <= i64[0]["iters"] + 3, (info[0]["iters"], i64[0]["iters"])
    tr = np.linalg.norm(b - P.A @ x) / np.linalg.norm(b)
    assert tr <= 1.1e-8, tr
    xo, _ = O.solve(Ho, b)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-6


@pytest.mark.parametrize("k", [2, 3, 8, 32])
@pytest.mark.parametrize("prec", [64, 32])
def test_multi_rhs(built, amg, k, prec):
    P, Ho, Hg = built["aniso64"]
    B = np.random.default_rng(k).uniform(-1, 1, (P.n, k))
    X, info, st = Hg.solve(B, options=amg.opts(cycle_precision=prec))
    assert st == amg.AMG_OK
    for c in range(k):
        _, res = O.solve(Ho, B[:, c])
        if prec == 64:
            assert abs(info[c]["iters"] - res[0].iters) <= 1
            xf, _ = O.solve(Ho, B[:, c], fixed_iters=info[c]["iters"])
            assert np.linalg.norm(X[:, c] - xf) / np.linalg.norm(xf) <= 1e-10
        else:
            assert info[c]["iters"] <= res[0].iters + 3
        tr = np.linalg.norm(B[:, c] - P.A @ X[:, c]) / np.linalg.norm(B[:, c])
        assert tr <= 1.1e-8


def test_graph_and_eager_agree(built, amg):
    P, Ho, Hg = built["cc32"]
    b = P.B[:, 0].copy()
    xg, ig, _ = Hg.solve(b, options=amg.opts(use_graph=1, check_every=5))
    xe, ie, _ = Hg.solve(b, options=amg.opts(use_graph=0, check_every=3))
    assert ig[0]["iters"] == ie[0]["iters"]
    np.testing.assert_array_equal(xg, xe)  # same kernels, same order: bitwise


def test_deterministic_repeat(built, amg):
    P, Ho, Hg = built["jump16"]
    b = P.B[:, 0].copy()
    x1, _, _ = Hg.solve(b)
    x2, _, _ = Hg.solve(b)
    np.testing.assert_array_equal(x1, x2)


def test_device_and_host_pointers_agree(built, amg):
    import torch
    P, Ho, Hg = built["poisson64"]
    b = P.B[:, 0].copy()
    xh, _, _ = Hg.solve(b)
    xd, _, _ = Hg.solve(torch.from_numpy(b).cuda())
    np.testing.assert_array_equal(xh, xd.cpu().numpy())


def test_initial_guess(built, amg):
    P, Ho, Hg = built["cc32"]
    b = P.B[:, 0].copy()
    x0 = np.random.default_rng(3).standard_normal(P.n)
    x, info, st = Hg.solve(b, x=x0.copy())
    assert st == amg.AMG_OK
    r = O.pcg(P.A, b, lambda v: O.vcycle(Ho, v), x0=x0)
    assert abs(info[0]["iters"] - r.iters) <= 1
    tr = np.linalg.norm(b - P.A @ x) / np.linalg.norm(b)
    assert tr <= 1.1e-8


def test_batched_uneven_systems(amg):
    batch = inputs.elasticity_batch(n_sys=3, sides=(4, 5, 6), nrhs=3, levels=3)
    batch[1].B = batch[1].B[:, :2].copy()   # uneven column counts as well
    Hs = [amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W) for P in batch]
    for prec in (64, 32):
        X, infos, st = amg.solve_batched(Hs, [P.B for P in batch], options=amg.opts(cycle_precision=prec))
        assert st == amg.AMG_OK
        for P, Xs, inf in zip(batch, X, infos):
            Ho = O.setup(P.A, P.aggs, P.n_nodes, P.W)
            for c in range(P.B.shape[1]):
                _, res = O.solve(Ho, P.B[:, c])
                tr = np.linalg.norm(P.B[:, c] - P.A @ Xs[:, c]) / np.linalg.norm(P.B[:, c])
                assert tr <= 1.1e-8
                if prec == 64:
                    assert abs(inf[c]["iters"] - res[0].iters) <= 1
                    xf, _ = O.solve(Ho, P.B[:, c], fixed_iters=inf[c]["iters"])
                    assert np.linalg.norm(Xs[:, c] - xf) / np.linalg.norm(xf) <= 1e-10
                else:
                    assert inf[c]["iters"] <= res[0].iters + 3


def test_adjoint_matches_oracle(amg):
    P = inputs.diffusion_cc(16, nrhs=2, max_coarse=64)
    Ho = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    Hg = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    o = amg.opts(rtol=1e-13)
    X, _, _ = Hg.solve(P.B, options=o)
    g = 2 * (X - P.meta["x_target"])
    lam, grad, info, st = Hg.adjoint(g, X, options=o)
    assert st == amg.AMG_OK
    lo, go, _ = O.adjoint(Ho, g, X, rtol=1e-13)
    assert np.linalg.norm(lam - lo) / np.linalg.norm(lo) <= 1e-9
    assert np.linalg.norm(grad - go) / np.linalg.norm(go) <= 1e-9


# ---------------------------------------------------------------- edges --

def test_zero_rhs_and_padding(amg, built):
    P, Ho, Hg = built["poisson64"]
    B = np.zeros((P.n, 3))
    B[:, 1] = P.B[:, 0]
    X, info, st = Hg.solve(B)
    assert st == amg.AMG_OK
    assert info[0]["iters"] == 0 and info[2]["iters"] == 0
    assert np.all(X[:, 0] == 0) and np.all(X[:, 2] == 0)
    assert info[1]["converged"]


def test_maxit_not_converged_writes_x(amg, built):
    P, Ho, Hg = built["aniso64"]
    b = P.B[:, 0].copy()
    x, info, st = Hg.solve(b, options=amg.opts(maxit=3))
    assert st == amg.AMG_ERR_NOT_CONVERGED
    assert info[0]["iters"] == 3 and not info[0]["converged"]
    xf, _ = O.solve(Ho, b, fixed_iters=3)
    assert np.linalg.norm(x - xf) / np.linalg.norm(xf) <= 1e-10


def test_nan_rhs_breakdown(amg, built):
    P, Ho, Hg = built["poisson64"]
    b = P.B[:, 0].copy()
    b[5] = np.nan
    x, info, st = Hg.solve(b)
    assert st == amg.AMG_ERR_BREAKDOWN


def test_one_level_direct(amg):
    A = problems.poisson5(10)
    W = np.ones((100, 1)) / 10
    Hg = amg.Hierarchy(A, [], [100], W)
    b = np.random.default_rng(0).uniform(-1, 1, 100)
    x, info, st = Hg.solve(b)
    assert st == amg.AMG_OK and info[0]["iters"] == 1
    np.testing.assert_allclose(A @ x, b, atol=1e-12)


def test_singletons_small_aggregates_and_truncation(amg):
    """Random aggregates with sizes 1..5 and m = 4 (n_a < m for many), and a
    threshold large enough to truncate some blocks."""
    A = problems.aniso9(20)
    n = A.shape[0]
    rng = np.random.default_rng(5)
    sizes = []
    tot = 0
    while tot < n:
        s = int(min(rng.integers(1, 6), n - tot))
        sizes.append(s)
        tot += s
    agg = np.repeat(np.arange(len(sizes)), sizes).astype(np.int32)
    agg = agg[rng.permutation(n)]
    W = np.concatenate([np.ones((n, 1)), rng.standard_normal((n, 3))], axis=1)
    W /= np.linalg.norm(W, axis=0)
    for tol in (0.1, 30.0):
        Ho = O.setup(A, [agg], [n, len(sizes)], W, tol=tol)
        Hg = amg.Hierarchy(A, [agg], [n, len(sizes)], W, amg.opts(tol_svd=tol))
        worst, ex, sig, sgn = compare_prolongators(Hg, Ho, atol=1e-10)
        compare_coarse_matrices(Ho, ex, sig, sgn)
        if tol > 1:
            assert Hg.info()["truncated_aggs"] > 0
        b = np.random.default_rng(1).uniform(-1, 1, n)
        x, info, st = Hg.solve(b)
        _, res = O.solve(Ho, b)
        assert abs(info[0]["iters"] - res[0].iters) <= 1


def test_invalid_inputs_rejected(amg):
    A = problems.poisson5(4)
    W = np.ones((16, 1))
    agg = (np.arange(16) // 4).astype(np.int32)
    bad = A.copy()
    bad.indices = bad.indices.copy()
    bad.indices[3] = 99
    with pytest.raises(amg.AMGError) as e:
        amg.Hierarchy(bad, [agg], [16, 4], W)
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    empty = agg.copy()
    empty[empty == 2] = 1
    with pytest.raises(amg.AMGError) as e:
        amg.Hierarchy(A, [empty], [16, 4], W)
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    with pytest.raises(amg.AMGError):
        amg.Hierarchy(A, [agg], [16, 4], np.ones((16, 17)))
    H = amg.Hierarchy(A, [agg], [16, 4], W)
    with pytest.raises(amg.AMGError):
        H.solve(np.ones((16, 1)), options=amg.opts(cycle_precision=16))


def test_indefinite_coarsest_not_spd(amg):
    A = sp.csr_matrix(np.array([[1.0, 2.0], [2.0, 1.0]]))
    with pytest.raises(amg.AMGError) as e:
        amg.Hierarchy(A, [], [2], np.ones((2, 1)))
    assert e.value.status == amg.AMG_ERR_NOT_SPD


def test_timer_counts_launches(amg, built):
    P, Ho, Hg = built["aniso64"]
    Hg.timer_enable(amg.KERNEL_SPMV_CG)
    x, info, st = Hg.solve(P.B[:, 0].copy())
    ms, n = Hg.timer_read()
    Hg.timer_enable(amg.KERNEL_SPMV_CG, False)
    assert n >= info[0]["iters"] and ms > 0
