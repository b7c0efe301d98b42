"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark times (graphs, autotuner, check interval, 32 right-hand sides).

* anisotropic 9-point, 1024 x 1024, m = 4, five levels: every prolongator
  block and coarse matrix against the oracle, one V-cycle, the FP64 PCG
  iteration count against the oracle's stored count, the FP64 iterate at a
  fixed iteration count element by element, and the FP32-cycle batch of the
  benchmark (true residual, iterations within three of FP64);
* jumping coefficients 128^3 (m = 3): setup, V-cycle and FP64 PCG against the
  oracle, FP32-cycle batch by its properties;
* uneven elasticity batch (eight systems, m = 6): the batched solve by its
  properties, one member's setup and FP64 PCG against the oracle;
* cell-centred diffusion 512^2 (m = 3): setup and FP64 PCG against the
  oracle, the adjoint gradient against its closed form with a direct solve,
  and dL/dk against central differences.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import inputs, problems

from .gpu_helpers import compare_coarse_matrices, compare_prolongators

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
RTOL_TRUE = 1.1e-8
# The oracle's counts are taken live on the host that runs the test for the
# 3D and cell-centred workloads: their inputs pass through libm and BLAS
# routines whose last bits differ between hosts, and a last-bit change of an
# edge weight can change a matching decision (the stored counts, from another
# host, differ by up to ten iterations).


@pytest.fixture(scope="module")
def amg():
    import torch  # noqa: F401
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


def _true_relres(A, B, X):
    B = B.reshape(B.shape[0], -1)
    X = X.reshape(B.shape)
    return np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)


def _setup_parity(P, Ho, Hg):
    info = Hg.info()
    assert info["levels"] == Ho.L
    assert info["n_level"] == [l.A.shape[0] for l in Ho.levels]
    assert info["nnz_level"] == [l.A.nnz for l in Ho.levels]
    assert info["opc"] == pytest.approx(O.operator_complexity(Ho), rel=1e-12)
    _, ex, sig, sgn = compare_prolongators(Hg, Ho, atol=1e-10)
    compare_coarse_matrices(Ho, ex, sig, sgn, rtol=1e-10)


def _fp64_parity(amg, P, Ho, Hg, b, expect_iters=None):
    x, info, st = Hg.solve(b, options=amg.opts(maxit=5000))
    assert st == amg.AMG_OK and info[0]["converged"]
    it = info[0]["iters"]
    if expect_iters is None:
        _, res = O.solve(Ho, b)
        expect_iters = res[0].iters
    assert abs(it - expect_iters) <= 1, (it, expect_iters)
    assert _true_relres(P.A, b, x)[0] <= RTOL_TRUE
    return it


def _fixed_iterate_parity(amg, Ho, Hg, b, k):
    x, info, st = Hg.solve(b, options=amg.opts(maxit=k))
    assert st == amg.AMG_ERR_NOT_CONVERGED and info[0]["iters"] == k
    xf, _ = O.solve(Ho, b, fixed_iters=k)
    err = np.linalg.norm(x - xf) / np.linalg.norm(xf)
    assert err <= 1e-10, err


def _batch_properties(amg, P, Hg, B, maxit=5000):
    """FP32-cycle and FP64 solves of the same block: every column reaches the
    true residual, FP32 needs at most three more iterations than FP64, and
    the two solutions agree to the accuracy the tolerance allows.  Both
    float32-cycle modes: the default (x, r, q double-float, p float32) and
    outer_fp64 (x, r, p, q and the CG arithmetic in float64)."""
    X64, i64, st64 = Hg.solve(B, options=amg.opts(cycle_precision=64, maxit=maxit))
    assert st64 == amg.AMG_OK
    r64 = _true_relres(P.A, B, X64)
    assert r64.max() <= RTOL_TRUE, r64.max()
    out = {}
    for outer in (0, 1):
        X32, i32, st32 = Hg.solve(B, options=amg.opts(cycle_precision=32, maxit=maxit, outer_fp64=outer))
        assert st32 == amg.AMG_OK, outer
        r32 = _true_relres(P.A, B, X32)
        assert r32.max() <= RTOL_TRUE, (outer, r32.max())
        for c in range(B.shape[1]):
            assert i32[c]["iters"] <= i64[c]["iters"] + 3, (outer, c, i32[c]["iters"], i64[c]["iters"])
        err = np.linalg.norm(X32 - X64, axis=0) / np.linalg.norm(X64, axis=0)
        assert err.max() <= 1e-6, (outer, err.max())
        out[outer] = i32
    return i64, out[0]


# ------------------------------------------------ anisotropic, 1024^2 --

@pytest.fixture(scope="module")
def aniso(amg):
    P = inputs.anisotropic(1024, nrhs=1)
    Ho = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    Hg = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    return P, Ho, Hg


def test_aniso_full_setup(aniso):
    P, Ho, Hg = aniso
    assert P.n_nodes == [1048576, 65536, 4096, 256, 16]
    _setup_parity(*aniso)


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 2e-5)])
def test_aniso_full_vcycle(amg, aniso, prec, tol):
    P, Ho, Hg = aniso
    R = np.random.default_rng(11).standard_normal((P.n, 3))
    Zg = Hg.vcycle(R, amg.opts(cycle_precision=prec))
    Zo = O.vcycle(Ho, R)
    assert np.linalg.norm(Zg - Zo) / np.linalg.norm(Zo) <= tol


def test_aniso_full_fp64_iterations_and_iterate(amg, aniso):
    P, Ho, Hg = aniso
    gold = json.load(open(os.path.join(HERE, "golden", "oracle_iterations.json")))["aniso9_1024x1024"]
    b = P.B[:, 0].copy()
    _fp64_parity(amg, P, Ho, Hg, b, expect_iters=gold["iters"])
    _fixed_iterate_parity(amg, Ho, Hg, b, 20)


def test_aniso_full_bench_batch(amg, aniso):
    """The benchmark's own block: 32 seeded columns, column 0 the workload's
    RHS, solved with the benchmark's options."""
    import bench
    P, Ho, Hg = aniso
    B = bench.rhs_block(P, 32, 0)
    gold = json.load(open(os.path.join(HERE, "golden", "oracle_iterations.json")))["aniso9_1024x1024"]
    i64, i32 = _batch_properties(amg, P, Hg, B)
    assert abs(i64[0]["iters"] - gold["iters"]) <= 1


# ------------------------------------------------ jumping 3D, 128^3 --

@pytest.fixture(scope="module")
def jump(amg):
    P = inputs.jumping3d(128, nrhs=32)
    Ho = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    Hg = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    return P, Ho, Hg


def test_jump_full_setup_vcycle_pcg(amg, jump):
    P, Ho, Hg = jump
    _setup_parity(P, Ho, Hg)
    R = np.random.default_rng(12).standard_normal((P.n, 2))
    Zg = Hg.vcycle(R)
    Zo = O.vcycle(Ho, R)
    assert np.linalg.norm(Zg - Zo) / np.linalg.norm(Zo) <= 1e-12
    it = _fp64_parity(amg, P, Ho, Hg, P.B[:, 0].copy())
    _fixed_iterate_parity(amg, Ho, Hg, P.B[:, 0].copy(), min(it, 10))


def test_jump_full_batch(amg, jump):
    P, Ho, Hg = jump
    _batch_properties(amg, P, Hg, P.B)


# ------------------------------------------------ elasticity batch --

def test_elasticity_full_batch(amg):
    batch = inputs.elasticity_batch()
    Hs = [amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W) for P in batch]
    res = {}
    # float64; the float32 cycle with double-float CG; the float32 cycle with float64 CG
    for key, prec, outer in ((64, 64, 0), (32, 32, 0), ("32f", 32, 1)):
        X, infos, st = amg.solve_batched(Hs, [P.B for P in batch],
                                         options=amg.opts(cycle_precision=prec, maxit=5000, outer_fp64=outer))
        assert st == amg.AMG_OK
        for s, (P, Xs) in enumerate(zip(batch, X)):
            r = _true_relres(P.A, P.B, Xs)
            assert r.max() <= RTOL_TRUE, (s, key, r.max())
        res[key] = infos
    for s in range(len(batch)):
        for c in range(batch[s].B.shape[1]):
            assert res[32][s][c]["iters"] <= res[64][s][c]["iters"] + 3
            assert res["32f"][s][c]["iters"] <= res[64][s][c]["iters"] + 3
    # the smallest member against the oracle, solved on its own
    s = int(np.argmin([P.n for P in batch]))
    P = batch[s]
    Ho = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    _setup_parity(P, Ho, Hs[s])
    it = _fp64_parity(amg, P, Ho, Hs[s], P.B[:, 0].copy())
    assert abs(res[64][s][0]["iters"] - it) <= 1


# ------------------------------------------------ cell-centred 512^2 --

@pytest.fixture(scope="module")
def ccd(amg):
    P = inputs.diffusion_cc(512)
    Ho = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    Hg = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    return P, Ho, Hg


def test_cc_full_setup_pcg_batch(amg, ccd):
    P, Ho, Hg = ccd
    _setup_parity(P, Ho, Hg)
    it = _fp64_parity(amg, P, Ho, Hg, P.B[:, 0].copy())
    _fixed_iterate_parity(amg, Ho, Hg, P.B[:, 0].copy(), min(it, 10))
    _batch_properties(amg, P, Hg, P.B)


def test_cc_full_adjoint(amg, ccd):
    """dL/da_ij = -sum_c lambda_ic x_jc with A lambda = dL/dx from a direct
    solve; dL/dk at sampled cells against that closed form pushed through a
    central difference of the numpy assembly.  (At 512^2 the loss is about
    1e14, so differences of two direct solves are dominated by rounding; the
    end-to-end finite-difference check runs on the 48^2 case.)"""
    import torch
    from paper_1907_04417_gb300.autograd import CellCentredDiffusion, solve
    P, Ho, Hg = ccd
    N = P.meta["grid"]
    k = P.meta["kcell"]
    Xt = P.meta["x_target"]
    dev = torch.device("cuda")
    asm = CellCentredDiffusion(N, device=dev)
    kt = torch.tensor(k, device=dev, requires_grad=True)
    vals = asm.values(kt)
    o = amg.opts(rtol=1e-12, cycle_precision=32, maxit=5000)
    X = solve(vals, torch.from_numpy(P.B).to(dev), Hg, o)
    loss = ((X - torch.from_numpy(Xt).to(dev)) ** 2).sum()
    vals.retain_grad()
    loss.backward()
    Xc = X.detach().cpu().numpy()
    lam = spla.splu(P.A.tocsc()).solve(2 * (Xc - Xt))
    rows = np.repeat(np.arange(P.n), np.diff(P.A.indptr))
    ga = -np.sum(lam[rows] * Xc[P.A.indices], axis=1)
    gv = vals.grad.cpu().numpy()
    assert np.linalg.norm(gv - ga) / np.linalg.norm(ga) <= 1e-8
    g = kt.grad.cpu().numpy().ravel()
    for c in np.random.default_rng(56).choice(N * N, 16, replace=False):
        h = 1e-5 * k.ravel()[c]
        kp = k.copy().ravel()
        kp[c] += h
        km = k.copy().ravel()
        km[c] -= h
        dv = (problems.cc5(N, kp.reshape(N, N)).data - problems.cc5(N, km.reshape(N, N)).data) / (2 * h)
        ref = float(ga @ dv)
        # lambda comes from an iterative solve (rtol 1e-12): per cell 1e-6 of
        # the value plus 1e-7 of the gradient's scale
        assert abs(ref - g[c]) <= 1e-6 * abs(ref) + 1e-7 * np.abs(g).max(), (c, ref, g[c])
