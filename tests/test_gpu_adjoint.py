"""Differentiable solve on the GPU: autograd gradients with respect to the
cell coefficients of the cell-centred diffusion workload, checked by central
finite differences (h = 1e-6 k, direct solves on the host) and against the
oracle's adjoint gradient, with the float64 cycle and with the float32 cycle."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import inputs, problems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


def _fd_loss(N, k, B, Xt):
    A = problems.cc5(N, k).tocsc()
    X = spla.splu(A).solve(B)
    return float(np.sum((X - Xt) ** 2))


@pytest.mark.parametrize("prec,rtol", [(64, 1e-13), (32, 1e-12)])
def test_autograd_gradient_matches_fd_and_oracle(amg, prec, rtol):
    import torch
    from paper_1907_04417_gb300.autograd import CellCentredDiffusion, solve

    N = 48
    P = inputs.diffusion_cc(N, nrhs=8, max_coarse=256)
    k = P.meta["kcell"]
    Xt = P.meta["x_target"]
    dev = torch.device("cuda")
    asm = CellCentredDiffusion(N, device=dev)
    kt = torch.tensor(k, device=dev, requires_grad=True)
    vals = asm.values(kt)
    H = amg.Hierarchy((asm.rowptr.to(dev), asm.col.to(dev), vals.detach().contiguous()), P.aggs, P.n_nodes,
                      torch.from_numpy(P.W).to(dev))
    o = amg.opts(rtol=rtol, cycle_precision=prec, maxit=5000)
    B = torch.from_numpy(P.B).to(dev)
    X = solve(vals, B, H, o)
    loss = ((X - torch.from_numpy(Xt).to(dev)) ** 2).sum()
    loss.backward()
    g = kt.grad.cpu().numpy().ravel()

    # central differences through independent direct solves
    rng = np.random.default_rng(55)
    cells = rng.choice(N * N, 20, replace=False)
    gmax = np.abs(g).max()
    for c in cells:
        h = 1e-6 * k.ravel()[c]
        kp = k.copy().ravel()
        kp[c] += h
        km = k.copy().ravel()
        km[c] -= h
        fd = (_fd_loss(N, kp.reshape(N, N), P.B, Xt) - _fd_loss(N, km.reshape(N, N), P.B, Xt)) / (2 * h)
        assert abs(fd - g[c]) <= 1e-5 * (abs(fd) + 1e-3 * gmax), (c, fd, g[c])

    # the oracle's adjoint gradient chained through the same assembly
    Ho = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    Xo, _ = O.solve(Ho, P.B, rtol=1e-13)
    _, go, _ = O.adjoint(Ho, 2 * (Xo - Xt), Xo, rtol=1e-13)
    from paper_1907_04417_gb300.autograd import CellCentredDiffusion as CCD
    asm_c = CCD(N)
    kc = torch.tensor(k, requires_grad=True)
    (asm_c.values(kc) * torch.from_numpy(go)).sum().backward()
    gor = kc.grad.numpy().ravel()
    err = np.linalg.norm(g - gor) / np.linalg.norm(gor)
    assert err <= (1e-8 if prec == 64 else 1e-7), err


def test_gradient_wrt_rhs_is_lambda(amg):
    import torch
    from paper_1907_04417_gb300.autograd import solve
    P = inputs.diffusion_cc(32, nrhs=2, max_coarse=128)
    dev = torch.device("cuda")
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    vals = torch.from_numpy(P.A.data).to(dev).requires_grad_(True)
    B = torch.from_numpy(P.B).to(dev).requires_grad_(True)
    o = amg.opts(rtol=1e-13)
    X = solve(vals, B, H, o)
    W = torch.from_numpy(np.random.default_rng(2).standard_normal(P.B.shape)).to(dev)
    (X * W).sum().backward()
    lam = spla.spsolve(P.A.tocsc(), W.cpu().numpy())
    np.testing.assert_allclose(B.grad.cpu().numpy(), lam, rtol=1e-9, atol=1e-12)
    # dL/da_ij = -lambda_i x_j on the pattern
    rows = np.repeat(np.arange(P.n), np.diff(P.A.indptr))
    Xc = X.detach().cpu().numpy()
    ga = -np.sum(lam[rows] * Xc[P.A.indices], axis=1)
    np.testing.assert_allclose(vals.grad.cpu().numpy(), ga, rtol=1e-8, atol=1e-12)
