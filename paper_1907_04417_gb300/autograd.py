"""Differentiable AMG-PCG solve: x = A^{-1} b with an adjoint backward.

``AMGSolve.apply(values, b, hierarchy, options)`` returns x.  Its backward
receives g = dL/dx and runs, through the C ABI (amg_adjoint), one more
preconditioned CG solve with the same hierarchy, A lambda = g (A is SPD, so
A^{-T} = A^{-1}), followed by the fused kernel that writes
dL/da_ij = -sum_c lambda[i, c] x[j, c] for every stored entry of A.  The
gradient with respect to b is lambda.  ``values`` must hold A's CSR values in
the CSR order the hierarchy was set up with, and equal them: the forward
solve refuses values that differ from the hierarchy's by more than rounding
(a changed matrix needs a new Hierarchy).  The hierarchy is a constant preconditioner (the derivative
of the exact solution does not depend on it).

``CellCentredDiffusion`` assembles the cell-centred 5-point operator of the
differentiable workload from a cell coefficient field with torch operations,
so that autograd carries dL/dA on to dL/dk.
"""
from __future__ import annotations

import numpy as np
import torch

from . import amg
from .hostsetup import problems


VALUES_RTOL = 1e-12


def check_values(values, hierarchy):
    """Refuse a solve whose matrix values differ from those the hierarchy was
    set up with: the forward solve and the gradient would belong to the old
    matrix.  A caller that changes A (an optimisation step on the
    coefficients) builds a new Hierarchy.  Differences of rounding size (two
    assemblies of the same coefficients, at most VALUES_RTOL of the largest
    entry) are accepted."""
    ref = hierarchy.setup_values
    v = values.detach()
    if isinstance(ref, np.ndarray):
        ref = torch.from_numpy(ref)
    if v.shape != ref.shape:
        raise ValueError("values differ from the matrix the hierarchy was set up with (size); "
                         "build a new Hierarchy for the new matrix")
    d = (v.to(device=ref.device, dtype=ref.dtype) - ref).abs().max()
    if not bool(d <= VALUES_RTOL * ref.abs().max()):
        raise ValueError("values differ from the matrix the hierarchy was set up with; "
                         "build a new Hierarchy for the new matrix")


class AMGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, b, hierarchy, options=None):
        check_values(values, hierarchy)
        x, info, status = hierarchy.solve(b.detach().contiguous(), options=options)
        if status != amg.AMG_OK:
            raise amg.AMGError(status, f"forward solve: {info}")
        ctx.hierarchy = hierarchy
        ctx.options = options
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam, grad_vals, info, status = ctx.hierarchy.adjoint(gx.contiguous(), x, options=ctx.options)
        if status != amg.AMG_OK:
            raise amg.AMGError(status, f"adjoint solve: {info}")
        return grad_vals, lam, None, None


def solve(values, b, hierarchy, options=None):
    """x = A^{-1} b, differentiable in ``values`` (A's CSR values) and ``b``."""
    return AMGSolve.apply(values, b, hierarchy, options)


class CellCentredDiffusion:
    """Torch assembly of the cell-centred 5-point -div(k grad u) on an N x N
    cell grid (harmonic-mean faces, Dirichlet faces with 2 k_cell), in the
    CSR layout of ``problems.cc5``."""

    def __init__(self, N: int, device="cpu"):
        self.N = N
        pairs, bcell = problems.cc5_structure(N)
        A = problems.cc5(N, np.ones((N, N)))
        self.rowptr = torch.from_numpy(A.indptr.astype(np.int32))
        self.col = torch.from_numpy(A.indices.astype(np.int32))
        n = N * N
        # position of every (i, j) entry in CSR order (keys i*n + j ascend)
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(A.indptr))
        keys = rows * n + A.indices
        off_ij = np.searchsorted(keys, pairs[:, 0].astype(np.int64) * n + pairs[:, 1])
        off_ji = np.searchsorted(keys, pairs[:, 1].astype(np.int64) * n + pairs[:, 0])
        diag = np.searchsorted(keys, np.arange(n, dtype=np.int64) * (n + 1))
        dev = torch.device(device)
        self.pairs = torch.from_numpy(pairs).to(dev)
        self.bcell = torch.from_numpy(bcell).to(dev)
        self.off_ij = torch.from_numpy(off_ij).to(dev)
        self.off_ji = torch.from_numpy(off_ji).to(dev)
        self.diag = torch.from_numpy(diag).to(dev)
        self.nnz = A.nnz
        self.n = n

    def values(self, kcell: torch.Tensor) -> torch.Tensor:
        k = kcell.reshape(-1)
        kp, kq = k[self.pairs[:, 0]], k[self.pairs[:, 1]]
        kf = 2.0 * kp * kq / (kp + kq)
        d = torch.zeros(self.n, dtype=k.dtype, device=k.device)
        d = d.index_add(0, self.pairs[:, 0], kf).index_add(0, self.pairs[:, 1], kf)
        d = d.index_add(0, self.bcell, 2.0 * k[self.bcell])
        v = torch.zeros(self.nnz, dtype=k.dtype, device=k.device)
        v = v.index_put((self.off_ij,), -kf).index_put((self.off_ji,), -kf).index_put((self.diag,), d)
        return v
