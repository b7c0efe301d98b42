"""Host-side pieces of the differentiable solve: the torch assembly of the
cell-centred operator matches the numpy one and differentiates correctly."""
import numpy as np
import torch

from paper_1907_04417_gb300.autograd import CellCentredDiffusion
from paper_1907_04417_gb300.hostsetup import problems


def test_torch_assembly_matches_numpy():
    N = 9
    k = problems.lognormal_field(N, 1.0, seed=3)
    A = problems.cc5(N, k)
    asm = CellCentredDiffusion(N)
    v = asm.values(torch.from_numpy(k))
    np.testing.assert_array_equal(asm.rowptr.numpy(), A.indptr)
    np.testing.assert_array_equal(asm.col.numpy(), A.indices)
    np.testing.assert_allclose(v.numpy(), A.data, rtol=1e-15)


def test_torch_assembly_jacobian_vector_product():
    N = 6
    k = torch.from_numpy(problems.lognormal_field(N, 1.0, seed=4)).requires_grad_(True)
    asm = CellCentredDiffusion(N)
    w = torch.randn(asm.nnz, dtype=torch.float64, generator=torch.Generator().manual_seed(0))
    (asm.values(k) * w).sum().backward()
    g = k.grad.numpy().ravel()
    kk = k.detach().numpy()
    for c in (0, 7, 20, 35):
        h = 1e-6 * kk.ravel()[c]
        kp = kk.copy().ravel(); kp[c] += h
        km = kk.copy().ravel(); km[c] -= h
        fd = (problems.cc5(N, kp.reshape(N, N)).data - problems.cc5(N, km.reshape(N, N)).data) @ w.numpy() / (2 * h)
        np.testing.assert_allclose(g[c], fd, rtol=1e-7)
