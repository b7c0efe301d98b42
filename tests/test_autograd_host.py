"""Host-side pieces of the differentiable solve: the torch assembly of the
cell-centred operator matches the numpy one and differentiates correctly."""
import numpy as np
import pytest
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


class _FakeHierarchy:
    """Stands in for a device hierarchy: only the values it was set up with."""

    def __init__(self, values):
        self.setup_values = values

    def solve(self, *a, **k):  # pragma: no cover - must not be reached
        raise AssertionError("a refused forward must not solve")


def test_forward_refuses_changed_values():
    from paper_1907_04417_gb300.autograd import AMGSolve, check_values
    N = 5
    asm = CellCentredDiffusion(N)
    k = torch.from_numpy(problems.lognormal_field(N, 1.0, seed=1))
    v = asm.values(k)
    H = _FakeHierarchy(v.numpy().copy())
    check_values(v, H)                                 # the same values pass
    v2 = v.clone()
    v2[3] *= 1.0 + 1e-9
    check_values(v * (1.0 + 1e-15), H)                 # rounding-size differences pass
    b = torch.ones(N * N, dtype=torch.float64)
    with pytest.raises(ValueError, match="differ"):
        AMGSolve.apply(v2.requires_grad_(True), b, H, None)
    with pytest.raises(ValueError, match="differ"):
        check_values(v[:-1], H)
