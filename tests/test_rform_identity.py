"""The algebra behind the library's restriction by R (CPU, no GPU).

With one pre-sweep of l1-Jacobi from zero, the iterate entering the
restriction of the V-cycle (Section 5) is u = D^{-1} f, and the restricted
residual P^T (f - A u) equals R f with R = P^T (I - A D^{-1}).  The library
keeps R by aggregate: every coarse dof of aggregate a has R's column pattern
equal to a's halo (a's rows and every column of those rows of A), so R is
block-structured with one shared pattern per aggregate.  These tests check
both facts on the oracle's hierarchies, with R formed densely from the
oracle's A, D and P (nothing of the library): the identity against the
oracle's own pre-sweep, residual and P^T on every level, and the pattern.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import inputs


@pytest.fixture(scope="module", params=["aniso32", "jump8", "elast4"])
def hier(request):
    mk = {"aniso32": lambda: inputs.anisotropic(32, nrhs=1, levels=4),
          "jump8": lambda: inputs.jumping3d(8, nrhs=1, max_coarse=64),
          "elast4": lambda: inputs.elasticity_grid(4, nrhs=1, levels=3)}[request.param]
    P = mk()
    return O.setup(P.A, P.aggs, P.n_nodes, P.W)


def test_restricted_residual_is_R_f(hier):
    H = hier
    rng = np.random.default_rng(31)
    for k in range(H.L - 1):
        A = H.levels[k].A.toarray()
        d = H.levels[k].d
        Pk = H.levels[k + 1].P.toarray()
        R = Pk.T @ (np.eye(A.shape[0]) - A / d[None, :])
        f = rng.uniform(-1.0, 1.0, (A.shape[0], 3))
        u = f / d[:, None]                      # the oracle's first pre-sweep from zero
        want = Pk.T @ (f - A @ u)               # its residual and restriction
        got = R @ f
        assert np.abs(got - want).max() <= 1e-13 * max(1.0, np.abs(want).max())


def test_R_pattern_is_the_aggregate_halo(hier):
    H = hier
    for k in range(H.L - 1):
        A = sp.csr_matrix(H.levels[k].A)
        d = H.levels[k].d
        Pk = sp.csr_matrix(H.levels[k + 1].P)
        R = (Pk.T @ (sp.identity(A.shape[0], format="csr") - A @ sp.diags(1.0 / d))).tocsr()
        R.eliminate_zeros()
        # the rows of each aggregate: the fine rows where its coarse dofs' P columns live
        Pc = Pk.tocsc()
        for c in range(Pk.shape[1]):
            rows = Pc.indices[Pc.indptr[c]:Pc.indptr[c + 1]]
            halo = set(rows.tolist())
            for i in rows:
                halo.update(A.indices[A.indptr[i]:A.indptr[i + 1]].tolist())
            cols = set(R.indices[R.indptr[c]:R.indptr[c + 1]].tolist())
            # R's non-zeros of a coarse dof lie in its aggregate's halo
            assert cols <= halo
