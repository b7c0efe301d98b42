"""Bootstrap of the smooth vectors (Algorithm 1, Section 2) with the testing
phase on the GPU.

Stage r = 1..m-1 builds the single-vector hierarchy B_r from w_{r-1}: the
composed pairwise aggregates of the compatible weighted matching on w_{r-1}
(Section 3, a host step, ``aggregate``) and the prolongator of w_{r-1}
alone.  The testing phase applies the composite error operator of B_1..B_r
(symmetrized by default, Section 5 (i)) nu times to the random vector
``starts[r-1]`` on the device (amg_bootstrap_test), and w_r = x^nu /
||x^nu||_A.  The stage count is fixed (the desired rate of Algorithm 1 is
taken as 0), which gives the m smooth vectors the single hierarchy uses.
"""
from __future__ import annotations

import numpy as np

from . import amg


def bootstrap(A, w0, m: int, nu: int, aggregate, starts, symmetric: bool = True, options=None):
    """Returns (W, rhos, hierarchies): W = [w_0, ..., w_{m-1}] (n x m float64,
    w_0 as given, the others A-normalised), the stage estimates rho and the
    stage hierarchies B_1..B_{m-1} (closed by the caller)."""
    n = A.shape[0]
    W = np.empty((n, m))
    W[:, 0] = w0
    Hs, rhos = [], []
    for r in range(1, m):
        w = W[:, r - 1]
        aggs, n_nodes = aggregate(w)
        Hs.append(amg.Hierarchy(A, aggs, n_nodes, (w / np.linalg.norm(w))[:, None]))
        x, rho, anorm = amg.bootstrap_test(Hs, np.asarray(starts[r - 1], dtype=np.float64), nu, symmetric,
                                           options)
        W[:, r] = np.asarray(x, dtype=np.float64).reshape(n) / anorm[0]
        rhos.append(float(rho[0]))
    return W, rhos, Hs
