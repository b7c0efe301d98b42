"""Algebraically smooth test vectors, host side (input data).

The paper takes its smooth vectors from the bootstrap of Algorithm 1 and
remarks (Section 5) that starting from a random vector smoothed by enough
symmetrized relaxation sweeps gives very similar results.  This generator
follows that remark for every vector after the first: w_0 is the constant
vector (optionally perturbed), and each further w_r is a seeded random
vector after ``sweeps`` damped-Jacobi sweeps on A x = 0 (a relaxation the
solve phase does not use: the solve smooths with l1-Jacobi).  Every vector
is scaled to unit 2-norm.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def relaxed_vector(A: sp.csr_matrix, x: np.ndarray, sweeps: int, omega: float = 2.0 / 3.0):
    dinv = 1.0 / A.diagonal()
    for _ in range(sweeps):
        x = x - omega * dinv * (A @ x)
    return x


def smooth_vectors(A: sp.csr_matrix, m: int, seed: int, sweeps: int = 30,
                   w0_perturb: float = 0.0) -> np.ndarray:
    """Return W, an (n, m) float64 array of unit-2-norm smooth vectors."""
    n = A.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    W = np.empty((n, m))
    w0 = np.ones(n)
    if w0_perturb:
        w0 = w0 + rng.uniform(-w0_perturb, w0_perturb, size=n)
    W[:, 0] = w0
    for r in range(1, m):
        W[:, r] = relaxed_vector(A, rng.standard_normal(n), sweeps)
    W /= np.linalg.norm(W, axis=0, keepdims=True)
    return W
