"""Seeded synthetic SPD operators standing in for the paper's test matrices.

The paper's matrices (Section 5: P1 finite elements from the MATLAB PDE toolbox
for the anisotropic diffusion problem, MFEM tetrahedral meshes for the Lame
equations) are not available, so every operator here is a finite-difference
stand-in with the same structure: SPD, Dirichlet dofs eliminated, O(1) entries
(everything is scaled by h^2).  All matrices are returned as scipy CSR with
int32 indices, sorted column indices and float64 values.

This module is problem definition only; it contains none of the solver's
arithmetic.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _csr(rows, cols, vals, n):
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    A.indptr = A.indptr.astype(np.int32)
    A.indices = A.indices.astype(np.int32)
    A.data = A.data.astype(np.float64)
    return A


def _stencil_2d(N, entries):
    """Assemble a constant-coefficient 2D stencil on an N x N interior grid.

    ``entries`` is a list of ((di, dj), value); couplings that leave the grid
    are Dirichlet neighbours and are dropped (their value is not moved to the
    diagonal: the diagonal entry is part of ``entries``).
    """
    I, J = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    I = I.ravel()
    J = J.ravel()
    idx = I * N + J
    rows, cols, vals = [], [], []
    for (di, dj), v in entries:
        if v == 0.0:
            continue
        I2, J2 = I + di, J + dj
        ok = (I2 >= 0) & (I2 < N) & (J2 >= 0) & (J2 < N)
        rows.append(idx[ok])
        cols.append((I2 * N + J2)[ok])
        vals.append(np.full(ok.sum(), v))
    return _csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), N * N)


def poisson5(N: int):
    """5-point Laplacian on an N x N interior grid (times h^2): 4 on the
    diagonal, -1 to each of the four neighbours.  nnz = 5 N^2 - 4 N."""
    e = [((0, 0), 4.0), ((1, 0), -1.0), ((-1, 0), -1.0), ((0, 1), -1.0), ((0, -1), -1.0)]
    return _stencil_2d(N, e)


def aniso9(N: int, eps: float = 1e-3, theta: float = np.pi / 6):
    """Rotated anisotropic diffusion -div(K grad u) with the coefficient
    matrix K = [[a, c], [c, b]], a = eps + cos^2 theta, b = eps + sin^2 theta,
    c = cos theta sin theta (the model problem of Section 5.1), discretised by
    the centred 9-point finite-difference stencil (times h^2):

      u_xx, u_yy: standard 3-point differences,
      u_xy ~ (u(i+1,j+1) - u(i+1,j-1) - u(i-1,j+1) + u(i-1,j-1)) / 4.

    The operator is SPD for every N because ab > c^2.  nnz = 9N^2 - 12N + 4.
    Index (i, j) -> i*N + j, with i along x.
    """
    ct, st = np.cos(theta), np.sin(theta)
    a = eps + ct * ct
    b = eps + st * st
    c = ct * st
    e = [
        ((0, 0), 2 * a + 2 * b),
        ((1, 0), -a), ((-1, 0), -a),
        ((0, 1), -b), ((0, -1), -b),
        ((1, 1), -c / 2), ((-1, -1), -c / 2),
        ((1, -1), c / 2), ((-1, 1), c / 2),
    ]
    return _stencil_2d(N, e)


def harmonic(k1, k2):
    return 2.0 * k1 * k2 / (k1 + k2)


def jump7(N: int, block: int = 8, seed: int = 2003, log10_range=(-3.0, 3.0)):
    """3D jumping-coefficient diffusion -div(k grad u) on an N^3 interior
    grid, 7-point stencil.  k is constant on each block^3 sub-cube with
    log10 k ~ U(log10_range).  The coupling between two neighbouring nodes is
    the harmonic mean of their k; a Dirichlet neighbour couples with the node's
    own k (kept on the diagonal, dropped off it).  nnz = 7 N^3 - 6 N^2.
    Returns (A, kfield)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = (N + block - 1) // block
    kb = 10.0 ** rng.uniform(log10_range[0], log10_range[1], size=(nb, nb, nb))
    I, J, K = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    kn = kb[I // block, J // block, K // block]
    idx = (I * N + J) * N + K
    n = N ** 3
    diag = np.zeros((N, N, N))
    rows, cols, vals = [], [], []
    for ax in range(3):
        for s in (1, -1):
            sl_src = [slice(None)] * 3
            sl_dst = [slice(None)] * 3
            if s == 1:
                sl_src[ax] = slice(0, N - 1)
                sl_dst[ax] = slice(1, N)
            else:
                sl_src[ax] = slice(1, N)
                sl_dst[ax] = slice(0, N - 1)
            kf = harmonic(kn[tuple(sl_src)], kn[tuple(sl_dst)])
            diag[tuple(sl_src)] += kf
            rows.append(idx[tuple(sl_src)].ravel())
            cols.append(idx[tuple(sl_dst)].ravel())
            vals.append(-kf.ravel())
            # boundary face in direction s along ax: Dirichlet neighbour
            sl_b = [slice(None)] * 3
            sl_b[ax] = N - 1 if s == 1 else 0
            diag[tuple(sl_b)] += kn[tuple(sl_b)]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return _csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n), kn


def elasticity(N: int, E: float = 1.0, nu: float = 0.3):
    """Navier-Cauchy operator -mu Lap u - (lambda + mu) grad div u on an
    N^3 node grid with 3 dofs per node, node-ordered (dof = 3*node + comp,
    as in the node-based ordering of Section 5.2).

    Compact centred differences (times h^2), interior stencil:
      * same component c, direction d: graph-Laplacian edge of weight
        mu + (lambda + mu) * delta_cd between the two neighbouring nodes;
      * cross components c != d: u_d(p + s_c e_c + s_d e_d) enters row (p, c)
        with -(lambda + mu) s_c s_d / 4.
    The face x = 0 is clamped: the plane x = -1 is a Dirichlet plane whose
    same-component edges stay on the diagonal.  Elsewhere same-component
    edges that leave the grid are dropped with their diagonal part.

    Boundary closure of the cross terms (energy form): the entry between
    (q, c) and (q', d) comes from the centred divergence at their common
    neighbour o = q - s_c e_c = q' - s_d e_d, and is kept only where o is a
    grid node whose centred differences in both directions c and d are
    complete (each neighbour a grid node or on the clamped plane).  The
    matrix is then mu * (clamped Laplacians) + (lambda + mu) * (sum over o of
    (discrete div at o)^2 + per-line compact minus centred-wide second
    differences), each part positive semi-definite, so A is SPD for every N.
    Dropping out-of-grid couplings alone leaves A indefinite from N = 16."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    I, J, K = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    P = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    node = (P[:, 0] * N + P[:, 1]) * N + P[:, 2]
    nn = N ** 3
    rows, cols, vals = [], [], []
    diag = np.zeros((nn, 3))
    unit = np.eye(3, dtype=np.int64)
    for c in range(3):
        for d in range(3):
            w = mu + (lam + mu) * (1.0 if c == d else 0.0)
            for s in (1, -1):
                Q = P + s * unit[d]
                inside = np.all((Q >= 0) & (Q < N), axis=1)
                clamped = (d == 0) & (Q[:, 0] < 0)
                diag[inside | clamped, c] += w
                qn = (Q[inside, 0] * N + Q[inside, 1]) * N + Q[inside, 2]
                rows.append(3 * node[inside] + c)
                cols.append(3 * qn + c)
                vals.append(np.full(inside.sum(), -w))
    g = (lam + mu) / 4.0
    for c in range(3):
        for d in range(3):
            if c == d:
                continue
            for sc in (1, -1):
                for sd in (1, -1):
                    Q = P + sc * unit[c] + sd * unit[d]
                    O = P + sc * unit[c]                     # centre of the divergence term
                    inside = np.all((O >= 0) & (O < N), axis=1)
                    for e in (c, d):
                        lo = -1 if e == 0 else 0              # x = -1 is the clamped plane
                        inside &= (O[:, e] - 1 >= lo) & (O[:, e] + 1 < N)
                    inside &= np.all((Q >= 0) & (Q < N), axis=1)  # a clamped-plane value is 0
                    qn = (Q[inside, 0] * N + Q[inside, 1]) * N + Q[inside, 2]
                    rows.append(3 * node[inside] + c)
                    cols.append(3 * qn + d)
                    vals.append(np.full(inside.sum(), -g * sc * sd))
    rows.append(np.arange(3 * nn))
    cols.append(np.arange(3 * nn))
    vals.append(diag.ravel())
    return _csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), 3 * nn)


def cc5_structure(N: int):
    """Face lists of the cell-centred 5-point scheme on an N x N cell grid.

    Returns (pairs, bcell): ``pairs`` is an (F, 2) array of neighbouring
    cells sharing an interior face, ``bcell`` lists, once per boundary face,
    the cell that owns it.  Cell (i, j) -> i*N + j."""
    I, J = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    idx = I * N + J
    px = np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], axis=1)
    py = np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], axis=1)
    pairs = np.concatenate([px, py], axis=0)
    bcell = np.concatenate([idx[0, :], idx[-1, :], idx[:, 0], idx[:, -1]])
    return pairs, bcell


def cc5(N: int, kcell: np.ndarray):
    """Cell-centred 5-point -div(k grad u) on an N x N cell grid (times h^2):
    interior face coefficient = harmonic mean of the two cells' k, a
    Dirichlet boundary face couples with 2 k_cell (half-cell distance).
    nnz = 5 N^2 - 4 N."""
    pairs, bcell = cc5_structure(N)
    k = kcell.ravel()
    kf = harmonic(k[pairs[:, 0]], k[pairs[:, 1]])
    n = N * N
    diag = np.zeros(n)
    np.add.at(diag, pairs[:, 0], kf)
    np.add.at(diag, pairs[:, 1], kf)
    np.add.at(diag, bcell, 2.0 * k[bcell])
    rows = np.concatenate([pairs[:, 0], pairs[:, 1], np.arange(n)])
    cols = np.concatenate([pairs[:, 1], pairs[:, 0], np.arange(n)])
    vals = np.concatenate([-kf, -kf, diag])
    return _csr(rows, cols, vals, n)


def lognormal_field(N: int, sigma: float = 1.0, seed: int = 2005):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(sigma * rng.standard_normal((N, N)))
