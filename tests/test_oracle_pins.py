"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's formula: each compares the oracle with a
closed form, a hand-derived value, an independent dense construction, a
brute-force computation or a library routine the oracle does not use.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import aggregation, inputs, problems

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals[key] = [float(x) for x in rest]
    return vals


def _lap1d(n):
    return sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(n, n), format="csr")


def _small(N=12, m=3, steps=(2, 2), seed=0, prob="aniso"):
    A = problems.aniso9(N) if prob == "aniso" else problems.poisson5(N)
    rng = np.random.default_rng(seed)
    W = np.concatenate([np.ones((A.shape[0], 1)), rng.standard_normal((A.shape[0], m - 1))], axis=1)
    W /= np.linalg.norm(W, axis=0)
    aggs, nn = aggregation.aggregate_hierarchy(A, np.ones(A.shape[0]), list(steps))
    return A, aggs, nn, W


# ---------------------------------------------------------------- golden ----

def test_golden_galerkin_1d_laplacian():
    g = _read_golden("galerkin_1d_laplacian.txt")
    A = _lap1d(8).tocsr()
    agg = np.array(g["agg"], dtype=np.int32)
    H = O.setup(A, [agg], [8, 4], np.ones((8, 1)) / np.sqrt(8))
    want = np.array([g[f"A1_row{i}"] for i in range(4)])
    np.testing.assert_allclose(H.levels[1].A.toarray(), want, atol=1e-15)
    np.testing.assert_allclose(H.levels[0].d, g["l1"], atol=0)
    blk = H.levels[1].P.toarray()[:2, 0]
    np.testing.assert_allclose(blk, g["P_block"], atol=1e-16)


def test_golden_svd_threshold():
    g = _read_golden("svd_threshold_block.txt")
    Wa = np.array([g[f"W_row{i}"] for i in range(4)])
    for case in ("caseA", "caseB", "caseC"):
        nA, keep = g[case]
        U, S = O.local_basis(Wa, 0.1 * 4 / nA)
        assert U.shape[1] == int(keep)
        np.testing.assert_allclose(S, g["sigma"], rtol=1e-15)
        for j in range(int(keep)):
            np.testing.assert_allclose(U[:, j], g[f"u{j}"], atol=1e-15)


# ------------------------------------------------------- local SVD pins ----

@pytest.mark.parametrize("na,m", [(16, 4), (5, 3), (3, 5), (1, 4), (64, 6), (9, 1)])
def test_local_basis_orthonormal_eigen_and_span(na, m):
    rng = np.random.default_rng(na * 10 + m)
    Wa = rng.standard_normal((na, m))
    U, S = O.local_basis(Wa, 0.0)
    r = U.shape[1]
    assert r == min(na, m)
    # orthonormal columns (Section 4: P~^T P~ = I)
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-14)
    # left singular vectors are eigenvectors of W W^T with eigenvalue sigma^2
    lam = sla.eigh(Wa.T @ Wa, eigvals_only=True)[::-1][:r]
    np.testing.assert_allclose(S[:r] ** 2, lam, rtol=1e-12, atol=1e-14)
    for j in range(r):
        np.testing.assert_allclose(Wa @ (Wa.T @ U[:, j]), S[j] ** 2 * U[:, j], atol=1e-12 * S[0] ** 2)
    # untruncated range contains every local smooth vector
    np.testing.assert_allclose(U @ (U.T @ Wa), Wa, atol=1e-13)
    # sign rule: largest-magnitude entry of each column is positive
    for j in range(r):
        assert U[np.argmax(np.abs(U[:, j])), j] > 0


def test_local_basis_eckart_young():
    """||(I - U U^T) W||_2 equals the first dropped singular value."""
    rng = np.random.default_rng(7)
    Wa = rng.standard_normal((12, 5)) @ np.diag([5.0, 2.0, 1.0, 0.03, 0.01])
    sig = np.sqrt(sla.eigh(Wa.T @ Wa, eigvals_only=True))[::-1]
    U, S = O.local_basis(Wa, (sig[2] + sig[3]) / 2)
    assert U.shape[1] == 3
    R = Wa - U @ (U.T @ Wa)
    resid2 = np.sqrt(sla.eigh(R.T @ R, eigvals_only=True).max())
    np.testing.assert_allclose(resid2, sig[3], rtol=1e-10)


def test_local_basis_degenerate():
    U, S = O.local_basis(np.zeros((4, 2)), 1e-3)
    assert U.shape == (4, 1)
    np.testing.assert_allclose(U[:, 0], 0.5)
    # nothing passes the threshold: still one column, the leading one
    U, S = O.local_basis(np.array([[1e-9], [2e-9]]), 1.0)
    assert U.shape == (2, 1)
    np.testing.assert_allclose(U[:, 0], np.array([1, 2]) / np.sqrt(5), rtol=1e-12)


# --------------------------------------------------------- Galerkin pins ----

def test_galerkin_piecewise_constant_closed_form():
    """m = 1, w = 1: P is the normalised piecewise constant, so
    A_c[a, b] = sum_{i in a, j in b} a_ij / sqrt(n_a n_b)."""
    A = problems.aniso9(10)
    aggs, nn = aggregation.aggregate_hierarchy(A, np.ones(100), [3])
    H = O.setup(A, aggs, nn, np.ones((100, 1)) / 10.0)
    g = aggs[0]
    na = np.bincount(g)
    Ad = A.toarray()
    Ac = np.zeros((nn[1], nn[1]))
    for i in range(100):
        for j in range(100):
            Ac[g[i], g[j]] += Ad[i, j]
    Ac /= np.sqrt(np.outer(na, na))
    np.testing.assert_allclose(H.levels[1].A.toarray(), Ac, atol=1e-14)


def test_prolongator_orthonormal_and_coarse_spd():
    A, aggs, nn, W = _small(16, 4, (2, 2, 2))
    H = O.setup(A, aggs, nn, W)
    for k in range(1, H.L):
        P = H.levels[k].P.toarray()
        np.testing.assert_allclose(P.T @ P, np.eye(P.shape[1]), atol=1e-14)
        Ak = H.levels[k].A.toarray()
        np.testing.assert_allclose(Ak, Ak.T, atol=1e-14)
        assert np.linalg.eigvalsh(Ak).min() > 0
        # every fine row belongs to exactly one aggregate
        assert np.all((P != 0).sum(axis=1) >= 1)
        # n_c = sum of kept columns (Section 4)
        assert P.shape[1] == H.levels[k].r.sum()


def test_range_contains_smooth_vectors_without_truncation():
    A, aggs, nn, W = _small(12, 3, (2,))
    H = O.setup(A, aggs, nn, W, tol=0.0)
    P = H.levels[1].P.toarray()
    np.testing.assert_allclose(P @ (P.T @ W), W, atol=1e-13)


def test_setup_rejects_empty_aggregate():
    A = _lap1d(4).tocsr()
    with pytest.raises(ValueError):
        O.setup(A, [np.array([0, 0, 2, 2], dtype=np.int32)], [4, 3], np.ones((4, 1)))


# ------------------------------------------------ cycle / solver pins ----

def _dense_B(H, n):
    return np.stack([O.vcycle(H, e) for e in np.eye(n)], axis=1)


def test_two_grid_error_operator_bruteforce():
    A, aggs, nn, W = _small(10, 3, (2,))
    H = O.setup(A, aggs, nn, W)
    n = A.shape[0]
    Ad = A.toarray()
    P = H.levels[1].P.toarray()
    Minv = np.diag(1.0 / np.abs(Ad).sum(axis=1))
    I = np.eye(n)
    S = I - Minv @ Ad
    CG = I - P @ np.linalg.inv(P.T @ Ad @ P) @ P.T @ Ad
    E = S @ CG @ S
    E_oracle = I - _dense_B(H, n) @ Ad
    np.testing.assert_allclose(E_oracle, E, atol=1e-12)
    # the two-grid error operator contracts in the A-norm
    Lc = np.linalg.cholesky(Ad)
    Ea = Lc.T @ E @ np.linalg.inv(Lc.T)
    assert np.linalg.norm(Ea, 2) < 1.0


def test_preconditioner_symmetric_positive():
    A, aggs, nn, W = _small(10, 3, (2, 2))
    H = O.setup(A, aggs, nn, W)
    B = _dense_B(H, A.shape[0])
    np.testing.assert_allclose(B, B.T, atol=1e-13 * np.abs(B).max())
    assert np.linalg.eigvalsh((B + B.T) / 2).min() > 0


def test_one_level_is_exact():
    A = problems.poisson5(8)
    H = O.setup(A, [], [64], np.ones((64, 1)))
    b = np.random.default_rng(0).uniform(-1, 1, 64)
    x, res = O.solve(H, b)
    assert res[0].iters == 1
    np.testing.assert_allclose(A @ x, b, atol=1e-12)


def test_square_orthogonal_P_gives_exact_coarse_correction():
    """n_a = r_a everywhere: P is square orthogonal, P A_c^{-1} P^T = A^{-1},
    the two-grid error vanishes and PCG stops after one iteration."""
    A = problems.poisson5(6)
    n = A.shape[0]
    agg = (np.arange(n) // 2).astype(np.int32)
    W = np.random.default_rng(3).standard_normal((n, 2))
    H = O.setup(A, [agg], [n, n // 2], W, tol=0.0)
    assert H.levels[1].A.shape[0] == n
    b = np.random.default_rng(4).uniform(-1, 1, n)
    x, res = O.solve(H, b, rtol=1e-12)
    assert res[0].iters == 1


def test_unpreconditioned_cg_matches_scipy_iterates():
    A = problems.poisson5(10)
    b = np.random.default_rng(5).uniform(-1, 1, 100)
    for k in (1, 3, 7):
        mine = O.pcg(A, b, None, fixed_iters=k).x
        ref, _ = spla.cg(A, b, x0=np.zeros(100), rtol=0.0, atol=0.0, maxiter=k)
        np.testing.assert_allclose(mine, ref, rtol=1e-10, atol=1e-12)


def test_pcg_solution_against_direct_solve():
    P = inputs.anisotropic(N=32, nrhs=2)
    H = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    X, res = O.solve(H, P.B)
    Xd = spla.spsolve(P.A.tocsc(), P.B)
    kappa = np.linalg.cond(P.A.toarray())
    for c in range(2):
        assert res[c].converged
        tr = np.linalg.norm(P.B[:, c] - P.A @ X[:, c]) / np.linalg.norm(P.B[:, c])
        assert tr <= 1.1e-8
        err = np.linalg.norm(X[:, c] - Xd[:, c]) / np.linalg.norm(Xd[:, c])
        assert err <= kappa * 1e-8


def test_zero_rhs():
    P = inputs.poisson(N=8)
    H = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    x, res = O.solve(H, np.zeros(64))
    assert res[0].iters == 0 and np.all(x == 0)


def test_residuals_preconditioner_orthogonal():
    """CG residuals are B-orthogonal: r_i^T B r_j = 0 for i != j."""
    P = inputs.poisson(N=12)
    H = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    A, b = P.A, P.B[:, 0]
    R = []
    for k in range(1, 6):
        x = O.pcg(A, b, lambda r: O.vcycle(H, r), fixed_iters=k).x
        R.append(b - A @ x)
    Z = [O.vcycle(H, r) for r in R]
    G = np.array([[ri @ zj for zj in Z] for ri in R])
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() <= 1e-8 * np.abs(np.diag(G)).max()


# ---------------------------------------------------------- adjoint pins ----

def test_adjoint_gradient_dense_and_fd():
    N = 12
    k = problems.lognormal_field(N, 1.0, seed=11)
    A = problems.cc5(N, k)
    n = A.shape[0]
    rng = np.random.default_rng(12)
    b = rng.uniform(-1, 1, (n, 2))
    aggs, nn = aggregation.aggregate_hierarchy(A, np.ones(n), [2, 2])
    W = np.concatenate([np.ones((n, 1)), rng.standard_normal((n, 1))], axis=1)
    W /= np.linalg.norm(W, axis=0)
    H = O.setup(A, aggs, nn, W)
    X, _ = O.solve(H, b, rtol=1e-13)
    xt = rng.standard_normal((n, 2))
    g = 2 * (X - xt)
    Lam, grad, _ = O.adjoint(H, g, X, rtol=1e-13)
    # dense: dL/dA = -A^{-1} g x^T, restricted to A's pattern
    Ad = A.toarray()
    Gd = -np.linalg.solve(Ad, g) @ X.T
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    np.testing.assert_allclose(grad, Gd[rows, A.indices], rtol=1e-9, atol=1e-11)

    # central differences through the assembly (cell coefficients)
    def loss(kk):
        Ak = problems.cc5(N, kk).toarray()
        x = np.linalg.solve(Ak, b)
        return np.sum((x - xt) ** 2)

    for c in rng.choice(n, 5, replace=False):
        h = 1e-6 * k.ravel()[c]
        kp = k.copy().ravel(); kp[c] += h
        km = k.copy().ravel(); km[c] -= h
        fd = (loss(kp.reshape(N, N)) - loss(km.reshape(N, N))) / (2 * h)
        # chain rule: dA/dk_c from a complex-step free finite difference of A
        dA = (problems.cc5(N, kp.reshape(N, N)) - problems.cc5(N, km.reshape(N, N))) / (2 * h)
        dA = dA.tocsr()
        an = 0.0
        for i in range(n):
            for p in range(dA.indptr[i], dA.indptr[i + 1]):
                an += Gd[i, dA.indices[p]] * dA.data[p]
        np.testing.assert_allclose(an, fd, rtol=1e-5)


def test_complexity_metrics():
    A, aggs, nn, W = _small(16, 2, (2, 2))
    H = O.setup(A, aggs, nn, W)
    opc = O.operator_complexity(H)
    assert opc == pytest.approx(sum(l.A.nnz for l in H.levels) / A.nnz)
    n = [l.A.shape[0] for l in H.levels]
    assert O.coarsening_ratio(H) == pytest.approx(np.mean([n[0] / n[1], n[1] / n[2]]))


# ------------------------------------------------- bootstrap (Algorithm 1) --

def _bootstrap_hierarchies(N=10):
    """Two single-vector hierarchies on one aniso9 operator, built from two
    different vectors (so the aggregates differ), as stages B_1, B_2."""
    A = problems.aniso9(N)
    n = A.shape[0]
    w1 = np.ones(n)
    w2 = np.random.default_rng(21).standard_normal(n)
    Hs = []
    for w, steps in ((w1, [2]), (w2, [2, 2])):
        aggs, nn = aggregation.aggregate_hierarchy(A, w, steps)
        Hs.append(O.setup(A, aggs, nn, (w / np.linalg.norm(w))[:, None]))
    return A, Hs


def test_bootstrap_composite_matches_dense_product():
    """Eq. (comp_AMG) applies (I - B_1 A) first; the symmetrized product of
    Section 5 (i) is (I - B_1 A)(I - B_2 A)(I - B_2 A)(I - B_1 A)."""
    A, Hs = _bootstrap_hierarchies()
    n = A.shape[0]
    Ad = A.toarray()
    E1 = np.eye(n) - _dense_B(Hs[0], n) @ Ad
    E2 = np.eye(n) - _dense_B(Hs[1], n) @ Ad
    x = np.random.default_rng(5).standard_normal((n, 3))
    np.testing.assert_allclose(O.composite_error(Hs, A, x, symmetric=False), E2 @ E1 @ x, atol=1e-12)
    np.testing.assert_allclose(O.composite_error(Hs, A, x, symmetric=True), E1 @ E2 @ E2 @ E1 @ x, atol=1e-12)
    # the order matters: the reversed product differs
    assert np.abs(E1 @ E2 @ x - E2 @ E1 @ x).max() > 1e-6


@pytest.mark.parametrize("smoother", ["l1jacobi", "gs"])
def test_bootstrap_symmetric_product_is_a_selfadjoint_contraction(smoother):
    """With SPD V-cycles (l1-Jacobi, or forward/backward Gauss-Seidel) each
    I - B_k A is A-self-adjoint with A-norm < 1, so the symmetrized product
    is A-self-adjoint with spectrum in [0, 1)."""
    A, Hs = _bootstrap_hierarchies()
    n = A.shape[0]
    E = np.stack([O.composite_error(Hs, A, e, symmetric=True, smoother=smoother) for e in np.eye(n)], axis=1)
    AE = A.toarray() @ E
    np.testing.assert_allclose(AE, AE.T, atol=1e-12 * np.abs(AE).max())
    lam = sla.eigh(AE, A.toarray(), eigvals_only=True)
    assert lam.min() > -1e-12 and lam.max() < 1.0


def test_bootstrap_rho_tends_to_the_largest_eigenvalue():
    """rho = (||x^nu||_A / ||x^0||_A)^(1/nu) is a power iteration on the
    symmetrized product: for large nu it approaches its largest eigenvalue."""
    A, Hs = _bootstrap_hierarchies()
    n = A.shape[0]
    E = np.stack([O.composite_error(Hs, A, e, symmetric=True) for e in np.eye(n)], axis=1)
    lam_max = sla.eigh(A.toarray() @ E, A.toarray(), eigvals_only=True).max()
    x0 = np.random.default_rng(8).standard_normal(n)
    x100, rho100 = O.bootstrap_test(Hs, A, x0, nu=100, symmetric=True)
    _, rho = O.bootstrap_test(Hs, A, x100, nu=100, symmetric=True)  # from an already aligned start
    assert abs(rho[0] - lam_max) <= 5e-3 * lam_max
    assert rho100[0] <= lam_max * (1 + 1e-12)  # no A-norm reduction factor exceeds the spectral radius
    _, rho1 = O.bootstrap_test(Hs, A, x0, nu=1, symmetric=True)
    np.testing.assert_allclose(rho1[0], O.a_norm(A, E @ x0)[0] / O.a_norm(A, x0)[0], rtol=1e-12)


def test_bootstrap_kcycle_composite_is_homogeneous_and_contracts():
    """With the paper's Gauss-Seidel K-cycles the composite operator is no
    longer linear, but it stays positively homogeneous, and on these stages
    it reduces the A-norm (the K-cycle approximates A^{-1} better than the
    V-cycle: its reduction is the smaller)."""
    A, Hs = _bootstrap_hierarchies(16)
    x = np.random.default_rng(9).standard_normal(A.shape[0])
    Ek = O.composite_error(Hs, A, x, smoother="gs", kind="K")
    np.testing.assert_allclose(O.composite_error(Hs, A, 2.5 * x, smoother="gs", kind="K"), 2.5 * Ek, rtol=1e-12)
    Ev = O.composite_error(Hs, A, x, smoother="gs", kind="V")
    assert O.a_norm(A, Ek)[0] < O.a_norm(A, Ev)[0] < O.a_norm(A, x)[0]
    _, rho = O.bootstrap_test(Hs, A, x, nu=3, smoother="gs", kind="K")
    assert 0.0 < rho[0] < 1.0


def test_bootstrap_one_level_stage_annihilates():
    """A one-level hierarchy solves exactly (B = A^{-1}): I - B A = 0."""
    A = problems.poisson5(8)
    H = O.setup(A, [], [64], np.ones((64, 1)))
    x0 = np.random.default_rng(2).standard_normal((64, 2))
    x, rho = O.bootstrap_test([H], A, x0, nu=3)
    assert np.abs(x).max() <= 1e-12 * np.abs(x0).max()
    assert np.all(rho <= 1e-10)


def test_bootstrap_driver_stages():
    """Stage r builds B_r from w_{r-1}, tests B_1..B_r on starts[r-1] and
    stores w_r = x^nu / ||x^nu||_A."""
    A = problems.poisson5(12)
    n = A.shape[0]
    agg = lambda w: aggregation.aggregate_hierarchy(A, w, [2, 2])
    starts = [np.random.default_rng(30 + r).standard_normal(n) for r in range(2)]
    W, rhos = O.bootstrap(A, np.ones(n), 3, 5, agg, starts)
    np.testing.assert_allclose(O.a_norm(A, W[:, 1:]), 1.0, rtol=1e-12)
    aggs, nn = agg(np.ones(n))
    H1 = O.setup(A, aggs, nn, np.full((n, 1), 1.0 / np.sqrt(n)))
    x1, r1 = O.bootstrap_test([H1], A, starts[0], 5)
    np.testing.assert_allclose(W[:, 1], x1 / O.a_norm(A, x1)[0], atol=1e-12)
    assert rhos[0] == pytest.approx(r1[0], rel=1e-12)
    assert 0.0 < rhos[1] < 1.0
