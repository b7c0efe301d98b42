"""Pins of the oracle's cycle variants (Section 5: forward/backward
Gauss-Seidel smoothing, K-cycles with two inner flexible-CG iterations)
against facts that do not re-type the oracle: the colouring computed in
Jones-Plassmann rounds,
closed forms on complete graphs, triangular solves of the permuted system,
Krylov and Galerkin minimisers, symmetry and homogeneity of the
preconditioners."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import aggregation, inputs, problems

MASK = (1 << 64) - 1


def _splitmix_int(i):
    z = (i + 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def _jones_plassmann(A):
    """Colouring in rounds (Jones & Plassmann 1993): in each round every
    uncoloured vertex whose higher-priority neighbours (larger
    (splitmix64(i), i)) are all coloured takes the smallest colour none of
    them holds.  A vertex's colour depends only on its higher-priority
    neighbours, so this gives the greedy colouring in priority order by
    another route (it is how the device computes it)."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    key = [(_splitmix_int(i), i) for i in range(n)]
    nbr = [[j for j in A.indices[A.indptr[v]:A.indptr[v + 1]] if j != v] for v in range(n)]
    higher = [[j for j in nbr[v] if key[j] > key[v]] for v in range(n)]
    colour = [-1] * n
    left = set(range(n))
    while left:
        ready = [v for v in left if all(colour[j] >= 0 for j in higher[v])]
        assert ready
        for v in ready:
            taken = {colour[j] for j in higher[v]}
            c = 0
            while c in taken:
                c += 1
            colour[v] = c
        left -= set(ready)
    return np.asarray(colour)


def _small_hierarchy(N=24, m=3, levels=3, prob="aniso", seed=0):
    A = problems.aniso9(N) if prob == "aniso" else problems.poisson5(N)
    rng = np.random.default_rng(seed)
    W = np.concatenate([np.ones((A.shape[0], 1)), rng.standard_normal((A.shape[0], m - 1))], axis=1)
    W /= np.linalg.norm(W, axis=0)
    aggs, n_nodes = aggregation.aggregate_hierarchy(A, W[:, 0], [2] * (levels - 1))
    return A, O.setup(A, aggs, n_nodes, W)


def _random_graph(n=300, p=0.03, seed=3):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=p, random_state=rng, format="csr")
    M = M + M.T + sp.eye(n)
    M.data[:] = 1.0
    return M.tocsr()


# ------------------------------------------------------------- colouring --

def test_splitmix64_matches_integer_definition():
    idx = np.array([0, 1, 2, 3, 12345, 2**31 - 1, 2**40 + 7], dtype=np.uint64)
    got = O.splitmix64(idx)
    for i, g in zip(idx.tolist(), got.tolist()):
        assert g == _splitmix_int(i)
    # a bijection of the state: no collisions on a range
    assert np.unique(O.splitmix64(np.arange(200000))).size == 200000


@pytest.mark.parametrize("which", ["poisson12", "aniso16", "coarse", "random"])
def test_colouring_equals_jones_plassmann_rounds(which):
    if which == "poisson12":
        A = problems.poisson5(12)
    elif which == "aniso16":
        A = problems.aniso9(16)
    elif which == "coarse":
        _, H = _small_hierarchy(16, 3, 3)
        A = H.levels[1].A
    else:
        A = _random_graph()
    np.testing.assert_array_equal(O.greedy_colouring(A), _jones_plassmann(A))


def test_colouring_complete_graph_closed_form():
    """On K_n every vertex sees all higher-priority vertices: its colour is
    the number of vertices ranked above it."""
    n = 40
    A = sp.csr_matrix(np.ones((n, n)))
    rank = O.priority_rank(n)
    np.testing.assert_array_equal(O.greedy_colouring(A), n - 1 - rank)


def test_colouring_valid_on_every_level():
    _, H = _small_hierarchy(64, 4, 4)
    for l in H.levels:
        A = l.A.tocoo()
        c = O.greedy_colouring(l.A)
        off = A.row != A.col
        assert np.all(c[A.row[off]] != c[A.col[off]])
        assert c.min() == 0
        # first fit: at most (max degree + 1) colours
        deg = np.diff(l.A.indptr).max()
        assert c.max() + 1 <= deg


# ------------------------------------------------------------ GS sweeps --

def _perm_split(A, colour, backward):
    n = A.shape[0]
    key = -colour if backward else colour
    pi = np.lexsort((np.arange(n), key))
    Ap = A[pi][:, pi].tocsr()
    return pi, Ap


@pytest.mark.parametrize("cols", [1, 3])
def test_gs_forward_is_lower_triangular_solve(cols):
    """A forward multicolour sweep is lexicographic GS on the system ordered
    colour by colour: u_new = (D + L)^{-1} (f - U u) in that order."""
    A = problems.aniso9(20)
    n = A.shape[0]
    rng = np.random.default_rng(5)
    f = rng.standard_normal((n, cols)).squeeze()
    u = rng.standard_normal((n, cols)).squeeze()
    colour = O.greedy_colouring(A)
    got = O.gs_sweep(A, A.diagonal(), colour, f, u)
    pi, Ap = _perm_split(A, colour, False)
    Lw = sp.tril(Ap, 0, format="csr")
    Us = sp.triu(Ap, 1, format="csr")
    want = np.empty_like(got)
    want[pi] = spla.spsolve_triangular(Lw, f[pi] - Us @ u[pi], lower=True)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_gs_backward_is_upper_triangular_solve():
    """A backward sweep visits the colours in reverse: in the colour-major
    order it is u_new = (D + U)^{-1} (f - L u)."""
    A = problems.poisson5(18)
    n = A.shape[0]
    rng = np.random.default_rng(6)
    f, u = rng.standard_normal(n), rng.standard_normal(n)
    colour = O.greedy_colouring(A)
    got = O.gs_sweep(A, A.diagonal(), colour, f, u, backward=True)
    pi, Ap = _perm_split(A, colour, False)
    Uw = sp.triu(Ap, 0, format="csr")
    Ls = sp.tril(Ap, -1, format="csr")
    want = np.empty_like(got)
    want[pi] = spla.spsolve_triangular(Uw, f[pi] - Ls @ u[pi], lower=False)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_gs_vcycle_is_symmetric():
    """Forward pre- and backward post-sweeps with Galerkin transfers and an
    exact coarse solve give a symmetric preconditioner: x.(B y) = y.(B x)."""
    A, H = _small_hierarchy(32, 3, 3)
    rng = np.random.default_rng(7)
    x, y = rng.standard_normal((2, A.shape[0]))
    for pre, post in [(1, 1), (2, 2)]:
        Bx = O.cycle(H, x, pre=pre, post=post, smoother="gs")
        By = O.cycle(H, y, pre=pre, post=post, smoother="gs")
        assert abs(x @ By - y @ Bx) <= 1e-12 * abs(x @ By)
    # a forward post-sweep would break it
    colour, dg = O.gs_data(H)[0]
    Bx1 = O.gs_sweep(A, dg, colour, x, np.zeros_like(x))
    By1 = O.gs_sweep(A, dg, colour, y, np.zeros_like(y))
    assert abs(x @ By1 - y @ Bx1) > 1e-6 * abs(x @ By1)


def test_gs_vcycle_jacobi_path_unchanged():
    """smoother l1jacobi, kind V is the V-cycle of ``vcycle``."""
    A, H = _small_hierarchy(24, 3, 3)
    f = np.random.default_rng(8).standard_normal((A.shape[0], 2))
    np.testing.assert_array_equal(O.cycle(H, f), O.vcycle(H, f))


# ---------------------------------------------------------------- FCG --

def _spd(n=60, seed=9):
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((n, n))
    return Q @ Q.T + n * np.eye(n)


def test_fcg_identity_is_two_step_cg():
    """With B = I two FCG steps are two CG steps: the A-norm minimiser over
    the Krylov space span{r, A r}."""
    A = _spd()
    r = np.random.default_rng(10).standard_normal(A.shape[0])
    e = O.fcg(A, r, lambda g: g.copy(), 2)
    V = np.stack([r, A @ r], axis=1)
    y = np.linalg.solve(V.T @ A @ V, V.T @ r)
    np.testing.assert_allclose(e, V @ y, rtol=1e-10)


def test_fcg_exact_preconditioner_and_zero_column():
    """B = A^{-1}: the first step is exact, the second has a zero residual
    and contributes nothing; a zero right-hand side column stays zero."""
    A = _spd()
    R = np.random.default_rng(11).standard_normal((A.shape[0], 2))
    R[:, 1] = 0.0
    e = O.fcg(A, R, lambda g: np.linalg.solve(A, g), 2)
    np.testing.assert_allclose(e[:, 0], np.linalg.solve(A, R[:, 0]), rtol=1e-10)
    assert np.all(e[:, 1] == 0.0)


def test_fcg_nonlinear_preconditioner_is_galerkin_projection():
    """For any (nonlinear) B, two FCG steps give the A-orthogonal projection
    of A^{-1} r onto span{c1, c2}, c1 = B(r), c2 = B(r - A e1), e1 the
    projection onto span{c1}."""
    A = _spd()
    n = A.shape[0]
    rng = np.random.default_rng(12)
    M = rng.standard_normal((n, n)) * 0.05 + np.eye(n)

    def B(g):
        return M @ g + 0.1 * np.tanh(g)

    r = rng.standard_normal(n)
    e = O.fcg(A, r, B, 2)
    c1 = B(r)
    e1 = (c1 @ r) / (c1 @ A @ c1) * c1
    c2 = B(r - A @ e1)
    V = np.stack([c1, c2], axis=1)
    y = np.linalg.solve(V.T @ A @ V, V.T @ r)
    np.testing.assert_allclose(e, V @ y, rtol=1e-9)


# ------------------------------------------------------------ K-cycle --

@pytest.mark.parametrize("smoother", ["l1jacobi", "gs"])
def test_kcycle_two_levels_is_vcycle(smoother):
    A, H = _small_hierarchy(24, 3, 2)
    f = np.random.default_rng(13).standard_normal(A.shape[0])
    np.testing.assert_array_equal(O.cycle(H, f, smoother=smoother, kind="K"),
                                  O.cycle(H, f, smoother=smoother, kind="V"))


def test_kcycle_homogeneous_not_additive():
    """The K-cycle is positively homogeneous (every FCG coefficient is a
    ratio of inner products) but not linear."""
    A, H = _small_hierarchy(32, 3, 4)
    rng = np.random.default_rng(14)
    f, g = rng.standard_normal((2, A.shape[0]))
    Bf = O.cycle(H, f, kind="K")
    np.testing.assert_allclose(O.cycle(H, 3.0 * f, kind="K"), 3.0 * Bf, rtol=1e-12)
    Bs = O.cycle(H, f + g, kind="K")
    Bg = O.cycle(H, g, kind="K")
    assert np.linalg.norm(Bs - Bf - Bg) > 1e-8 * np.linalg.norm(Bs)


def test_kcycle_columns_are_independent():
    A, H = _small_hierarchy(24, 3, 4)
    F = np.random.default_rng(15).standard_normal((A.shape[0], 3))
    F[:, 2] = 0.0
    Z = O.cycle(H, F, smoother="gs", kind="K")
    for c in range(2):
        np.testing.assert_allclose(Z[:, c], O.cycle(H, F[:, c], smoother="gs", kind="K"), rtol=1e-12, atol=1e-14)
    assert np.all(Z[:, 2] == 0.0)


def test_variant_iteration_ordering():
    """On the anisotropic problem, Gauss-Seidel smoothing and the K-cycle
    each cut the PCG iteration count of the l1-Jacobi V-cycle."""
    P = inputs.anisotropic(64, nrhs=1, levels=4)
    H = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    it = {}
    for sm in ("l1jacobi", "gs"):
        for kind in ("V", "K"):
            _, res = O.solve_variant(H, P.B[:, 0], smoother=sm, kind=kind)
            assert res[0].converged
            it[sm, kind] = res[0].iters
    assert it["gs", "V"] < it["l1jacobi", "V"]
    assert it["l1jacobi", "K"] < it["l1jacobi", "V"]
    assert it["gs", "K"] < it["gs", "V"]


def test_gs_sweep_on_a_coarse_level():
    """The triangular-solve identity on a Galerkin level, whose rows couple
    through dense aggregate blocks (many colours)."""
    _, H = _small_hierarchy(32, 4, 3)
    A = H.levels[1].A
    n = A.shape[0]
    rng = np.random.default_rng(16)
    f, u = rng.standard_normal((2, n))
    colour = O.greedy_colouring(A)
    assert colour.max() + 1 >= 8
    got = O.gs_sweep(A, A.diagonal(), colour, f, u)
    pi, Ap = _perm_split(A, colour, False)
    want = np.empty_like(got)
    want[pi] = spla.spsolve_triangular(sp.tril(Ap, 0, format="csr"), f[pi] - sp.triu(Ap, 1) @ u[pi], lower=True)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("sm,kind", [("gs", "V"), ("l1jacobi", "K"), ("gs", "K")])
def test_variant_pcg_reaches_the_direct_solution(sm, kind):
    """PCG with each variant stops at the 1e-8 recursive residual; the true
    residual agrees and the error against a direct solve is within the
    condition number's allowance."""
    P = inputs.anisotropic(48, nrhs=1, levels=4)
    H = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    b = P.B[:, 0]
    x, res = O.solve_variant(H, b, smoother=sm, kind=kind)
    assert res[0].converged
    assert np.linalg.norm(b - P.A @ x) <= 1.5e-8 * np.linalg.norm(b)
    xd = spla.spsolve(P.A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-4 * np.linalg.norm(xd)
