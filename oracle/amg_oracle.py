"""FP64 CPU oracle for the single-hierarchy multiple-vector aggregation AMG
(D'Ambra & Vassilevski, "Improving Solve Time of Aggregation-based Adaptive
AMG") used as a CG preconditioner.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA library is checked against.  Only the test-suite, the smoke check and
the CPU-baseline leg of the benchmark may import it; the library never calls
it and has no CPU fallback.  It shares no code with the CUDA path.

Everything is float64, numpy/scipy, one aggregate at a time, in the order
the paper states the steps.  Readings of points the paper leaves open:

* W|_a is the plain row restriction of each smooth vector to the aggregate;
  the smooth vectors arrive with unit 2-norm, so the threshold
  TOL * size(a) / size(A) (Section 5) is compared with the singular values
  themselves, size(a) = rows of the aggregate at the current level,
  size(A) = order of the current-level matrix.
* At most min(n_a, m) columns can be kept.  If no singular value passes
  the threshold the leading left singular vector is still kept (an
  aggregate must own at least one coarse dof); if W vanishes on the
  aggregate that vector is the normalised constant.
* Signs: each kept column is flipped so that its entry of largest magnitude
  (lowest row on ties) is positive.  The preconditioner does not depend on
  these signs; they only fix P and A^k for comparison.
* Coarse dofs are numbered aggregate by aggregate in aggregate-index order,
  columns in descending singular-value order (the matrix Q of Section 4.1).
* The smoother is l1-Jacobi, M = diag(d), d_i = sum_j |a_ij|, one pre- and
  one post-sweep, no damping; the first pre-sweep from zero is u = f / d.
* The coarsest level is solved exactly by a dense Cholesky factorisation
  (the paper uses a sparse LU; the result is the same exact solve).
* PCG (Section 5): zero initial guess, stop when the recursive residual
  satisfies ||r||_2 <= rtol ||b||_2, Fletcher-Reeves beta.
* Cycle variants (Section 5 names K-cycles with two inner flexible-CG
  iterations and forward/backward Gauss-Seidel as the smoother of the
  bootstrap's hierarchies): Gauss-Seidel visits the rows colour by colour,
  the colours from a greedy colouring in decreasing priority
  (splitmix64(i), i) of the row index i in the numbering above (the paper's
  sweep is lexicographic); the inner flexible CG keeps one previous
  direction and always runs two iterations; a column whose step
  denominator is zero takes no step.  The outer PCG keeps the
  Fletcher-Reeves beta for the K-cycle too.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


# --------------------------------------------------------------------------
# setup (Section 4: Eq. (svd), the block prolongator, Galerkin, Section 4.1)
# --------------------------------------------------------------------------

def l1_diagonal(A: sp.csr_matrix) -> np.ndarray:
    """d_i = sum_j |a_ij| (the l1-Jacobi diagonal)."""
    return np.asarray(abs(A).sum(axis=1)).ravel()


def local_basis(Wa: np.ndarray, threshold: float):
    """Eq. (svd) for one aggregate: thin SVD of the local smooth-vector block
    P_a = [w_0|_a, ..., w_{nw}|_a] (n_a x m), keep the left singular vectors
    whose singular value exceeds ``threshold`` (Section 5, TOL rule).

    Returns (U_kept, sigma) with U_kept of shape (n_a, r_a)."""
    na = Wa.shape[0]
    U, S, _ = np.linalg.svd(Wa, full_matrices=False)
    r = int(np.count_nonzero(S > threshold))
    r = max(r, 1)
    U = U[:, :r].copy()
    if S[0] == 0.0:
        U[:, 0] = 1.0 / np.sqrt(na)
    for j in range(r):
        i = int(np.argmax(np.abs(U[:, j])))
        if U[i, j] < 0:
            U[:, j] = -U[:, j]
    return U, S


@dataclass
class Level:
    A: sp.csr_matrix
    d: np.ndarray = None                 # l1 diagonal (non-coarsest levels)
    P: sp.csr_matrix = None              # prolongator from this level to the previous one
    r: np.ndarray = None                 # kept columns per aggregate (coarse levels)
    owner: np.ndarray = None             # coarse dof -> aggregate (the matrix Q)
    sigma: list = field(default_factory=list)


@dataclass
class Hierarchy:
    levels: list
    chol: tuple = None

    @property
    def L(self):
        return len(self.levels)


def setup(A: sp.csr_matrix, aggs, n_nodes, W: np.ndarray, tol: float = 0.1) -> Hierarchy:
    """Build P^k and A^k = (P^k)^T A^{k-1} P^k for k = 1..L-1 (Section 4).

    aggs[k][i] is the level-(k+1) aggregate of level-k node i; the level-k
    dofs of node a are the coarse dofs generated by aggregate a (for k = 0,
    the dof itself), so the aggregate of dof i at level k is
    aggs[k][owner_k(i)] (the composite operator Q pi^{k+1} of Section 4.1)."""
    A = sp.csr_matrix(A, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    if W.ndim == 1:
        W = W[:, None]
    levels = [Level(A=A)]
    owner = np.arange(A.shape[0])
    Wk = W
    for k, agg in enumerate(aggs):
        Ak = levels[-1].A
        nprev = Ak.shape[0]
        nagg = int(n_nodes[k + 1])
        g = np.asarray(agg)[owner]
        order = np.argsort(g, kind="stable")
        counts = np.bincount(g, minlength=nagg)
        if counts.size != nagg or np.any(counts == 0):
            raise ValueError(f"level {k + 1}: empty or out-of-range aggregate")
        starts = np.concatenate([[0], np.cumsum(counts)])
        prow, pcol, pval, new_owner, rkept, sig = [], [], [], [], [], []
        col = 0
        for a in range(nagg):
            R = order[starts[a]:starts[a + 1]]
            U, S = local_basis(Wk[R], tol * R.size / nprev)
            r = U.shape[1]
            prow.append(np.repeat(R, r))
            pcol.append(np.tile(np.arange(col, col + r), R.size))
            pval.append(U.ravel())
            new_owner.append(np.full(r, a))
            rkept.append(r)
            sig.append(S)
            col += r
        P = sp.csr_matrix((np.concatenate(pval), (np.concatenate(prow), np.concatenate(pcol))),
                          shape=(nprev, col))
        Anext = (P.T @ Ak @ P).tocsr()
        Anext.sort_indices()
        Wk = P.T @ Wk
        owner = np.concatenate(new_owner)
        levels[-1].d = l1_diagonal(Ak)
        levels.append(Level(A=Anext, P=P, r=np.asarray(rkept), owner=owner, sigma=sig))
    Ac = levels[-1].A.toarray()
    try:
        cf = sla.cho_factor(Ac, lower=True)
    except np.linalg.LinAlgError as e:
        raise ValueError("coarsest matrix is not SPD") from e
    return Hierarchy(levels, cf)


# --------------------------------------------------------------------------
# solve: V-cycle (Section 5) and PCG (Section 5)
# --------------------------------------------------------------------------

def coarse_solve(H: Hierarchy, f):
    return sla.cho_solve(H.chol, f)


def vcycle(H: Hierarchy, f, k: int = 0, pre: int = 1, post: int = 1):
    """One V-cycle on level k for right-hand side f (vector or n x K)."""
    if k == H.L - 1:
        return coarse_solve(H, f)
    lev = H.levels[k]
    A = lev.A
    d = lev.d if np.ndim(f) == 1 else lev.d[:, None]
    u = f / d
    for _ in range(pre - 1):
        u = u + (f - A @ u) / d
    P = H.levels[k + 1].P
    fc = P.T @ (f - A @ u)
    u = u + P @ vcycle(H, fc, k + 1, pre, post)
    for _ in range(post):
        u = u + (f - A @ u) / d
    return u


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    relres: float
    converged: bool
    history: list


def pcg(A, b, precond=None, rtol: float = 1e-8, maxit: int = 1000, x0=None,
        fixed_iters: int | None = None) -> PCGResult:
    """Preconditioned CG for one right-hand side (Section 5).

    ``precond`` maps a residual to z = B r (None: B = I).  With
    ``fixed_iters`` the loop runs exactly that many iterations (used to
    compare iterates at equal iteration counts)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r)]
    if bn == 0.0:
        return PCGResult(np.zeros_like(b), 0, 0.0, True, hist)
    z = r if precond is None else precond(r)
    p = z.copy()
    rho = float(r @ z)
    it = 0
    limit = maxit if fixed_iters is None else fixed_iters
    converged = False
    while it < limit:
        it += 1
        q = A @ p
        alpha = rho / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rn = np.linalg.norm(r)
        hist.append(rn)
        if fixed_iters is None and rn <= rtol * bn:
            converged = True
            break
        z = r if precond is None else precond(r)
        rho_new = float(r @ z)
        beta = rho_new / rho
        rho = rho_new
        p = z + beta * p
    if fixed_iters is not None:
        converged = hist[-1] <= rtol * bn
    return PCGResult(x, it, hist[-1] / bn, converged, hist)


def solve(H: Hierarchy, b, rtol=1e-8, maxit=1000, fixed_iters=None):
    """AMG-PCG for every column of b (n or n x K); returns (X, results)."""
    A = H.levels[0].A
    B = np.asarray(b, dtype=np.float64)
    cols = B[:, None] if B.ndim == 1 else B
    res = [pcg(A, cols[:, c], lambda r: vcycle(H, r), rtol, maxit,
               fixed_iters=None if fixed_iters is None else int(np.broadcast_to(fixed_iters, cols.shape[1])[c]))
           for c in range(cols.shape[1])]
    X = np.stack([r.x for r in res], axis=1)
    return (X[:, 0] if B.ndim == 1 else X), res


# --------------------------------------------------------------------------
# adjoint: lambda = A^{-1} g (A SPD), dL/da_ij = -sum_b lambda_{b,i} x_{b,j}
# --------------------------------------------------------------------------

def adjoint(H: Hierarchy, g, x, rtol=1e-8, maxit=1000):
    """Returns (Lambda, grad_val, results): Lambda solves A Lambda = g by the
    same AMG-PCG, grad_val holds -sum_b Lambda[i, b] x[j, b] for every stored
    entry (i, j) of A, in A's CSR order."""
    A = H.levels[0].A
    Lam, res = solve(H, g, rtol, maxit)
    L2 = Lam[:, None] if Lam.ndim == 1 else Lam
    X2 = np.asarray(x, dtype=np.float64)
    X2 = X2[:, None] if X2.ndim == 1 else X2
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    grad = -np.sum(L2[rows] * X2[A.indices], axis=1)
    return Lam, grad, res


# --------------------------------------------------------------------------
# reported characteristics (Section 5: nl, opc, cr)
# --------------------------------------------------------------------------

def operator_complexity(H: Hierarchy) -> float:
    return sum(l.A.nnz for l in H.levels) / H.levels[0].A.nnz


def coarsening_ratio(H: Hierarchy) -> float:
    """Mean of n(A^{k-1}) / n(A^k) over the nl - 1 coarsening steps."""
    n = [l.A.shape[0] for l in H.levels]
    if len(n) < 2:
        return 1.0
    return float(np.mean([n[k - 1] / n[k] for k in range(1, len(n))]))


# --------------------------------------------------------------------------
# bootstrap (Algorithm 1, Section 2): the testing phase and the driver
# --------------------------------------------------------------------------

def composite_error(Hs, A, x, symmetric: bool = True, smoother: str = "l1jacobi", kind: str = "V"):
    """One application of the composite error operator of Algorithm 1 to x
    (vector or n x K).  With hierarchies H_1..H_r (B_k one cycle of H_k:
    the V-cycle with l1-Jacobi by default, or the ``cycle`` variant that
    smoother and kind select, e.g. the paper's Gauss-Seidel K-cycles) the
    plain product is E = (I - B_r A) ... (I - B_1 A), Eq. (comp_AMG): the
    rightmost factor acts first.  The symmetrized product of Section 5 (i)
    is (I - B_1 A) ... (I - B_r A) (I - B_r A) ... (I - B_1 A): factors
    1, 2, ..., r, then r, ..., 2, 1."""
    order = list(range(len(Hs)))
    seq = order + order[::-1] if symmetric else order
    v = np.array(x, dtype=np.float64)
    for k in seq:
        g = A @ v
        if smoother == "l1jacobi" and kind == "V":
            v = v - vcycle(Hs[k], g)
        else:
            v = v - cycle(Hs[k], g, smoother=smoother, kind=kind)
    return v


def a_norm(A, x):
    """||x||_A per column."""
    X = np.asarray(x, dtype=np.float64)
    X2 = X[:, None] if X.ndim == 1 else X
    return np.sqrt(np.einsum("ij,ij->j", X2, A @ X2))


def bootstrap_test(Hs, A, x0, nu: int, symmetric: bool = True, smoother: str = "l1jacobi", kind: str = "V"):
    """Testing phase of Algorithm 1: x^j = E x^{j-1}, j = 1..nu, from x^0 =
    x0.  Returns (x^nu, rho) with the convergence estimate rho =
    (||x^nu||_A / ||x^0||_A)^(1/nu) per column (the paper leaves the estimate
    unstated; this is the mean A-norm reduction per application)."""
    x = np.array(x0, dtype=np.float64)
    n0 = a_norm(A, x)
    for _ in range(nu):
        x = composite_error(Hs, A, x, symmetric, smoother, kind)
    n1 = a_norm(A, x)
    with np.errstate(divide="ignore", invalid="ignore"):
        rho = np.where(n0 > 0, (n1 / n0) ** (1.0 / nu), 0.0)
    return x, rho


def bootstrap(A, w0, m: int, nu: int, aggregate, starts, symmetric: bool = True, tol: float = 0.1,
              smoother: str = "l1jacobi", kind: str = "V"):
    """Algorithm 1 with maxstage = m - 1 and rho_des = 0 (the number of
    smooth vectors is fixed instead of the target rate).  Stage r = 1..m-1
    builds B_r from w_{r-1}: ``aggregate(w)`` gives the composed pairwise
    aggregates (aggs, n_nodes) of the weighted matching on w (Section 3), and
    the hierarchy holds the single smooth vector w (m = 1).  The testing
    phase applies the composite operator of B_1..B_r nu times to the random
    vector starts[r-1] and takes w_r = x^nu / ||x^nu||_A.  Returns (W, rhos)
    with W = [w_0, ..., w_{m-1}] (n x m) and the stage estimates rho."""
    n = A.shape[0]
    W = np.empty((n, m))
    W[:, 0] = w0
    Hs, rhos = [], []
    for r in range(1, m):
        w = W[:, r - 1]
        aggs, n_nodes = aggregate(w)
        Hs.append(setup(A, aggs, n_nodes, (w / np.linalg.norm(w))[:, None], tol))
        x, rho = bootstrap_test(Hs, A, starts[r - 1], nu, symmetric, smoother, kind)
        W[:, r] = x / a_norm(A, x)[0]
        rhos.append(float(rho[0]))
    return W, rhos


# --------------------------------------------------------------------------
# cycle variants (Section 5): forward/backward Gauss-Seidel smoothing, here
# in multicolour order, and the K-cycle with two inner flexible-CG
# iterations on every level but the coarsest
# --------------------------------------------------------------------------

def splitmix64(i):
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; Vigna's splitmix64.c)
    output for state i: the state plus the golden-ratio increment
    0x9e3779b97f4a7c15, then the finaliser z ^= z >> 30, z *= 0xbf58476d1ce4e5b9,
    z ^= z >> 27, z *= 0x94d049bb133111eb, z ^= z >> 31, all mod 2^64.
    Vectorised over integer arrays (uint64 result)."""
    z = np.atleast_1d(np.asarray(i)).astype(np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def priority_rank(n: int) -> np.ndarray:
    """rank[i] = position of vertex i in the increasing order of the keys
    (splitmix64(i), i); a larger rank is a higher priority."""
    idx = np.arange(n)
    order = np.lexsort((idx, splitmix64(idx)))
    rank = np.empty(n, dtype=np.int64)
    rank[order] = idx
    return rank


def greedy_colouring(A: sp.csr_matrix) -> np.ndarray:
    """Greedy colouring of the graph of A (its stored off-diagonal pattern),
    one vertex at a time in decreasing priority (splitmix64(i), i): every
    vertex takes the smallest colour that none of its already coloured
    neighbours holds (those are exactly its higher-priority neighbours)."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    rank = priority_rank(n)
    order = np.empty(n, dtype=np.int64)
    order[n - 1 - rank] = np.arange(n)          # order[0] = highest priority
    indptr = A.indptr.tolist()
    indices = A.indices.tolist()
    colour = [-1] * n
    for v in order.tolist():
        taken = set()
        for q in range(indptr[v], indptr[v + 1]):
            j = indices[q]
            if j != v and colour[j] >= 0:
                taken.add(colour[j])
        c = 0
        while c in taken:
            c += 1
        colour[v] = c
    return np.asarray(colour, dtype=np.int64)


def gs_sweep(A: sp.csr_matrix, diag, colour, f, u, backward: bool = False):
    """One multicolour Gauss-Seidel sweep: colours in increasing order
    (forward) or decreasing order (backward); within a colour every row i
    becomes u_i + (f_i - (A u)_i) / a_ii with the current u (rows of one
    colour share no edge, so their order is immaterial)."""
    u = np.array(u, dtype=np.float64)
    d = diag if np.ndim(f) == 1 else diag[:, None]
    ncol = int(colour.max()) + 1 if colour.size else 0
    seq = range(ncol - 1, -1, -1) if backward else range(ncol)
    for c in seq:
        S = np.flatnonzero(colour == c)
        u[S] = u[S] + (f[S] - A[S] @ u) / d[S]
    return u


def gs_data(H: Hierarchy):
    """Colours and diagonals of the smoothed levels (cached on H)."""
    if getattr(H, "_gs", None) is None:
        H._gs = [(greedy_colouring(l.A), l.A.diagonal().copy()) for l in H.levels[:-1]]
    return H._gs


def _cdot(x, y):
    """Column-wise inner products (a scalar for vectors)."""
    return np.sum(x * y, axis=0)


def fcg(A, r, precond, iters: int = 2):
    """Flexible CG (Notay 2000) on A e = r from e = 0, each new direction
    A-orthogonalised against the previous one only, ``iters`` iterations.
    Columns of r are independent problems.  A zero denominator (a column
    that has already converged exactly) contributes no step."""
    r = np.array(r, dtype=np.float64)
    e = np.zeros_like(r)
    d_prev = Ad_prev = dAd_prev = None
    for _ in range(iters):
        c = precond(r)
        Ac = A @ c
        d, Ad = c, Ac
        if d_prev is not None:
            with np.errstate(divide="ignore", invalid="ignore"):
                g = np.where(dAd_prev > 0, _cdot(c, Ad_prev) / dAd_prev, 0.0)
            d = c - g * d_prev
            Ad = Ac - g * Ad_prev
        dAd = _cdot(d, Ad)
        with np.errstate(divide="ignore", invalid="ignore"):
            alpha = np.where(dAd > 0, _cdot(d, r) / dAd, 0.0)
        e = e + alpha * d
        r = r - alpha * Ad
        d_prev, Ad_prev, dAd_prev = d, Ad, dAd
    return e


def cycle(H: Hierarchy, f, k: int = 0, pre: int = 1, post: int = 1,
          smoother: str = "l1jacobi", kind: str = "V"):
    """One multigrid cycle on level k (Section 5 variants).

    smoother "l1jacobi": the V-cycle smoother above (first sweep from zero
    u = f / d).  smoother "gs": u starts at zero, ``pre`` forward multicolour
    Gauss-Seidel sweeps before the coarse correction and ``post`` backward
    sweeps after it (forward/backward GS as pre-/post-smoother, which keeps
    the preconditioner symmetric).

    kind "V": the coarse correction is one cycle on level k+1.  kind "K":
    on every level k+1 but the coarsest the correction is two flexible-CG
    iterations on A^{k+1} e = P^T (f - A u), each preconditioned by one
    cycle on level k+1 (the K-cycle, a nonlinear AMLI cycle)."""
    if k == H.L - 1:
        return coarse_solve(H, f)
    A = H.levels[k].A
    P = H.levels[k + 1].P
    if smoother == "l1jacobi":
        d = H.levels[k].d if np.ndim(f) == 1 else H.levels[k].d[:, None]
        u = f / d
        for _ in range(pre - 1):
            u = u + (f - A @ u) / d
    elif smoother == "gs":
        colour, dg = gs_data(H)[k]
        u = np.zeros_like(np.asarray(f, dtype=np.float64))
        for _ in range(pre):
            u = gs_sweep(A, dg, colour, f, u)
    else:
        raise ValueError(smoother)
    fc = P.T @ (f - A @ u)
    inner = lambda g: cycle(H, g, k + 1, pre, post, smoother, kind)  # noqa: E731
    if kind == "K" and k + 1 < H.L - 1:
        e = fcg(H.levels[k + 1].A, fc, inner, 2)
    elif kind in ("V", "K"):
        e = inner(fc)
    else:
        raise ValueError(kind)
    u = u + P @ e
    for _ in range(post):
        if smoother == "l1jacobi":
            u = u + (f - A @ u) / d
        else:
            u = gs_sweep(A, dg, colour, f, u, backward=True)
    return u


def solve_variant(H: Hierarchy, b, rtol=1e-8, maxit=1000, fixed_iters=None, pre=1, post=1,
                  smoother="l1jacobi", kind="V"):
    """PCG (the same Fletcher-Reeves loop as ``solve``) preconditioned by one
    ``cycle`` per iteration; returns (X, results)."""
    A = H.levels[0].A
    B = np.asarray(b, dtype=np.float64)
    cols = B[:, None] if B.ndim == 1 else B
    pc = lambda r: cycle(H, r, 0, pre, post, smoother, kind)  # noqa: E731
    res = [pcg(A, cols[:, c], pc, rtol, maxit, fixed_iters=fixed_iters) for c in range(cols.shape[1])]
    X = np.stack([r.x for r in res], axis=1)
    return (X[:, 0] if B.ndim == 1 else X), res


# --------------------------------------------------------------------------
# compatible weighted matching (Section 3): one pairwise aggregation step
# --------------------------------------------------------------------------

def matching_weight(a_ii, a_jj, a_ij, w_i, w_j):
    """Edge weight of the compatible weighted matching for the edge (i, j):
    the diagonal entry of A_f = P_f^T A P_f that the D-orthogonal local
    vector w_e^perp of Eq. (vector w_e) produces, normalised by its D_e-norm,
        (w_e^perp)^T A_e w_e^perp / (w_e^perp)^T D_e w_e^perp
            = 1 - 2 a_ij w_i w_j / (a_ii w_i^2 + a_jj w_j^2).
    Section 3 asks for the matching that maximises the product of these
    entries.  The right-hand form is evaluated in float64, one rounded
    operation at a time, left to right: den = a_ii w_i w_i + a_jj w_j w_j,
    then 1 - (2 a_ij w_i w_j) / den.  A non-positive denominator gives 0
    (the edge takes no part)."""
    den = a_ii * w_i * w_i + a_jj * w_j * w_j
    if not den > 0.0:
        return 0.0
    return 1.0 - 2.0 * a_ij * w_i * w_j / den


def matching_edges(A: sp.csr_matrix, w):
    """The edges (i, j), i < j, of the graph of A (its stored upper entries,
    row by row) with their weights c_ij."""
    A = sp.csr_matrix(A)
    diag = A.diagonal()
    w = [float(v) for v in np.asarray(w, dtype=np.float64)]
    edges = []
    for i in range(A.shape[0]):
        for q in range(A.indptr[i], A.indptr[i + 1]):
            j = int(A.indices[q])
            if j > i:
                c = matching_weight(float(diag[i]), float(diag[j]), float(A.data[q]), w[i], w[j])
                edges.append((i, j, c))
    return edges


def greedy_matching(n: int, edges):
    """The matching of one pairwise step: the edges with c_ij > 0 are visited
    one at a time in the strict order (c_ij descending, then i, then j) and an
    edge joins the matching when neither end is matched yet.  This greedy
    matching stands in for the maximum product matching of Section 3 (it is a
    1/2-approximation of the maximum weight matching).  Returns mate[v], the
    partner of v or -1."""
    mate = np.full(n, -1, dtype=np.int64)
    for i, j, c in sorted((e for e in edges if e[2] > 0.0), key=lambda e: (-e[2], e[0], e[1])):
        if mate[i] < 0 and mate[j] < 0:
            mate[i] = j
            mate[j] = i
    return mate


def pairwise_prolongator(w, mate):
    """Eq. (prol): the aggregates of one pairwise step and the prolongator
    P_c with one column per aggregate.  Each pair {i, j} and each unmatched
    vertex k is an aggregate; the aggregates are numbered by their smallest
    member, in increasing order (the paper lists pairs before singletons;
    the numbering does not change the coarse space).  Column values: the
    local vector w_e = [w_i, w_j] / sqrt(w_i^2 + w_j^2) of Eq. (vector w_e)
    for a pair, w_k / |w_k| for a singleton (the matrix W of Eq. (prol)).
    Where the paper's formula divides by zero: a singleton with w_k = 0 takes
    1, a pair with w_i = w_j = 0 takes equal weights 1/sqrt(2).
    Returns (agg, P_c) with agg[v] the aggregate of v."""
    w = np.asarray(w, dtype=np.float64)
    n = w.size
    agg = np.full(n, -1, dtype=np.int64)
    na = 0
    for v in range(n):                       # smallest member first
        if agg[v] >= 0:
            continue
        agg[v] = na
        if mate[v] >= 0:
            agg[mate[v]] = na
        na += 1
    vals = np.empty(n)
    for v in range(n):
        u = mate[v]
        if u < 0:
            vals[v] = -1.0 if w[v] < 0 else 1.0
        else:
            nrm = np.sqrt(w[v] * w[v] + w[u] * w[u])
            vals[v] = w[v] / nrm if nrm > 0 else np.sqrt(0.5)
    P = sp.csr_matrix((vals, (np.arange(n), agg)), shape=(n, na))
    return agg, P


def pairwise_step(A: sp.csr_matrix, w):
    """One pairwise aggregation step of Section 3 on (A, w): weights,
    greedy matching, Eq. (prol), then the next graph A_c = P_c^T A P_c and
    the next vector w_c = P_c^T w (the coarse level the following step
    matches on).  Returns (agg, mate, P_c, A_c, w_c)."""
    A = sp.csr_matrix(A, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    mate = greedy_matching(A.shape[0], matching_edges(A, w))
    agg, P = pairwise_prolongator(w, mate)
    Ac = (P.T @ A @ P).tocsr()
    Ac.sort_indices()
    return agg, mate, P, Ac, P.T @ w


def aggregate_hierarchy(A: sp.csr_matrix, w, steps_per_level):
    """Aggressive coarsening (end of Section 3): steps_per_level[k]
    consecutive pairwise steps make the level-(k+1) aggregates of the
    level-k nodes; the composed map is the product of the pairwise maps.
    Returns (aggs, n_nodes) in the form ``setup`` takes."""
    aggs, n_nodes = [], [A.shape[0]]
    Ak, wk = sp.csr_matrix(A, dtype=np.float64), np.asarray(w, dtype=np.float64)
    for s in steps_per_level:
        comp = np.arange(Ak.shape[0])
        for _ in range(s):
            agg, _, _, Ak, wk = pairwise_step(Ak, wk)
            comp = agg[comp]
        aggs.append(comp.astype(np.int32))
        n_nodes.append(int(Ak.shape[0]))
    return aggs, n_nodes
