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

def composite_error(Hs, A, x, symmetric: bool = True):
    """One application of the composite error operator of Algorithm 1 to x
    (vector or n x K).  With hierarchies H_1..H_r (B_k one V-cycle of H_k)
    the plain product is E = (I - B_r A) ... (I - B_1 A), Eq. (comp_AMG):
    the rightmost factor acts first.  The symmetrized product of Section 5
    (i) is (I - B_1 A) ... (I - B_r A) (I - B_r A) ... (I - B_1 A): factors
    1, 2, ..., r, then r, ..., 2, 1."""
    order = list(range(len(Hs)))
    seq = order + order[::-1] if symmetric else order
    v = np.array(x, dtype=np.float64)
    for k in seq:
        v = v - vcycle(Hs[k], A @ v)
    return v


def a_norm(A, x):
    """||x||_A per column."""
    X = np.asarray(x, dtype=np.float64)
    X2 = X[:, None] if X.ndim == 1 else X
    return np.sqrt(np.einsum("ij,ij->j", X2, A @ X2))


def bootstrap_test(Hs, A, x0, nu: int, symmetric: bool = True):
    """Testing phase of Algorithm 1: x^j = E x^{j-1}, j = 1..nu, from x^0 =
    x0.  Returns (x^nu, rho) with the convergence estimate rho =
    (||x^nu||_A / ||x^0||_A)^(1/nu) per column (the paper leaves the estimate
    unstated; this is the mean A-norm reduction per application)."""
    x = np.array(x0, dtype=np.float64)
    n0 = a_norm(A, x)
    for _ in range(nu):
        x = composite_error(Hs, A, x, symmetric)
    n1 = a_norm(A, x)
    with np.errstate(divide="ignore", invalid="ignore"):
        rho = np.where(n0 > 0, (n1 / n0) ** (1.0 / nu), 0.0)
    return x, rho


def bootstrap(A, w0, m: int, nu: int, aggregate, starts, symmetric: bool = True, tol: float = 0.1):
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
        x, rho = bootstrap_test(Hs, A, starts[r - 1], nu, symmetric)
        W[:, r] = x / a_norm(A, x)[0]
        rhos.append(float(rho[0]))
    return W, rhos
