"""Pins of the oracle's compatible weighted matching (Section 3) against
facts that do not re-type it:

* the weight c_ij is the diagonal entry of A_f built from the local vectors
  w_e, w_e^perp of Eq. (vector w_e) (2 x 2 products, not the closed form);
* the greedy matching is the lexicographically first maximal matching in
  the strict edge order (found by enumerating every matching of tiny
  graphs), and it carries at least half the weight of a maximum weight
  matching (the greedy bound, against brute force);
* the prolongator of Eq. (prol) has orthonormal columns, holds w in its
  range, is D-orthogonal to the complement P_f built from w_e^perp, and its
  aggregates are the matched pairs and the singletons, numbered by smallest
  member;
* A_c equals the dense product P_c^T A P_c;
* the composed maps of several steps are the products of the step maps.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import problems


def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    M = np.triu(rng.random((n, n)) < p, 1)
    M = M | M.T
    A = -rng.uniform(0.2, 1.0, (n, n)) * M
    A = (A + A.T) / 2
    A[np.arange(n), np.arange(n)] = np.abs(A).sum(axis=1) + rng.uniform(0.1, 1.0, n)
    return sp.csr_matrix(A)


def test_weight_is_fine_diagonal_of_local_vectors():
    """c_ij = (w_e^perp)^T A_e w_e^perp / (w_e^perp)^T D_e w_e^perp with
    w_e^perp = [-w_j / a_ii, w_i / a_jj] (Eq. (vector w_e)); the scale of
    w_e^perp cancels."""
    rng = np.random.default_rng(4)
    for A in (problems.aniso9(6), problems.elasticity(3), _random_graph(30, 0.2, 1)):
        A = sp.csr_matrix(A)
        n = A.shape[0]
        w = rng.uniform(-1.5, 1.5, n)
        Ad = A.toarray()
        edges = O.matching_edges(A, w)
        assert len(edges) == (np.count_nonzero(Ad) - n) // 2
        for i, j, c in edges:
            assert i < j and Ad[i, j] != 0
            Ae = Ad[np.ix_([i, j], [i, j])]
            De = np.diag(np.diag(Ae))
            v = np.array([-w[j] / Ae[0, 0], w[i] / Ae[1, 1]])
            we = np.array([w[i], w[j]])
            assert abs(we @ De @ v) <= 1e-14 * np.abs(we).max() * np.abs(v).max() * Ae.max()
            assert c == pytest.approx((v @ Ae @ v) / (v @ De @ v), rel=1e-12, abs=1e-14)


def test_weight_special_cases():
    # w = 1 on a Laplacian edge: c = 1 - 2 a_ij / (a_ii + a_jj)
    assert O.matching_weight(2.0, 2.0, -1.0, 1.0, 1.0) == 1.5
    # w_i = 0: the local vector w_e^perp is [-w_j/a_ii, 0], c = 1
    assert O.matching_weight(2.0, 3.0, -1.0, 0.0, 1.0) == 1.0
    # both zero: no weight
    assert O.matching_weight(2.0, 3.0, -1.0, 0.0, 0.0) == 0.0


def _all_matchings(n, edges):
    """Every matching of the edge list (backtracking over edges)."""
    out = []

    def rec(k, used, chosen):
        if k == len(edges):
            out.append(list(chosen))
            return
        rec(k + 1, used, chosen)
        i, j, _ = edges[k]
        if i not in used and j not in used:
            chosen.append(k)
            rec(k + 1, used | {i, j}, chosen)
            chosen.pop()

    rec(0, frozenset(), [])
    return out


@pytest.mark.parametrize("seed", range(12))
def test_greedy_is_lexicographically_first_maximal_matching(seed):
    n = 7 + seed % 3
    A = _random_graph(n, 0.45, 100 + seed)
    rng = np.random.default_rng(seed)
    w = rng.uniform(-1.0, 1.0, n) if seed % 2 else np.ones(n)
    edges = [e for e in O.matching_edges(A, w) if e[2] > 0]
    order = sorted(range(len(edges)), key=lambda k: (-edges[k][2], edges[k][0], edges[k][1]))
    rank = {k: r for r, k in enumerate(order)}
    best = None
    best_w = 0.0
    for M in _all_matchings(n, edges):
        ends = {v for k in M for v in edges[k][:2]}
        maximal = all(i in ends or j in ends for i, j, _ in edges)
        key = sorted(rank[k] for k in M)
        if maximal and (best is None or key < best[0]):
            best = (key, M)
        best_w = max(best_w, sum(edges[k][2] for k in M))
    mate = O.greedy_matching(n, O.matching_edges(A, w))
    want = np.full(n, -1)
    for k in best[1]:
        i, j, _ = edges[k]
        want[i], want[j] = j, i
    np.testing.assert_array_equal(mate, want)
    got_w = sum(edges[k][2] for k in best[1])
    assert got_w >= 0.5 * best_w - 1e-12


def test_greedy_ties_fall_back_to_indices():
    """A path with equal weights: edges in index order, (0,1), (2,3), ..."""
    n = 9
    A = sp.diags([np.full(n - 1, -1.0), np.full(n, 2.0), np.full(n - 1, -1.0)], [-1, 0, 1], format="csr")
    mate = O.greedy_matching(n, O.matching_edges(A, np.ones(n)))
    np.testing.assert_array_equal(mate, [1, 0, 3, 2, 5, 4, 7, 6, -1])


def test_edges_with_nonpositive_weight_take_no_part():
    # a_ij > (a_ii + a_jj) / 2 with w_i = w_j = 1 drives c_ij below zero
    A = sp.csr_matrix(np.array([[1.0, 1.2, 0.0], [1.2, 1.0, -0.1], [0.0, -0.1, 1.0]]))
    edges = O.matching_edges(A, np.ones(3))
    assert edges[0][2] < 0 < edges[1][2]
    np.testing.assert_array_equal(O.greedy_matching(3, edges), [-1, 2, 1])


@pytest.mark.parametrize("which", ["poisson", "aniso", "random"])
def test_prolongator_of_eq_prol(which):
    rng = np.random.default_rng(7)
    A = {"poisson": problems.poisson5(9), "aniso": problems.aniso9(8),
         "random": _random_graph(40, 0.1, 3)}[which]
    A = sp.csr_matrix(A)
    n = A.shape[0]
    w = rng.uniform(-1.5, 1.5, n)
    w[3] = 0.0                    # a zero entry: a singleton of value 1 or a pair member
    agg, mate, P, Ac, wc = O.pairwise_step(A, w)
    Pd = P.toarray()
    # aggregates: the pairs and the singletons, numbered by smallest member
    for v in range(n):
        members = np.flatnonzero(agg == agg[v])
        assert set(members) == ({v, mate[v]} if mate[v] >= 0 else {v})
    first = [np.flatnonzero(agg == a).min() for a in range(agg.max() + 1)]
    assert first == sorted(first)
    # orthonormal columns, w in the range (w = P_c w_c), one entry per row
    np.testing.assert_allclose(Pd.T @ Pd, np.eye(Pd.shape[1]), atol=1e-15)
    np.testing.assert_allclose(Pd @ wc, w, atol=1e-15)
    assert np.all(np.diff(P.indptr) == 1)      # one stored entry per row (it may be 0)
    # P_c^T D P_f = 0 with P_f = blockdiag(w_e^perp) over the pairs
    D = A.diagonal()
    pairs = [(v, mate[v]) for v in range(n) if 0 <= v < mate[v]]
    Pf = np.zeros((n, len(pairs)))
    for e, (i, j) in enumerate(pairs):
        Pf[i, e], Pf[j, e] = -w[j] / D[i], w[i] / D[j]
    np.testing.assert_allclose(Pd.T @ (D[:, None] * Pf), 0.0, atol=1e-15)
    # A_c = P_c^T A P_c (dense)
    np.testing.assert_allclose(Ac.toarray(), Pd.T @ A.toarray() @ Pd, rtol=0, atol=1e-14)


def test_singleton_values():
    """Singletons take w_k / |w_k| (1 for w_k = 0); a pair of zeros 1/sqrt(2)."""
    w = np.array([-2.0, 0.0, 3.0, 0.0, 0.0])
    mate = np.array([-1, -1, -1, 4, 3])
    agg, P = O.pairwise_prolongator(w, mate)
    np.testing.assert_array_equal(agg, [0, 1, 2, 3, 3])
    np.testing.assert_allclose(P.toarray(), [[-1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0],
                                             [0, 0, 0, np.sqrt(0.5)], [0, 0, 0, np.sqrt(0.5)]])


def test_composed_maps_are_products_of_steps():
    A = problems.aniso9(24)
    w = np.random.default_rng(2).standard_normal(A.shape[0])
    aggs, n_nodes = O.aggregate_hierarchy(A, w, [2, 3])
    Ak, wk, maps = A, w, []
    for _ in range(5):
        agg, _, _, Ak, wk = O.pairwise_step(Ak, wk)
        maps.append(agg)
    np.testing.assert_array_equal(aggs[0], maps[1][maps[0]])
    np.testing.assert_array_equal(aggs[1], maps[4][maps[3][maps[2]]])
    assert n_nodes == [A.shape[0], maps[1].max() + 1, maps[4].max() + 1]
    assert np.bincount(aggs[0]).max() <= 4 and np.bincount(aggs[1]).max() <= 8
