"""Coarsening based on compatible weighted matching (Section 3), host side.

This is the one-off host step that turns (A, w) into the nested aggregate
maps the multiple-vector hierarchy is built on (Section 4, Eq. (aggs) and
Eq. (binmat)).  Its output is input data for both the GPU library and the
oracle; it performs none of the solve-phase arithmetic.

Steps, each in the paper's order:

* edge weights: the diagonal entry of A_f = P_f^T A P_f for a matched edge
  e = (i, j), built from the local vectors w_e and w_e^perp of Eq. (vector
  w_e), scaled by its D-norm, gives
      c_ij = 1 - 2 a_ij w_i w_j / (a_ii w_i^2 + a_jj w_j^2)
  (Section 3 chooses the matching that maximises the product of these
  diagonal entries);
* matching: the maximum product matching is approximated by the greedy
  matching on the strict order (c desc, min index asc, max index asc);
  it is computed as a locally-dominant matching, which yields the same
  result as the sequential greedy sweep for a strict order.  Only edges
  with c_ij > 0 take part; unmatched vertices become singletons;
* pairwise prolongator P_c of Eq. (prol): one column per pair,
  [w_i, w_j] / sqrt(w_i^2 + w_j^2), and w_k/|w_k| for a singleton;
* the next pairwise level uses A_c = P_c^T A P_c and w_c = P_c^T w;
* aggressive coarsening composes s consecutive pairwise steps into one
  aggregate map (Section 3, last paragraph; Section 5 composes several
  pairwise prolongators of the bootstrap hierarchy).

The greedy matching is a 1/2-approximation of the paper's (auction-based)
maximum product matching.  On the sparse, tree-like graphs of deep coarse
levels it leaves many vertices unmatched, so a level whose composed steps
shrink the node count by less than half of 2^s may be completed by
``merge_singletons``: every aggregate made of a single node joins the
aggregate of its most strongly coupled neighbour.  ``aggregate_operator``
then forms the next level's graph with the w-weighted piecewise-constant
prolongator (the pairwise P_c of Eq. (prol) extended to larger aggregates).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def matching_weights(A: sp.csr_matrix, w: np.ndarray):
    """Edge list (i < j) of A's graph with the compatible weights c_ij."""
    C = sp.triu(A, k=1, format="coo")
    i = C.row.astype(np.int64)
    j = C.col.astype(np.int64)
    a = C.data
    d = A.diagonal()
    den = d[i] * w[i] * w[i] + d[j] * w[j] * w[j]
    c = np.zeros_like(a)
    ok = den > 0
    c[ok] = 1.0 - 2.0 * a[ok] * w[i[ok]] * w[j[ok]] / den[ok]
    return i, j, c


def greedy_matching(n: int, i: np.ndarray, j: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Greedy matching on the strict edge order (c desc, i asc, j asc), i < j.

    Returns ``mate`` with mate[v] = partner or -1 for unmatched vertices."""
    keep = c > 0
    i, j, c = i[keep], j[keep], c[keep]
    mate = np.full(n, -1, dtype=np.int64)
    if i.size == 0:
        return mate
    order = np.lexsort((j, i, -c))
    rank = np.empty(order.size, dtype=np.int64)
    rank[order] = np.arange(order.size)
    ends = np.concatenate([i, j])
    other = np.concatenate([j, i])
    er = np.concatenate([rank, rank])
    o = np.lexsort((er, ends))
    ends, other = ends[o], other[o]
    start = np.searchsorted(ends, np.arange(n + 1))
    ptr = start[:-1].copy()
    end = start[1:]
    while True:
        # advance each free vertex past incident edges whose other end is taken
        live = np.flatnonzero((mate < 0) & (ptr < end))
        while live.size:
            stale = live[mate[other[ptr[live]]] >= 0]
            ptr[stale] += 1
            live = stale[ptr[stale] < end[stale]]
        v = np.flatnonzero((mate < 0) & (ptr < end))
        if v.size == 0:
            break
        u = other[ptr[v]]
        mutual = (ptr[u] < end[u]) & (other[np.minimum(ptr[u], other.size - 1)] == v) & (v < u)
        vv, uu = v[mutual], u[mutual]
        if vv.size == 0:  # cannot happen for a strict order; guard anyway
            break
        mate[vv] = uu
        mate[uu] = vv
    return mate


def pairwise_step(A: sp.csr_matrix, w: np.ndarray):
    """One pairwise aggregation step.  Returns (agg, A_c, w_c) where agg maps
    each vertex to its pair/singleton index (numbered by smallest member)."""
    n = A.shape[0]
    i, j, c = matching_weights(A, w)
    mate = greedy_matching(n, i, j, c)
    v = np.arange(n)
    rep = np.where(mate >= 0, np.minimum(v, mate), v)
    reps, agg = np.unique(rep, return_inverse=True)
    nc = reps.size
    norm = np.sqrt(np.bincount(agg, weights=w * w, minlength=nc))
    vals = np.empty(n)
    ok = norm[agg] > 0
    vals[ok] = w[ok] / norm[agg][ok]
    single = (mate < 0)
    # singleton: w_k/|w_k| (1 when w_k == 0); zero pair: equal weights
    vals[single] = np.where(w[single] < 0, -1.0, 1.0)
    zero_pair = (~single) & (~ok)
    vals[zero_pair] = np.sqrt(0.5)
    P = sp.csr_matrix((vals, (v, agg)), shape=(n, nc))
    Ac = (P.T @ A @ P).tocsr()
    Ac.sort_indices()
    wc = P.T @ w
    return agg.astype(np.int64), Ac, wc


def aggregate_hierarchy(A: sp.csr_matrix, w: np.ndarray, steps_per_level, min_nodes: int = 1):
    """Compose pairwise steps into nested aggregate maps.

    ``steps_per_level[k]`` pairwise steps form the level-(k+1) aggregates of
    the level-k nodes.  Returns (aggs, n_nodes) with aggs[k][node] = level-
    (k+1) aggregate, n_nodes[k] = number of level-k nodes (n_nodes[0] = n)."""
    aggs = []
    n_nodes = [A.shape[0]]
    Ak, wk = A, np.asarray(w, dtype=np.float64)
    for s in steps_per_level:
        comp = np.arange(Ak.shape[0])
        for _ in range(s):
            if Ak.shape[0] <= min_nodes:
                break
            agg, Ak, wk = pairwise_step(Ak, wk)
            comp = agg[comp]
        aggs.append(comp.astype(np.int32))
        n_nodes.append(int(Ak.shape[0]))
    return aggs, n_nodes


def merge_singletons(A: sp.csr_matrix, agg: np.ndarray) -> np.ndarray:
    """Attach each single-node aggregate to the aggregate of its neighbour
    with the largest |a_ij| (ties: lowest index); renumber by first member."""
    agg = np.asarray(agg, dtype=np.int64).copy()
    n = A.shape[0]
    size = np.bincount(agg)
    C = sp.coo_matrix(A)
    off = C.row != C.col
    r, c, v = C.row[off], C.col[off], np.abs(C.data[off])
    single = size[agg] == 1
    cand = single[r] & ~single[c]
    r, c, v = r[cand], c[cand], v[cand]
    if r.size:
        order = np.lexsort((c, -v, r))
        r, c = r[order], c[order]
        first = np.unique(r, return_index=True)[1]
        agg[r[first]] = agg[c[first]]
    _, agg = np.unique(agg, return_inverse=True)
    # renumber by smallest member so the map is canonical
    first_member = np.full(agg.max() + 1, n, dtype=np.int64)
    np.minimum.at(first_member, agg, np.arange(n))
    rank = np.empty_like(first_member)
    rank[np.argsort(first_member, kind="stable")] = np.arange(first_member.size)
    return rank[agg]


def aggregate_operator(A: sp.csr_matrix, w: np.ndarray, agg: np.ndarray):
    """A_c = P^T A P and w_c = P^T w for the w-weighted piecewise-constant
    prolongator of the aggregates ``agg``."""
    n = A.shape[0]
    nc = int(agg.max()) + 1
    norm = np.sqrt(np.bincount(agg, weights=w * w, minlength=nc))
    vals = np.where(norm[agg] > 0, w / np.where(norm[agg] > 0, norm[agg], 1.0), 1.0)
    P = sp.csr_matrix((vals, (np.arange(n), agg)), shape=(n, nc))
    Ac = (P.T @ A @ P).tocsr()
    Ac.sort_indices()
    return Ac, P.T @ w
