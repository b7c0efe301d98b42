"""Host-side input generation: operators and compatible-matching aggregation."""
import numpy as np
import pytest

from paper_1907_04417_gb300.hostsetup import aggregation, inputs, problems


def _greedy_bruteforce(n, i, j, c):
    mate = -np.ones(n, dtype=np.int64)
    for _, a, b in sorted(zip(-c[c > 0], i[c > 0], j[c > 0])):
        if mate[a] < 0 and mate[b] < 0:
            mate[a], mate[b] = b, a
    return mate


@pytest.mark.parametrize("seed", range(8))
def test_matching_equals_sequential_greedy(seed):
    rng = np.random.default_rng(seed)
    A = problems.aniso9(9) if seed % 2 else problems.elasticity(3)
    w = 1 + 0.5 * rng.standard_normal(A.shape[0])
    i, j, c = aggregation.matching_weights(A, w)
    assert np.array_equal(aggregation.greedy_matching(A.shape[0], i, j, c),
                          _greedy_bruteforce(A.shape[0], i, j, c))


def test_matching_weight_is_fine_diagonal():
    """c_ij equals (w_e^perp)^T A_e w_e^perp / (w_e^perp)^T D_e w_e^perp for
    the local vectors of Eq. (vector w_e)."""
    A = problems.aniso9(5)
    w = np.random.default_rng(1).uniform(0.5, 1.5, 25)
    i, j, c = aggregation.matching_weights(A, w)
    Ad = A.toarray()
    for e in range(len(i)):
        a, b = i[e], j[e]
        Ae = Ad[np.ix_([a, b], [a, b])]
        De = np.diag(np.diag(Ae))
        v = np.array([-w[b] / Ae[0, 0], w[a] / Ae[1, 1]])
        assert c[e] == pytest.approx((v @ Ae @ v) / (v @ De @ v), rel=1e-12)


def test_pairwise_prolongator_properties():
    A = problems.poisson5(8)
    w = np.random.default_rng(2).uniform(0.5, 1.5, 64)
    agg, Ac, wc = aggregation.pairwise_step(A, w)
    sizes = np.bincount(agg)
    assert sizes.max() <= 2
    # w is in the range of P_c: w = P_c w_c
    P = np.zeros((64, sizes.size))
    for a in range(sizes.size):
        idx = np.flatnonzero(agg == a)
        P[idx, a] = w[idx] / np.linalg.norm(w[idx])
    np.testing.assert_allclose(P @ wc, w, rtol=1e-14)


@pytest.mark.parametrize("N,fn,nnz", [(16, problems.poisson5, lambda N: 5 * N * N - 4 * N),
                                      (16, problems.aniso9, lambda N: 9 * N * N - 12 * N + 4)])
def test_operator_nnz_2d(N, fn, nnz):
    A = fn(N)
    assert A.nnz == nnz(N)
    assert abs(A - A.T).max() == 0
    assert np.linalg.eigvalsh(A.toarray()).min() > 0


def test_operators_3d_and_cc():
    A, _ = problems.jump7(6, 3)
    assert A.nnz == 7 * 216 - 6 * 36
    for M in (A, problems.elasticity(5), problems.cc5(9, problems.lognormal_field(9))):
        D = M.toarray()
        assert np.abs(D - D.T).max() == 0
        assert np.linalg.eigvalsh(D).min() > 0
    assert problems.cc5(9, np.ones((9, 9))).nnz == 5 * 81 - 36


def test_workload_builders_nested_maps():
    for P in (inputs.poisson(16), inputs.anisotropic(32, levels=3), inputs.jumping3d(8, nrhs=2),
              inputs.elasticity_grid(5, nrhs=2, levels=3), inputs.diffusion_cc(16, nrhs=2)):
        assert P.A.indptr.dtype == np.int32 and P.A.indices.dtype == np.int32
        assert len(P.n_nodes) == len(P.aggs) + 1
        for k, a in enumerate(P.aggs):
            assert a.shape == (P.n_nodes[k],)
            assert np.array_equal(np.unique(a), np.arange(P.n_nodes[k + 1]))
        np.testing.assert_allclose(np.linalg.norm(P.W, axis=0), 1.0)


def test_elasticity_batch_same_depth():
    batch = inputs.elasticity_batch(n_sys=3, sides=(4, 5), nrhs=2, levels=3)
    assert len({P.levels for P in batch}) == 1


def test_merge_singletons_joins_strongest_neighbour():
    A = problems.cc5(12, problems.lognormal_field(12, 1.0, seed=9))
    n = A.shape[0]
    rng = np.random.default_rng(4)
    agg = np.arange(n) // 2
    single = rng.choice(n, 30, replace=False)
    agg = agg.astype(np.int64)
    agg[single] = n + np.arange(30)                 # thirty forced singletons
    _, agg = np.unique(agg, return_inverse=True)
    out = aggregation.merge_singletons(A, agg)
    size_in = np.bincount(agg)
    Ad = A.toarray()
    for v in range(n):
        if size_in[agg[v]] != 1:
            continue
        nb = [u for u in np.flatnonzero(Ad[v]) if u != v and size_in[agg[u]] > 1]
        if not nb:
            continue
        best = min(nb, key=lambda u: (-abs(Ad[v, u]), u))
        assert out[v] == out[best]
    # aggregates of size > 1 stay together and apart
    for a in np.flatnonzero(size_in > 1):
        assert len(set(out[agg == a])) == 1
    assert np.array_equal(np.unique(out), np.arange(out.max() + 1))
    first = [np.flatnonzero(out == a)[0] for a in range(out.max() + 1)]
    assert np.all(np.diff(first) > 0)


def test_aggregate_operator_galerkin():
    A = problems.poisson5(6)
    w = np.random.default_rng(3).uniform(0.5, 1.5, 36)
    agg = np.arange(36) // 4
    Ac, wc = aggregation.aggregate_operator(A, w, agg)
    P = np.zeros((36, 9))
    for a in range(9):
        idx = np.flatnonzero(agg == a)
        P[idx, a] = w[idx] / np.linalg.norm(w[idx])
    np.testing.assert_allclose(Ac.toarray(), P.T @ A.toarray() @ P, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(P @ wc, w, rtol=1e-13)


def test_cc_hierarchy_reaches_dense_limit():
    P = inputs.diffusion_cc(128, nrhs=1)
    assert 3 * P.n_nodes[-1] <= 1024 and len(P.n_nodes) <= 6


@pytest.mark.parametrize("N", [16])
def test_elasticity_spd_beyond_small_grids(N):
    """Symmetric ordering, no pivoting: every pivot of the LU factorisation of
    an SPD matrix is positive (a truncated cross stencil fails this at 16^3)."""
    import scipy.sparse.linalg as spla
    A = problems.elasticity(N)
    assert abs(A - A.T).max() == 0
    lu = spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    assert np.array_equal(lu.perm_r, lu.perm_c)
    assert lu.U.diagonal().min() > 0


def test_bootstrap_starts_and_stage_aggregator():
    A = problems.aniso9(16)
    s1 = inputs.bootstrap_starts(A.shape[0], 4)
    s2 = inputs.bootstrap_starts(A.shape[0], 4)
    assert len(s1) == 3 and all(np.array_equal(a, b) for a, b in zip(s1, s2))
    assert not np.array_equal(s1[0], s1[1])
    w = np.ones(A.shape[0])
    aggs, nn = inputs.stage_aggregator(A, [2, 2])(w)
    aggs2, nn2 = aggregation.aggregate_hierarchy(A, w, [2, 2])
    assert nn == nn2 and all(np.array_equal(a, b) for a, b in zip(aggs, aggs2))
