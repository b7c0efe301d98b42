"""GPU compatible weighted matching (Section 3) against the oracle, index
for index.

amg_pairwise_matching computes the edge weights c_ij on the device, with
every float64 operation rounded on its own, and the greedy matching on the
strict order (c desc, smaller end, larger end) as a locally-dominant
matching.  The oracle visits the edges one at a time in that order (its
matching is pinned against brute-force enumeration on tiny graphs); both
give the same partner for every vertex on the workloads' operators, with
smooth and random vectors, on irregular coarse graphs, and when every
weight ties.  The whole pairwise step and its composition are compared with
the oracle's Eq. (prol) step the same way.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import problems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import torch  # noqa: F401
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


def _oracle(A, w):
    return O.greedy_matching(A.shape[0], O.matching_edges(A, w)).astype(np.int32)


def _graphs():
    rng = np.random.default_rng(17)
    k = problems.lognormal_field(32, 1.0, seed=5)
    out = {
        "aniso9_64": problems.aniso9(64),
        "poisson5_50": problems.poisson5(50),
        "jump7_12": problems.jump7(12, 4, seed=3)[0],
        "elasticity_6": problems.elasticity(6),
        "cc5_32": problems.cc5(32, k),
    }
    A = problems.aniso9(48)
    Ac = O.pairwise_step(A, np.ones(A.shape[0]))[3]
    Ac2 = O.pairwise_step(Ac, rng.standard_normal(Ac.shape[0]))[3]
    out["aniso9_48_coarse2"] = Ac2
    return out


GRAPHS = list(_graphs())


@pytest.mark.parametrize("name", GRAPHS)
@pytest.mark.parametrize("wkind", ["ones", "random"])
def test_matching_matches_oracle(amg, name, wkind):
    A = sp.csr_matrix(_graphs()[name])
    A.sort_indices()
    n = A.shape[0]
    w = np.ones(n) if wkind == "ones" else np.random.default_rng(n).standard_normal(n)
    mate = amg.pairwise_matching(A, w)
    ref = _oracle(A, w)
    np.testing.assert_array_equal(mate, ref)
    m = mate >= 0
    assert np.all(mate[mate[m]] == np.flatnonzero(m))  # a matching: partners point back
    assert m.sum() > 0


def test_matching_all_weights_tie(amg):
    """A path graph with equal weights: the order falls back to the indices."""
    n = 9
    A = sp.diags([np.full(n - 1, -1.0), np.full(n, 2.0), np.full(n - 1, -1.0)], [-1, 0, 1], format="csr")
    w = np.ones(n)
    np.testing.assert_array_equal(amg.pairwise_matching(A, w), _oracle(A, w))


def test_matching_rejects_non_symmetric_pattern(amg):
    A = sp.csr_matrix(np.array([[2.0, -1.0, 0.0], [0.0, 2.0, -1.0], [0.0, -1.0, 2.0]]))
    with pytest.raises(amg.AMGError) as e:
        amg.pairwise_matching(A, np.ones(3))
    assert e.value.status == amg.AMG_ERR_INVALID_ARG


@pytest.mark.parametrize("name", GRAPHS)
@pytest.mark.parametrize("wkind", ["ones", "random"])
def test_pairwise_step_matches_oracle(amg, name, wkind):
    """One step from the same (A, w): aggregates and the coarse pattern index
    for index, A_c and w_c to rounding (the sums run in another order)."""
    A = sp.csr_matrix(_graphs()[name])
    A.sort_indices()
    n = A.shape[0]
    w = np.ones(n) if wkind == "ones" else np.random.default_rng(n + 1).standard_normal(n)
    agg, Ac, wc = amg.pairwise_step(A, w)
    agg_h, _, _, Ac_h, wc_h = O.pairwise_step(A, w)
    np.testing.assert_array_equal(agg, agg_h)
    np.testing.assert_array_equal(Ac.indptr, Ac_h.indptr)
    np.testing.assert_array_equal(Ac.indices, Ac_h.indices)
    np.testing.assert_allclose(Ac.data, Ac_h.data, rtol=1e-12, atol=1e-13 * np.abs(Ac_h.data).max())
    np.testing.assert_allclose(wc, wc_h, rtol=1e-13, atol=1e-14 * np.abs(wc_h).max())


def test_composed_steps_match_oracle(amg):
    """Four levels of composed steps entirely on the device (random vector, so
    no two edge weights tie) against the oracle's composition."""
    A = problems.aniso9(64)
    w = np.random.default_rng(9).standard_normal(A.shape[0])
    aggs, nn = amg.aggregate_hierarchy(A, w, [2, 2, 2])
    aggs_h, nn_h = O.aggregate_hierarchy(A, w, [2, 2, 2])
    assert nn == nn_h
    for a, b in zip(aggs, aggs_h):
        np.testing.assert_array_equal(a, b)
