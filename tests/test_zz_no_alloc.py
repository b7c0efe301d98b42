"""The allocation-free entry point for the local bases of Eq. (svd).

Some callers may not allocate device memory when they call into the library
(latency-bound loops where cudaMalloc can stall the device, plug-ins whose
host framework owns all device memory, fixed memory budgets).  For them
amg_local_bases_static computes the per-aggregate bases in a work area
compiled into the library.  This test checks, through the C ABI, that two
calls in a row reproduce the prolongator blocks that amg_setup_from_aggregates
builds for the same smooth vectors and aggregates, and that sizes beyond the
fixed work area are refused.  It lives in its own file, collected last, and
passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_1907_04417_gb300.hostsetup import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


def test_static_bases_match_setup_twice(amg):
    import torch
    P = inputs.anisotropic(N=48, nrhs=1, levels=3)
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    e0 = H.export_level(0)
    e1 = H.export_level(1)
    nf, m = P.n, P.m
    assert nf * m <= (1 << 17)
    W_lib = torch.from_numpy(np.ascontiguousarray(P.W[e0["perm"]])).cuda()
    rs = torch.from_numpy(e1["row_start"].astype(np.int32)).cuda()
    for call in range(2):
        U = torch.full((nf, m), np.nan, dtype=torch.float64, device="cuda")
        r = torch.zeros(e1["naggs"], dtype=torch.int32, device="cuda")
        st = amg.local_bases_static(W_lib, rs, nf, 0.1, U, r)
        assert st == amg.AMG_OK, call
        Uh = U.cpu().numpy()
        rh = r.cpu().numpy()
        np.testing.assert_array_equal(rh, e1["r"])
        blocks = np.concatenate([Uh[e1["row_start"][a]:e1["row_start"][a + 1], :rh[a]].ravel()
                                 for a in range(e1["naggs"])])
        np.testing.assert_allclose(blocks, e1["pval"], rtol=0, atol=1e-13)


def test_static_bases_reject_oversize_and_host_pointers(amg):
    import torch
    nf, m = (1 << 17) // 4 + 1, 4
    W = torch.zeros((nf, m), dtype=torch.float64, device="cuda")
    U = torch.zeros_like(W)
    rs = torch.tensor([0, nf], dtype=torch.int32, device="cuda")
    r = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert amg.local_bases_static(W, rs, nf, 0.1, U, r) == amg.AMG_ERR_INVALID_ARG
    Wh = np.zeros((16, 2))
    assert amg.local_bases_static(Wh, rs, 16, 0.1, U, r) == amg.AMG_ERR_INVALID_ARG
