"""The double-float q = A p reading the level-0 values as (hi, lo) pairs.

The paired read only changes how val_hi and val_lo reach the registers (one
8-byte load per non-zero instead of two 4-byte loads), so the solve must be
bit for bit the one without it.  AMG_Q_PAIRED=1 forces the paired read (on
an unstaged launch), =0 forbids it.  Both float32-cycle solves of the same
block replay one tuning cache, so that every other launch choice (and with
it every rounding order) is the same; they must agree exactly in every
column's iterate and iteration count, and reach the 1e-8 true residual.
"""
import numpy as np
import pytest

from paper_1907_04417_gb300.hostsetup import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import torch  # noqa: F401
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


@pytest.mark.parametrize("mk", [lambda: inputs.anisotropic(128, nrhs=1, levels=4),
                                lambda: inputs.jumping3d(16, nrhs=1, max_coarse=256)])
def test_paired_values_bitwise(amg, monkeypatch, tmp_path, mk):
    P = mk()
    B = np.random.default_rng(23).uniform(-1.0, 1.0, (P.n, 32))
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("AMG_Q_PAIRED", mode)
        monkeypatch.setenv("AMG_TUNE_CACHE", str(tmp_path / "tune.txt"))
        H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
        X, info, st = H.solve(B, options=amg.opts(cycle_precision=32))
        H.close()
        assert st == amg.AMG_OK
        out[mode] = (np.asarray(X), [i["iters"] for i in info])
    X0, it0 = out["0"]
    X1, it1 = out["1"]
    assert it0 == it1
    assert np.array_equal(X0, X1)
    tr = np.linalg.norm(B - P.A @ X1, axis=0) / np.linalg.norm(B, axis=0)
    assert tr.max() <= 1.1e-8
