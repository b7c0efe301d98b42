"""GPU parity of the grouped coarse-level kernels.

On a Galerkin level the coarse dofs of one aggregate share one column
pattern, so the grouped sweep and the grouped fused restriction gather each
neighbouring coarse row once per aggregate instead of once per row.  The
environment variable AMG_COARSE_KERNELS fixes the kernel choice that the
tuner makes when a hierarchy first solves with a given column count:
"grouped" takes the grouped kernels wherever a level allows them, "csr"
never does.  These tests force each choice, read the choices back from the
tuning cache, and check the solves against the FP64 oracle (iteration counts
within one, iterate at the GPU's count within 1e-10) and the float32 cycle
against the same true residual within three extra iterations.
"""
import numpy as np
import pytest

from oracle import amg_oracle as O
from paper_1907_04417_gb300.hostsetup import inputs

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "aniso64": lambda: inputs.anisotropic(64, nrhs=1, levels=4),     # r = 4 per aggregate
    "jump16": lambda: inputs.jumping3d(16, nrhs=1, max_coarse=256),  # r <= 3
    "elast6": lambda: inputs.elasticity_grid(6, nrhs=1, levels=3),   # r <= 6 (groups of up to 8 rows)
    "cc32": lambda: inputs.diffusion_cc(32, nrhs=1, max_coarse=256),
}


@pytest.fixture(scope="module")
def amg():
    import torch  # noqa: F401
    from paper_1907_04417_gb300 import amg as A, build
    build.build()
    return A


@pytest.fixture(scope="module")
def problems():
    out = {}
    for name, mk in PROBLEMS.items():
        P = mk()
        out[name] = (P, O.setup(P.A, P.aggs, P.n_nodes, P.W))
    return out


def _choices(path, levels):
    """(lanes per smoothed level, kernel per transfer) of the last cached line."""
    line = [l for l in open(path) if " | " in l][-1]
    v = [int(t) for t in line.split(" | ")[1].split()]
    nt = levels - 1
    nzl = [v[3 * k + 2] for k in range(nt)]
    kern = [v[3 * nt + 3 * k + 2] % 4 for k in range(nt)]  # restriction kernel (the prolongation's is / 4)
    return nzl, kern


def _solve(amg, monkeypatch, tmp_path, P, mode, B, **kw):
    cache = tmp_path / f"tune_{mode}.txt"
    monkeypatch.setenv("AMG_COARSE_KERNELS", mode)
    monkeypatch.setenv("AMG_TUNE_CACHE", str(cache))
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    X, info, st = H.solve(B, options=amg.opts(**kw))
    nzl, kern = _choices(cache, H.info()["levels"])
    H.close()
    return X, info, st, nzl, kern


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("k", [8, 32])
def test_grouped_fp64_matches_oracle_and_csr(amg, problems, monkeypatch, tmp_path, name, k):
    P, Ho = problems[name]
    B = np.random.default_rng(k).uniform(-1.0, 1.0, (P.n, k))
    Xg, ig, st, nzl, kern = _solve(amg, monkeypatch, tmp_path, P, "grouped", B)
    assert st == amg.AMG_OK
    L = Ho.L
    # every smoothed coarse level and every transfer out of one took the grouped kernels
    assert all(n <= 0 for n in nzl[1:]), nzl
    assert all(t == 2 for t in kern[1:]), kern
    for c in (0, k // 2, k - 1):
        _, res = O.solve(Ho, B[:, c])
        assert abs(ig[c]["iters"] - res[0].iters) <= 1, (c, ig[c]["iters"], res[0].iters)
        xf, _ = O.solve(Ho, B[:, c], fixed_iters=ig[c]["iters"])
        assert np.linalg.norm(Xg[:, c] - xf) / np.linalg.norm(xf) <= 1e-10
    Xc, ic_, st, nzl, kern = _solve(amg, monkeypatch, tmp_path, P, "csr", B)
    assert st == amg.AMG_OK
    assert all(n > 0 for n in nzl) and all(t != 2 for t in kern), (nzl, kern)
    same = [c for c in range(k) if ic_[c]["iters"] == ig[c]["iters"]]
    assert len(same) >= k // 2
    for c in same:
        assert np.linalg.norm(Xg[:, c] - Xc[:, c]) / np.linalg.norm(Xc[:, c]) <= 1e-10
    assert L >= 3


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_grouped_fp32_cycle(amg, problems, monkeypatch, tmp_path, name):
    P, Ho = problems[name]
    k = 32
    B = np.random.default_rng(5).uniform(-1.0, 1.0, (P.n, k))
    X64, i64, st64, _, _ = _solve(amg, monkeypatch, tmp_path, P, "grouped", B)
    X32, i32, st32, nzl, kern = _solve(amg, monkeypatch, tmp_path, P, "grouped", B, cycle_precision=32)
    assert st64 == amg.AMG_OK and st32 == amg.AMG_OK
    assert all(n <= 0 for n in nzl[1:]) and all(t == 2 for t in kern[1:]), (nzl, kern)
    tr = np.linalg.norm(B - P.A @ X32, axis=0) / np.linalg.norm(B, axis=0)
    assert tr.max() <= 1.1e-8, tr.max()
    for c in range(k):
        assert i32[c]["iters"] <= i64[c]["iters"] + 3, (c, i32[c]["iters"], i64[c]["iters"])


SWEEP_CODE = {"groupwarp": -16, "groupslot": -17}


@pytest.mark.parametrize("mode", list(SWEEP_CODE))
@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("k", [8, 32])
def test_group_warp_sweep_fp64_matches_oracle(amg, problems, monkeypatch, tmp_path, name, k, mode):
    """The sweep with one warp, or one slot of lanes, per row group (an
    entry-major copy of the level's values, patterns padded to multiples of
    8 entries, each pattern row of u gathered once per group)."""
    P, Ho = problems[name]
    B = np.random.default_rng(40 + k).uniform(-1.0, 1.0, (P.n, k))
    Xg, ig, st, nzl, kern = _solve(amg, monkeypatch, tmp_path, P, mode, B)
    assert st == amg.AMG_OK
    assert all(n == SWEEP_CODE[mode] for n in nzl[1:]), nzl
    for c in (0, k // 2, k - 1):
        _, res = O.solve(Ho, B[:, c])
        assert abs(ig[c]["iters"] - res[0].iters) <= 1, (c, ig[c]["iters"], res[0].iters)
        xf, _ = O.solve(Ho, B[:, c], fixed_iters=ig[c]["iters"])
        assert np.linalg.norm(Xg[:, c] - xf) / np.linalg.norm(xf) <= 1e-10


@pytest.mark.parametrize("mode", list(SWEEP_CODE))
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_group_warp_sweep_fp32_cycle(amg, problems, monkeypatch, tmp_path, name, mode):
    P, Ho = problems[name]
    k = 32
    B = np.random.default_rng(6).uniform(-1.0, 1.0, (P.n, k))
    X64, i64, st64, _, _ = _solve(amg, monkeypatch, tmp_path, P, mode, B)
    X32, i32, st32, nzl, kern = _solve(amg, monkeypatch, tmp_path, P, mode, B, cycle_precision=32)
    assert st64 == amg.AMG_OK and st32 == amg.AMG_OK
    assert all(n == SWEEP_CODE[mode] for n in nzl[1:]), nzl
    tr = np.linalg.norm(B - P.A @ X32, axis=0) / np.linalg.norm(B, axis=0)
    assert tr.max() <= 1.1e-8, tr.max()
    for c in range(k):
        assert i32[c]["iters"] <= i64[c]["iters"] + 3, (c, i32[c]["iters"], i64[c]["iters"])


@pytest.mark.parametrize("mode", list(SWEEP_CODE))
def test_group_warp_sweep_vcycle(amg, problems, monkeypatch, tmp_path, mode):
    """One float64 V-cycle with the warp- or slot-per-group sweep on every
    coarse level against the oracle's, element by element."""
    P, Ho = problems["aniso64"]
    R = np.random.default_rng(8).uniform(-1.0, 1.0, (P.n, 16))
    monkeypatch.setenv("AMG_COARSE_KERNELS", mode)
    monkeypatch.setenv("AMG_FUSED_COARSE", "0")
    monkeypatch.setenv("AMG_TUNE_CACHE", str(tmp_path / "tune_vc.txt"))
    H = amg.Hierarchy(P.A, P.aggs, P.n_nodes, P.W)
    Z = H.vcycle(R)
    H.close()
    Zo = O.vcycle(Ho, R)
    assert np.abs(Z - Zo).max() <= 1e-12 * np.abs(Zo).max()
