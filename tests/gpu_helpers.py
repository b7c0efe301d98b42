"""Helpers shared by the GPU parity tests: map the library's internal
numbering (aggregates contiguous) and column signs onto the oracle's."""
import numpy as np
import scipy.sparse as sp


def oracle_coarse_start(Ho, k):
    return np.concatenate([[0], np.cumsum(Ho.levels[k].r)]).astype(np.int64)


def _block_entries(e):
    """Flatten the exported prolongator blocks of one level: for every stored
    value its library fine row and library coarse column."""
    r = e["r"].astype(np.int64)
    rs = e["row_start"].astype(np.int64)
    na = np.diff(rs)
    size = na * r
    t = np.repeat(np.arange(e["naggs"]), size)
    loc = np.arange(size.sum()) - np.repeat(np.cumsum(size) - size, size)
    col0 = np.cumsum(r) - r
    return t, rs[t] + loc // r[t], col0[t] + loc % r[t]


def level_maps(Hg, Ho):
    """For every level k: sigma_k (library dof -> oracle dof) and the signs
    s_k (library column = s_k * oracle column).  Also returns the exports."""
    ex = [Hg.export_level(k) for k in range(Ho.L)]
    sig = [ex[0]["perm"].astype(np.int64)]
    sgn = [np.ones(ex[0]["n"])]
    for k in range(1, Ho.L):
        e = ex[k]
        cs = oracle_coarse_start(Ho, k)
        r = e["r"].astype(np.int64)
        r_orc = Ho.levels[k].r[e["agg_id"]]
        assert np.array_equal(r_orc, r), "kept-column counts differ from the oracle"
        owner = np.repeat(np.arange(e["naggs"]), r)
        s_map = cs[e["agg_id"]][owner] + np.arange(r.sum()) - np.repeat(np.cumsum(r) - r, r)
        _, frow, ccol = _block_entries(e)
        Porc = Ho.levels[k].P.tocsr()
        ob = np.asarray(Porc[sig[k - 1][frow], s_map[ccol]]).ravel() * sgn[k - 1][frow]
        d = np.bincount(ccol, weights=e["pval"] * ob, minlength=e["n"])
        sig.append(s_map.astype(np.int64))
        sgn.append(np.where(d < 0, -1.0, 1.0))
    return ex, sig, sgn


def compare_prolongators(Hg, Ho, atol=1e-10):
    ex, sig, sgn = level_maps(Hg, Ho)
    worst = 0.0
    for k in range(1, Ho.L):
        e = ex[k]
        _, frow, ccol = _block_entries(e)
        Porc = Ho.levels[k].P.tocsr()
        ob = np.asarray(Porc[sig[k - 1][frow], sig[k][ccol]]).ravel()
        # every nonzero of the oracle's P lies inside the library's block pattern
        assert np.count_nonzero(ob) == np.count_nonzero(Porc.data)
        ob = ob * sgn[k - 1][frow] * sgn[k][ccol]
        worst = max(worst, float(np.abs(e["pval"] - ob).max(initial=0.0)))
    assert worst <= atol, worst
    return worst, ex, sig, sgn


def compare_coarse_matrices(Ho, ex, sig, sgn, rtol=1e-10):
    worst = 0.0
    for k in range(Ho.L):
        e = ex[k]
        n = e["n"]
        rows = np.repeat(np.arange(n), np.diff(e["rowptr"]))
        vals = e["val"] * sgn[k][rows] * sgn[k][e["col"]]
        Ag = sp.csr_matrix((vals, (sig[k][rows], sig[k][e["col"]])), shape=(n, n))
        Ao = Ho.levels[k].A
        diff = abs(Ag - Ao).max()
        scale = abs(Ao).max()
        worst = max(worst, diff / scale)
    assert worst <= rtol, worst
    return worst
