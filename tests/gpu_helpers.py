"""Helpers shared by the GPU parity tests: map the library's internal
numbering (aggregates contiguous) and column signs onto the oracle's."""
import numpy as np
import scipy.sparse as sp


def oracle_coarse_start(Ho, k):
    return np.concatenate([[0], np.cumsum(Ho.levels[k].r)]).astype(np.int64)


def level_maps(Hg, Ho):
    """For every level k: sigma_k (library dof -> oracle dof) and the signs
    s_k (library column = s_k * oracle column).  Also returns the exports."""
    ex = [Hg.export_level(k) for k in range(Ho.L)]
    sig = [ex[0]["perm"].astype(np.int64)]
    sgn = [np.ones(ex[0]["n"])]
    for k in range(1, Ho.L):
        e = ex[k]
        cs = oracle_coarse_start(Ho, k)
        r_orc = Ho.levels[k].r[e["agg_id"]]
        assert np.array_equal(r_orc, e["r"]), "kept-column counts differ from the oracle"
        s_map = np.concatenate([cs[a] + np.arange(r) for a, r in zip(e["agg_id"], e["r"])]).astype(np.int64)
        Porc = Ho.levels[k].P.tocsr()
        signs = np.empty(e["n"])
        off = 0
        cpos = 0
        rs = e["row_start"]
        for t in range(e["naggs"]):
            na = rs[t + 1] - rs[t]
            r = e["r"][t]
            blk = e["pval"][off:off + na * r].reshape(na, r)
            rows_o = sig[k - 1][rs[t]:rs[t + 1]]
            cols_o = s_map[cpos:cpos + r]
            ob = Porc[rows_o][:, cols_o].toarray() * sgn[k - 1][rs[t]:rs[t + 1], None]
            d = np.sum(blk * ob, axis=0)
            signs[cpos:cpos + r] = np.where(d < 0, -1.0, 1.0)
            off += na * r
            cpos += r
        sig.append(s_map)
        sgn.append(signs)
    return ex, sig, sgn


def compare_prolongators(Hg, Ho, atol=1e-10):
    ex, sig, sgn = level_maps(Hg, Ho)
    worst = 0.0
    for k in range(1, Ho.L):
        e = ex[k]
        rs = e["row_start"]
        Porc = Ho.levels[k].P.tocsr()
        off = 0
        cpos = 0
        for t in range(e["naggs"]):
            na = rs[t + 1] - rs[t]
            r = e["r"][t]
            blk = e["pval"][off:off + na * r].reshape(na, r)
            ob = Porc[sig[k - 1][rs[t]:rs[t + 1]]][:, sig[k][cpos:cpos + r]].toarray()
            ob = ob * sgn[k - 1][rs[t]:rs[t + 1], None] * sgn[k][None, cpos:cpos + r]
            worst = max(worst, float(np.abs(blk - ob).max()))
            off += na * r
            cpos += r
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
