"""Python binding of the C ABI in include/amg.h (argument marshalling only).

Every function here forwards to ``libamg_gb300.so``; no step of the method
runs in Python.  Arrays may be numpy arrays (host memory) or torch tensors
(host or CUDA memory); they must be C-contiguous with the documented dtype.
If the shared library has not been built, loading raises ``RuntimeError``:
there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libamg_gb300.so")

AMG_OK = 0
AMG_ERR_INVALID_ARG = 1
AMG_ERR_NOT_SPD = 2
AMG_ERR_NOT_CONVERGED = 3
AMG_ERR_BREAKDOWN = 4
AMG_ERR_TIMEOUT = 5
AMG_ERR_CUDA = 6
AMG_ERR_ALLOC = 7
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOT_SPD", 3: "NOT_CONVERGED", 4: "BREAKDOWN",
                5: "TIMEOUT", 6: "CUDA", 7: "ALLOC"}

KERNEL_SPMV_CG = 1
KERNEL_RESTRICT_L0 = 2
KERNEL_SMOOTH_L0 = 3
KERNEL_PROLONG_L0 = 4
KERNEL_CG_UPDATE = 5
KERNEL_GS_L0 = 6
KERNEL_CG_DIRECTION = 7
KERNEL_COARSE_LEVELS = 8


class AMGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class amg_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class amg_opts(C.Structure):
    _fields_ = [("tol_svd", C.c_double), ("pre", C.c_int32), ("post", C.c_int32),
                ("cycle_precision", C.c_int32), ("rtol", C.c_double), ("maxit", C.c_int32),
                ("use_graph", C.c_int32), ("check_every", C.c_int32), ("autotune", C.c_int32),
                ("outer_fp64", C.c_int32), ("smoother", C.c_int32), ("cycle", C.c_int32)]

SMOOTHER_L1JACOBI = 0
SMOOTHER_GS = 1
CYCLE_V = 0
CYCLE_K = 1


class amg_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("status", C.c_int32),
                ("reserved", C.c_int32), ("relres", C.c_double)]


class amg_hier_info(C.Structure):
    _fields_ = [("levels", C.c_int32), ("m", C.c_int32), ("opc", C.c_double), ("cr", C.c_double),
                ("n_level", C.c_int64 * 16), ("nnz_level", C.c_int64 * 16),
                ("truncated_aggs", C.c_int64), ("device_bytes", C.c_int64)]


_lib = None

# name -> (restype, argtypes); every function declared in include/amg.h
SIGNATURES = {
    "amg_default_opts": (None, [C.POINTER(amg_opts)]),
    "amg_setup_from_aggregates": (C.c_int, [C.POINTER(amg_csr), C.c_int32, C.POINTER(C.c_void_p),
                                            C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(amg_opts),
                                            C.c_void_p, C.POINTER(C.c_void_p)]),
    "amg_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(amg_opts),
                            C.c_void_p, C.POINTER(amg_info)]),
    "amg_solve_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p),
                                    C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(amg_opts), C.c_void_p,
                                    C.POINTER(amg_info)]),
    "amg_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                              C.POINTER(amg_opts), C.c_void_p, C.POINTER(amg_info)]),
    "amg_vcycle": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(amg_opts),
                             C.c_void_p]),
    "amg_hierarchy_info": (C.c_int, [C.c_void_p, C.POINTER(amg_hier_info)]),
    "amg_export_level": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]),
    "amg_level_colours": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32)]),
    "amg_timer_enable": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "amg_timer_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "amg_restriction_info": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                       C.POINTER(C.c_int32)]),
    "amg_kernel_launches": (C.c_int, [C.POINTER(C.c_int64)]),
    "amg_local_bases_static": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                         C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "amg_bootstrap_test": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                     C.c_int32, C.POINTER(amg_opts), C.c_void_p, C.c_void_p, C.c_void_p]),
    "amg_pairwise_matching": (C.c_int, [C.POINTER(amg_csr), C.c_void_p, C.c_void_p, C.c_void_p]),
    "amg_pairwise_step": (C.c_int, [C.POINTER(amg_csr), C.c_void_p, C.c_void_p, C.POINTER(C.c_int32),
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p,
                                    C.c_void_p]),
    "amg_destroy": (None, [C.c_void_p]),
    "amg_last_error": (C.c_char_p, []),
}


def lib():
    """Load the shared library (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing ({LIB_PATH}); build it with "
                               "paper_1907_04417_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().amg_last_error().decode()


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    n = C.c_int64()
    _check(lib().amg_kernel_launches(C.byref(n)))
    return n.value


def local_bases_static(W, row_start, nf, tol, U, r, stream=None) -> int:
    """Eq. (svd) bases into caller-owned device tensors without any device
    allocation (see amg_local_bases_static in include/amg.h).  W, U: (nf, m)
    float64 CUDA tensors; row_start: (nagg + 1,) int32; r: (nagg,) int32.
    Returns the amg_status."""
    keep = []
    m = int(W.shape[1])
    nagg = int(row_start.shape[0]) - 1
    return lib().amg_local_bases_static(_ptr(W, np.float64, keep), m, _ptr(row_start, np.int32, keep), nagg,
                                        int(nf), float(tol), _ptr(U, np.float64, keep),
                                        _ptr(r, np.int32, keep), _stream(stream))


def opts(**kw) -> amg_opts:
    o = amg_opts()
    lib().amg_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _check(status, allowed=(AMG_OK,)):
    if status not in allowed:
        raise AMGError(status, last_error())
    return status


def _ptr(a, dtype, keep):
    """Raw pointer of a C-contiguous numpy array or torch tensor of ``dtype``."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
            if a.dtype != tdt or not a.is_contiguous():
                raise TypeError(f"tensor must be contiguous {tdt}")
            keep.append(a)
            return a.data_ptr()
    except ImportError:  # pragma: no cover
        pass
    arr = np.asarray(a)
    if arr.dtype != dtype or not arr.flags["C_CONTIGUOUS"]:
        raise TypeError(f"array must be C-contiguous {np.dtype(dtype)}")
    keep.append(arr)
    return arr.ctypes.data


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return None


class Hierarchy:
    """Handle of a device hierarchy built by amg_setup_from_aggregates."""

    def __init__(self, A, aggs, n_nodes, W, options: amg_opts | None = None, stream=None):
        keep = []
        if hasattr(A, "indptr"):
            rowptr, col, val = A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64)
            n = A.shape[0]
        else:
            rowptr, col, val = A
            n = int(rowptr.shape[0]) - 1
        csr = amg_csr(n, int(col.shape[0]), _ptr(rowptr, np.int32, keep), _ptr(col, np.int32, keep),
                      _ptr(val, np.float64, keep))
        nl = len(aggs)
        agg_ptrs = (C.c_void_p * max(nl, 1))(*[_ptr(np.ascontiguousarray(a, dtype=np.int32)
                                                     if not _is_torch(a) else a, np.int32, keep)
                                                for a in aggs])
        nn = np.ascontiguousarray(np.asarray(n_nodes, dtype=np.int32))
        Wc = W
        if not _is_torch(W):
            W2 = np.asarray(W, dtype=np.float64)
            if W2.ndim == 1:
                W2 = W2[:, None]
            Wc = np.ascontiguousarray(W2.T)  # n x m column-major == m x n row-major
            m = W2.shape[1]
        else:
            m = W.shape[1] if W.dim() == 2 else 1
            Wc = W.t().contiguous() if W.dim() == 2 else W.contiguous()
        out = C.c_void_p()
        st = lib().amg_setup_from_aggregates(C.byref(csr), nl, agg_ptrs, _ptr(nn, np.int32, keep),
                                             _ptr(Wc, np.float64, keep), m,
                                             C.byref(options) if options is not None else None,
                                             _stream(stream), C.byref(out))
        _check(st)
        self.h = out.value
        self.n = n
        self.nnz = int(col.shape[0])
        self.m = m
        # the matrix values the hierarchy was built from (caller CSR order),
        # so that a caller can check that a solve still belongs to them
        self.setup_values = val.detach().clone() if _is_torch(val) else np.array(val, dtype=np.float64)

    def close(self):
        if getattr(self, "h", None):
            lib().amg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def solve(self, b, x=None, options: amg_opts | None = None, stream=None):
        """x = A^{-1} b by AMG-PCG.  b: (n,) or (n, k) float64, numpy or torch.
        Returns (x, infos, status); raises for errors other than
        NOT_CONVERGED / BREAKDOWN (where x is still written)."""
        return _solve(self, b, x, options, stream)

    def vcycle(self, r, options: amg_opts | None = None, stream=None):
        keep = []
        r2, shape = _as2d(r)
        z = _empty_like(r2)
        _check(lib().amg_vcycle(self.h, _ptr(r2, np.float64, keep), _ptr(z, np.float64, keep), r2.shape[1],
                                C.byref(options) if options is not None else None, _stream(stream)))
        return _reshape(z, shape)

    def adjoint(self, g, x, options: amg_opts | None = None, stream=None):
        """Returns (lambda, grad_val, infos, status)."""
        keep = []
        g2, shape = _as2d(g)
        x2, _ = _as2d(x)
        lam = _empty_like(g2)
        grad = _empty_vec_like(g2, self.nnz)
        k = g2.shape[1]
        infos = (amg_info * k)()
        st = lib().amg_adjoint(self.h, _ptr(g2, np.float64, keep), _ptr(x2, np.float64, keep), k,
                               _ptr(lam, np.float64, keep), _ptr(grad, np.float64, keep),
                               C.byref(options) if options is not None else None, _stream(stream), infos)
        _check(st, (AMG_OK, AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN))
        return _reshape(lam, shape), grad, [_info_dict(i) for i in infos], st

    def info(self) -> dict:
        hi = amg_hier_info()
        _check(lib().amg_hierarchy_info(self.h, C.byref(hi)))
        L = hi.levels
        return {"levels": L, "m": hi.m, "opc": hi.opc, "cr": hi.cr,
                "n_level": list(hi.n_level[:L]), "nnz_level": list(hi.nnz_level[:L]),
                "truncated_aggs": hi.truncated_aggs, "device_bytes": hi.device_bytes}

    def level_colours(self, k: int):
        """(colour, ncolours) of the Gauss-Seidel smoother on level k, the
        colours in the caller's numbering of that level."""
        n = self.info()["n_level"][k]
        colour = np.zeros(max(n, 1), np.int32)
        nc = C.c_int32()
        _check(lib().amg_level_colours(self.h, k, colour.ctypes.data, C.byref(nc)))
        return colour[:n], nc.value

    def export_level(self, k: int) -> dict:
        sizes = np.zeros(6, dtype=np.int64)
        _check(lib().amg_export_level(self.h, k, sizes.ctypes.data, None, None, None, None, None, None,
                                      None, None))
        n, nnz, nagg, npv, nf, m = (int(v) for v in sizes)
        out = {"n": n, "nnz": nnz, "naggs": nagg, "nf": nf, "m": m,
               "rowptr": np.zeros(n + 1, np.int32), "col": np.zeros(max(nnz, 1), np.int32),
               "val": np.zeros(max(nnz, 1), np.float64)}
        ptrs = [out["rowptr"].ctypes.data, out["col"].ctypes.data, out["val"].ctypes.data]
        if k == 0:
            out["perm"] = np.zeros(n, np.int32)
            ptrs += [out["perm"].ctypes.data, None, None, None, None]
        else:
            out["agg_id"] = np.zeros(nagg, np.int32)
            out["r"] = np.zeros(nagg, np.int32)
            out["row_start"] = np.zeros(nagg + 1, np.int32)
            out["pval"] = np.zeros(max(npv, 1), np.float64)
            ptrs += [None, out["agg_id"].ctypes.data, out["r"].ctypes.data, out["row_start"].ctypes.data,
                     out["pval"].ctypes.data]
        _check(lib().amg_export_level(self.h, k, sizes.ctypes.data, *ptrs))
        out["col"] = out["col"][:nnz]
        out["val"] = out["val"][:nnz]
        if k > 0:
            out["pval"] = out["pval"][:npv]
        return out

    def timer_enable(self, kernel_id: int, enable: bool = True):
        _check(lib().amg_timer_enable(self.h, kernel_id, 1 if enable else 0))

    def timer_read(self):
        ms = C.c_double()
        n = C.c_int64()
        _check(lib().amg_timer_read(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def restriction_info(self, k: int) -> dict:
        """How the most recent V-cycle of a solve restricted out of level k:
        by_r (R = P^T (I - A D^{-1}) applied), R's pattern entries and values
        per entry."""
        by_r = C.c_int32()
        ent = C.c_int64()
        rs = C.c_int32()
        _check(lib().amg_restriction_info(self.h, k, C.byref(by_r), C.byref(ent), C.byref(rs)))
        return {"by_r": bool(by_r.value), "entries": ent.value, "values_per_entry": rs.value}


def _is_torch(a):
    try:
        import torch
        return isinstance(a, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _as2d(a):
    if _is_torch(a):
        a2 = a if a.dim() == 2 else a.reshape(-1, 1)
        return a2.contiguous(), tuple(a.shape)
    arr = np.asarray(a, dtype=np.float64)
    a2 = arr if arr.ndim == 2 else arr.reshape(-1, 1)
    return np.ascontiguousarray(a2), arr.shape


def _empty_like(a2):
    if _is_torch(a2):
        import torch
        return torch.zeros_like(a2)
    return np.zeros_like(a2)


def _empty_vec_like(a2, n):
    if _is_torch(a2):
        import torch
        return torch.zeros(n, dtype=torch.float64, device=a2.device)
    return np.zeros(n, dtype=np.float64)


def _reshape(a2, shape):
    return a2.reshape(shape)


def _info_dict(i):
    return {"iters": i.iters, "converged": bool(i.converged), "status": i.status, "relres": i.relres}


def _solve(h, b, x, options, stream):
    keep = []
    b2, shape = _as2d(b)
    if x is None:
        x2 = _empty_like(b2)
    else:
        x2, _ = _as2d(x)
    k = b2.shape[1]
    infos = (amg_info * k)()
    st = lib().amg_solve(h.h, _ptr(b2, np.float64, keep), _ptr(x2, np.float64, keep), k,
                         C.byref(options) if options is not None else None, _stream(stream), infos)
    _check(st, (AMG_OK, AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN))
    return _reshape(x2, shape), [_info_dict(i) for i in infos], st


def solve_batched(hs, bs, xs=None, options: amg_opts | None = None, stream=None):
    """Solve several systems (one hierarchy each) in one launch sequence.
    bs[s]: (n_s, k_s) float64.  Returns (xs, infos per system, status)."""
    keep = []
    ns = len(hs)
    b2 = [_as2d(b)[0] for b in bs]
    x2 = [(_empty_like(b) if xs is None else _as2d(xs[s])[0]) for s, b in enumerate(b2)]
    nr = np.array([b.shape[1] for b in b2], dtype=np.int32)
    hp = (C.c_void_p * ns)(*[h.h for h in hs])
    bp = (C.c_void_p * ns)(*[_ptr(b, np.float64, keep) for b in b2])
    xp = (C.c_void_p * ns)(*[_ptr(x, np.float64, keep) for x in x2])
    infos = (amg_info * int(nr.sum()))()
    st = lib().amg_solve_batched(hp, ns, bp, xp, nr.ctypes.data, C.byref(options) if options is not None else None,
                                 _stream(stream), infos)
    _check(st, (AMG_OK, AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN))
    out, o = [], 0
    for s in range(ns):
        out.append([_info_dict(infos[o + c]) for c in range(int(nr[s]))])
        o += int(nr[s])
    return x2, out, st


def bootstrap_test(hs, x, nu: int, symmetric: bool = True, options: amg_opts | None = None, stream=None):
    """Testing phase of the bootstrap (amg_bootstrap_test in include/amg.h):
    returns (E^nu x, rho, ||E^nu x||_A) for the composite error operator of
    the hierarchies ``hs``.  x: (n,) or (n, k) float64, numpy or torch; the
    input is not modified (a copy is passed)."""
    keep = []
    x2, shape = _as2d(x)
    x2 = x2.clone() if _is_torch(x2) else x2.copy()
    k = int(x2.shape[1])
    rho = np.zeros(k, dtype=np.float64)
    anorm = np.zeros(k, dtype=np.float64)
    hp = (C.c_void_p * len(hs))(*[h.h for h in hs])
    _check(lib().amg_bootstrap_test(hp, len(hs), _ptr(x2, np.float64, keep), k, int(nu), 1 if symmetric else 0,
                                    C.byref(options) if options is not None else None, _stream(stream),
                                    rho.ctypes.data, anorm.ctypes.data))
    return _reshape(x2, shape), rho, anorm


def pairwise_matching(A, w, stream=None) -> np.ndarray:
    """Compatible weighted matching of one pairwise step on the device
    (amg_pairwise_matching in include/amg.h).  A: scipy CSR matrix; w: (n,)
    float64.  Returns mate (n,) int32, -1 for unmatched vertices."""
    keep = []
    rowptr = np.ascontiguousarray(A.indptr, dtype=np.int32)
    col = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    wv = np.ascontiguousarray(w, dtype=np.float64)
    n = int(A.shape[0])
    csr = amg_csr(n, int(col.size), rowptr.ctypes.data, col.ctypes.data, val.ctypes.data)
    keep += [rowptr, col, val, wv]
    mate = np.empty(n, dtype=np.int32)
    _check(lib().amg_pairwise_matching(C.byref(csr), wv.ctypes.data, mate.ctypes.data, _stream(stream)))
    return mate


def pairwise_step(A, w, stream=None):
    """One pairwise aggregation step on the device (amg_pairwise_step in
    include/amg.h).  A: scipy CSR matrix; w: (n,) float64.  Returns (agg,
    A_c, w_c) with agg (n,) int32, A_c a scipy CSR matrix and w_c (nc,)."""
    import scipy.sparse as sp
    rowptr = np.ascontiguousarray(A.indptr, dtype=np.int32)
    col = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    wv = np.ascontiguousarray(w, dtype=np.float64)
    n, nnz = int(A.shape[0]), int(col.size)
    csr = amg_csr(n, nnz, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data)
    agg = np.empty(n, dtype=np.int32)
    rpc = np.empty(n + 1, dtype=np.int32)
    colc = np.empty(max(nnz, 1), dtype=np.int32)
    valc = np.empty(max(nnz, 1), dtype=np.float64)
    wc = np.empty(max(n, 1), dtype=np.float64)
    nc = C.c_int32()
    nnzc = C.c_int32()
    _check(lib().amg_pairwise_step(C.byref(csr), wv.ctypes.data, agg.ctypes.data, C.byref(nc), rpc.ctypes.data,
                                   colc.ctypes.data, valc.ctypes.data, C.byref(nnzc), wc.ctypes.data,
                                   _stream(stream)))
    k, z = nc.value, nnzc.value
    Ac = sp.csr_matrix((valc[:z].copy(), colc[:z].copy(), rpc[:k + 1].copy()), shape=(k, k))
    return agg, Ac, wc[:k].copy()


def aggregate_hierarchy(A, w, steps_per_level, min_nodes: int = 1):
    """Nested aggregate maps from composed pairwise steps, every step on the
    device (the composition of Section 3, aggressive coarsening): aggs[k][node]
    is the level-(k+1) aggregate of level-k node, n_nodes[k] the level-k node
    count."""
    aggs, n_nodes = [], [A.shape[0]]
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
