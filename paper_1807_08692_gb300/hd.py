"""Thin ctypes binding of libhd.so (include/hd.h), same entry-point names.

Only argument marshalling happens here: torch tensors pass their data_ptr(),
numpy arrays pass host pointers, and every computation runs in the library's
CUDA kernels.  PyTorch provides device memory and the current CUDA stream.
If the library is missing, loading raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhd.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4
ERR_NOT_CONVERGED = -5
PENDING = -6
F32, BF16, FP8 = 0, 1, 2
SYM_UNION, SYM_MUTUAL = 0, 1
MODE_PAPER, MODE_PROJ, MODE_PCG = 0, 1, 2
MODE_TEMPORAL_ONLY = 0x100
COL_CONVERGED, COL_MAX_ITER, COL_BREAKDOWN, COL_EMPTY, COL_CANCELLED, COL_STAGNATED = 0, 1, 2, 3, 4, 5

MODES = {"paper": MODE_PAPER, "proj": MODE_PROJ, "pcg": MODE_PCG,
         "paper_temporal": MODE_PAPER | MODE_TEMPORAL_ONLY, "proj_temporal": MODE_PROJ | MODE_TEMPORAL_ONLY}
STORAGES = {"f32": F32, "bf16": BF16, "fp8": FP8}

_lib = None

vp, i32, i64, f32, f64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double, C.c_uint64

_SIGS = {
    "hd_create": (C.c_int, [C.POINTER(vp), C.c_int, vp]),
    "hd_set_stream": (C.c_int, [vp, vp]),
    "hd_destroy": (C.c_int, [vp]),
    "hd_last_error": (C.c_char_p, [vp]),
    "hd_launch_count": (i64, [vp]),
    "hd_workspace_bytes": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
    "hd_num_sms": (C.c_int, [vp]),
    "hd_profile_enable": (C.c_int, [vp, C.c_int]),
    "hd_profile_read": (C.c_int, [vp, C.c_char_p, C.POINTER(i64), C.POINTER(f64), C.POINTER(i64)]),
    "hd_graph_from_csr": (C.c_int, [vp, i64, i64, vp, vp, vp, C.c_int, C.POINTER(vp)]),
    "hd_build_graph": (C.c_int, [vp, vp, i64, i32, C.c_int, i32, f32, C.c_int, C.POINTER(vp)]),
    "hd_knn": (C.c_int, [vp, vp, i64, i32, C.c_int, vp, i64, i32, C.c_int, vp, vp]),
    "hd_observe": (C.c_int, [vp, vp, i64, i32, C.c_int, vp, i32, i32, f32, vp, vp, vp]),
    "hd_graph_info": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i64)]),
    "hd_graph_tuning": (C.c_int, [vp, i32, C.POINTER(i32), C.POINTER(i32)]),
    "hd_graph_export": (C.c_int, [vp, vp, vp, vp, vp, vp]),
    "hd_graph_destroy": (C.c_int, [vp]),
    "hd_eig_from_host": (C.c_int, [vp, vp, i32, vp, vp, C.c_int, C.POINTER(vp)]),
    "hd_eigendecompose": (C.c_int, [vp, vp, i32, i32, i32, f64, i32, C.c_int, u64, C.POINTER(vp), vp, vp]),
    "hd_spectrum_min": (C.c_int, [vp, vp, f64, i32, u64, C.POINTER(f64)]),
    "hd_cg_bound": (C.c_int, [C.c_int, f64, f64, f64, f64, C.POINTER(f64), C.POINTER(i32), C.POINTER(i32)]),
    "hd_eig_info": (C.c_int, [vp, C.POINTER(i32), C.POINTER(C.c_int)]),
    "hd_eig_restarts": (C.c_int, [vp, C.POINTER(i32)]),
    "hd_eig_sparsify": (C.c_int, [vp, vp, f64, C.POINTER(vp)]),
    "hd_filter_poly": (C.c_int, [vp, vp, vp, i32, vp, vp, vp, vp, i32, vp, i32]),
    "hd_selftest_wait": (C.c_int, [vp, C.c_uint32, vp]),
    "hd_graph_save": (C.c_int, [vp, vp, C.c_char_p]),
    "hd_graph_load": (C.c_int, [vp, C.c_char_p, C.POINTER(vp)]),
    "hd_eig_save": (C.c_int, [vp, vp, C.c_char_p]),
    "hd_eig_load": (C.c_int, [vp, C.c_char_p, C.POINTER(vp)]),
    "hd_temporal_truncated": (C.c_int, [vp, vp, i32, vp, vp, vp, vp, vp, f64, vp, i32, vp, i32, vp, vp, vp]),
    "hd_eig_nnz": (C.c_int, [vp, C.POINTER(C.c_int64)]),
    "hd_eig_export": (C.c_int, [vp, vp, vp, vp]),
    "hd_eig_destroy": (C.c_int, [vp]),
    "hd_query_batch": (C.c_int, [vp, vp, vp, C.c_int, i32, vp, vp, vp, f64, vp, i32, vp, i32, vp, vp, vp]),
    "hd_rank": (C.c_int, [vp, vp, i64, i32, i32, vp, i32, i32, vp, vp]),
    "hd_eig_project": (C.c_int, [vp, vp, vp, i32, vp]),
    "hd_rank_static": (C.c_int, [vp, vp, i64, i32, i32, vp, i32, vp, vp]),
    "hd_serve_open": (C.c_int, [vp, vp, vp, C.c_int, f64, i32, C.c_size_t, i32, i32, C.POINTER(vp)]),
    "hd_serve_slots": (C.c_int, [vp]),
    "hd_serve_submit": (C.c_int, [vp, i32, vp, vp, f32, i32, C.POINTER(u64)]),
    "hd_serve_step": (C.c_int, [vp, i32, C.POINTER(i32)]),
    "hd_serve_poll": (C.c_int, [vp, u64, vp, vp, vp]),
    "hd_serve_completed": (C.c_int, [vp, vp, i32, C.POINTER(i32)]),
    "hd_serve_cancel": (C.c_int, [vp, u64]),
    "hd_serve_close": (C.c_int, [vp]),
    "hd_eig_expand": (C.c_int, [vp, vp, vp, i32, vp]),
}


class HDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hd error {code}: {msg}")
        self.code = code


def lib():
    """Load libhd.so (built by paper_1807_08692_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return [n for n in _SIGS if hasattr(lib(), n)]


def _typed(x, np_dtype, torch_name: str):
    """numpy input as a contiguous array of np_dtype; a tensor must already have
    that element type (it is passed by pointer)."""
    if x is None or isinstance(x, np.ndarray) or isinstance(x, (list, tuple)):
        return None if x is None else np.ascontiguousarray(x, np_dtype)
    if hasattr(x, "dtype") and str(x.dtype) != f"torch.{torch_name}":
        raise TypeError(f"expected a {torch_name} tensor, got {x.dtype}")
    return x


def _ptr(x):
    """Pointer of a torch tensor, a numpy array or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "numpy arrays must be C-contiguous"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.dim() == 0 or x.stride(-1) == 1, "tensors must be row-major with unit column stride"
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(type(x))


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Context:
    """A library context on one device and one stream (hd_create)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        torch.cuda.init()
        self._h = vp()
        rc = lib().hd_create(C.byref(self._h), device, _stream_handle(stream))
        if rc != OK:
            raise HDError(rc, "hd_create failed")
        self.device = device
        # servers keep a pointer to the context: they are closed before it
        self._servers = weakref.WeakSet()

    @property
    def handle(self):
        return self._h

    def check(self, rc, what=""):
        if rc != OK:
            raise HDError(rc, f"{what}: {lib().hd_last_error(self._h).decode()}")
        return rc

    def set_stream(self, stream=None):
        self.check(lib().hd_set_stream(self._h, _stream_handle(stream)), "hd_set_stream")

    def launches(self) -> int:
        return int(lib().hd_launch_count(self._h))

    def workspace_bytes(self) -> int:
        """Device workspace the context holds (hd_workspace_bytes)."""
        b = C.c_size_t()
        self.check(lib().hd_workspace_bytes(self._h, C.byref(b)), "hd_workspace_bytes")
        return int(b.value)

    def num_sms(self) -> int:
        return int(lib().hd_num_sms(self._h))

    def profile(self, on: bool = True):
        self.check(lib().hd_profile_enable(self._h, int(on)), "hd_profile_enable")

    def profile_read(self, name: str, busy: bool = False):
        """(launches, total_ms[, busy_launches]) of a kernel family since the last read."""
        cnt, ms, b = i64(), f64(), i64()
        self.check(lib().hd_profile_read(self._h, name.encode(), C.byref(cnt), C.byref(ms), C.byref(b)),
                   "hd_profile_read")
        return (cnt.value, ms.value, b.value) if busy else (cnt.value, ms.value)

    def close(self):
        if self._h:
            for s in list(self._servers):
                s.close()
            lib().hd_destroy(self._h)
            self._h = vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    def __init__(self, ctx: Context, h):
        self.ctx, self._h = ctx, h
        n, nnz = i64(), i64()
        lib().hd_graph_info(h, C.byref(n), C.byref(nnz))
        self.n, self.nnz = n.value, nnz.value

    @property
    def handle(self):
        return self._h

    def save(self, path: str):
        """Write the graph to a checkpoint file (hd_graph_save)."""
        self.ctx.check(lib().hd_graph_save(self.ctx.handle, self._h, str(path).encode()), "hd_graph_save")

    def tuning(self, B: int):
        """(slab, segments) the SpMM measured for batch width B, or None before any solve at that width."""
        sl, sg = i32(), i32()
        if lib().hd_graph_tuning(self._h, (B + 3) // 4 * 4, C.byref(sl), C.byref(sg)) != OK:
            return None
        return sl.value, sg.value

    def export(self):
        """(row_ptr, col, val, dinv) as numpy arrays (host copies)."""
        rp = np.empty(self.n + 1, np.int32)
        col = np.empty(self.nnz, np.int32)
        val = np.empty(self.nnz, np.float32)
        dinv = np.empty(self.n, np.float32)
        self.ctx.check(lib().hd_graph_export(self.ctx.handle, self._h, _ptr(rp), _ptr(col), _ptr(val), _ptr(dinv)),
                       "hd_graph_export")
        return rp, col, val, dinv

    def close(self):
        if self._h:
            lib().hd_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Eig:
    def __init__(self, ctx: Context, h, n):
        self.ctx, self._h, self.n = ctx, h, n
        r, st = i32(), C.c_int()
        lib().hd_eig_info(h, C.byref(r), C.byref(st))
        self.r, self.storage = r.value, st.value

    @property
    def handle(self):
        return self._h

    @property
    def restarts(self) -> int:
        """Thick restarts of the Lanczos run that computed these eigenpairs (-1 otherwise)."""
        v = i32()
        lib().hd_eig_restarts(self._h, C.byref(v))
        return v.value

    @property
    def nnz(self) -> int:
        """Stored entries of U (n * r unless sparsified)."""
        v = C.c_int64()
        lib().hd_eig_nnz(self._h, C.byref(v))
        return v.value

    def save(self, path: str):
        """Write the eigenpairs to a checkpoint file (hd_eig_save)."""
        self.ctx.check(lib().hd_eig_save(self.ctx.handle, self._h, str(path).encode()), "hd_eig_save")

    def sparsify(self, sparsity: float) -> "Eig":
        """SHybrid (Sec. 5.3): a new handle keeping the largest-magnitude
        entries of U, round(sparsity * n * r) of them set to zero."""
        h = vp()
        self.ctx.check(lib().hd_eig_sparsify(self.ctx.handle, self._h, float(sparsity), C.byref(h)),
                       "hd_eig_sparsify")
        return Eig(self.ctx, h, self.n)

    def export(self):
        lam = np.empty(self.r, np.float64)
        U = np.empty((self.n, self.r), np.float32)
        self.ctx.check(lib().hd_eig_export(self.ctx.handle, self._h, _ptr(lam), _ptr(U)), "hd_eig_export")
        return lam, U

    def close(self):
        if self._h:
            lib().hd_eig_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dtype_code(X):
    import torch
    if isinstance(X, np.ndarray):
        if X.dtype == np.float32:
            return F32
        if X.dtype == np.uint16:
            return BF16
        raise TypeError(X.dtype)
    if X.dtype == torch.float32:
        return F32
    if X.dtype == torch.bfloat16:
        return BF16
    raise TypeError(X.dtype)


def graph_from_csr(ctx: Context, row_ptr, col, val, normalized: bool = False) -> Graph:
    n = len(row_ptr) - 1
    nnz = len(col)
    h = vp()
    ctx.check(lib().hd_graph_from_csr(ctx.handle, n, nnz, _ptr(row_ptr), _ptr(col), _ptr(val), int(normalized),
                                      C.byref(h)), "hd_graph_from_csr")
    return Graph(ctx, h)


def build_graph(ctx: Context, X, k: int, gamma: float = 3.0, sym: int = SYM_UNION) -> Graph:
    n, d = X.shape
    h = vp()
    ctx.check(lib().hd_build_graph(ctx.handle, _ptr(X), n, d, _dtype_code(X), k, gamma, sym, C.byref(h)),
              "hd_build_graph")
    return Graph(ctx, h)


def knn(ctx: Context, X, Q, k: int, exclude_self: bool = False):
    """Neighbour lists (idx, sim) as device tensors when X is on the device, else numpy."""
    import torch
    n, d = X.shape
    nq = Q.shape[0]
    if hasattr(X, "is_cuda") and X.is_cuda:
        idx = torch.empty((nq, k), dtype=torch.int32, device=X.device)
        sim = torch.empty((nq, k), dtype=torch.float32, device=X.device)
    else:
        idx = np.empty((nq, k), np.int32)
        sim = np.empty((nq, k), np.float32)
    ctx.check(lib().hd_knn(ctx.handle, _ptr(X), n, d, _dtype_code(X), _ptr(Q), nq, k, int(exclude_self), _ptr(idx),
                           _ptr(sim)), "hd_knn")
    return idx, sim


def observe(ctx: Context, X, Q, k_y: int, gamma: float = 3.0):
    """Observation vectors: (y_ptr, y_idx, y_val) host numpy arrays."""
    n, d = X.shape
    nq = Q.shape[0]
    ptr = np.empty(nq + 1, np.int32)
    idx = np.empty(nq * k_y, np.int32)
    val = np.empty(nq * k_y, np.float32)
    ctx.check(lib().hd_observe(ctx.handle, _ptr(X), n, d, _dtype_code(X), _ptr(Q), nq, k_y, gamma, _ptr(ptr),
                               _ptr(idx), _ptr(val)), "hd_observe")
    m = int(ptr[-1])
    return ptr, idx[:m].copy(), val[:m].copy()


def graph_load(ctx: Context, path: str) -> "Graph":
    """A graph from a checkpoint written by Graph.save."""
    h = vp()
    ctx.check(lib().hd_graph_load(ctx.handle, str(path).encode(), C.byref(h)), "hd_graph_load")
    return Graph(ctx, h)


def eig_load(ctx: Context, path: str) -> "Eig":
    """Eigenpairs from a checkpoint written by Eig.save."""
    h = vp()
    ctx.check(lib().hd_eig_load(ctx.handle, str(path).encode(), C.byref(h)), "hd_eig_load")
    with open(path, "rb") as f:
        f.seek(8)
        n = int(np.frombuffer(f.read(8), np.int64)[0])
    return Eig(ctx, h, n)


def selftest_wait(ctx: Context, limit_us: int = 20000):
    """(gave_up_on_timeout, gave_up_on_abort) of the bounded-wait self-test."""
    g = np.zeros(2, np.int32)
    rc = lib().hd_selftest_wait(ctx.handle, limit_us, _ptr(g))
    if rc not in (OK, ERR_TIMEOUT):
        ctx.check(rc, "hd_selftest_wait")
    return bool(g[0]), bool(g[1])


def observe_regional(ctx: Context, X, Q, regions: int, k_y: int, gamma: float = 3.0):
    """Regional queries: each image's `regions` consecutive rows of Q observe
    their own top-k_y and the image's observation is the concatenation (the
    solver sums duplicate ids).  (y_ptr, y_idx, y_val), one segment per image."""
    p, i, v = observe(ctx, X, Q, k_y, gamma)
    nimg = (len(p) - 1) // regions
    return np.ascontiguousarray(p[::regions][:nimg + 1], np.int32), i, v


def eig_from_host(ctx: Context, g: Graph, lam, U, storage="bf16") -> Eig:
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    r = lam.size
    if not hasattr(U, "data_ptr"):
        U = np.ascontiguousarray(U, dtype=np.float32)
    h = vp()
    ctx.check(lib().hd_eig_from_host(ctx.handle, g.handle, r, _ptr(lam), _ptr(U),
                                     STORAGES.get(storage, storage), C.byref(h)), "hd_eig_from_host")
    return Eig(ctx, h, g.n)


def eigendecompose(ctx: Context, g: Graph, r: int, block: int = 32, max_basis: int = 0, tol: float = 1e-6,
                   max_restarts: int = 30, storage="bf16", seed: int = 1):
    """Largest r eigenpairs by block Lanczos: (Eig, eigenvalues, residuals, converged)."""
    lam = np.zeros(r, np.float64)
    res = np.zeros(r, np.float64)
    h = vp()
    rc = lib().hd_eigendecompose(ctx.handle, g.handle, r, block, max_basis, tol, max_restarts,
                                 STORAGES.get(storage, storage), seed, C.byref(h), _ptr(lam), _ptr(res))
    if rc not in (OK, ERR_NOT_CONVERGED):
        ctx.check(rc, "hd_eigendecompose")
    return Eig(ctx, h, g.n), lam, res, rc == OK


def spectrum_min(ctx: Context, g: Graph, tol: float = 1e-6, max_restarts: int = 50, seed: int = 7):
    """lambda_n(W) by Lanczos on -W: (estimate, converged)."""
    lam = f64()
    rc = lib().hd_spectrum_min(ctx.handle, g.handle, tol, max_restarts, seed, C.byref(lam))
    if rc not in (OK, ERR_NOT_CONVERGED):
        ctx.check(rc, "hd_spectrum_min")
    return lam.value, rc == OK


def cg_bound(mode, alpha: float, lam_next: float, lam_min: float, tol: float):
    """(kappa, iterations for an A-norm reduction by tol, iterations bounding
    the residual stopping rule) from Eq. 21-23."""
    if isinstance(mode, str):
        mode = MODES[mode]
    k, ia, ir = f64(), i32(), i32()
    rc = lib().hd_cg_bound(mode, alpha, lam_next, lam_min, tol, C.byref(k), C.byref(ia), C.byref(ir))
    if rc != OK:
        raise HDError(rc, "hd_cg_bound: invalid arguments")
    return k.value, ia.value, ir.value


def convergence_table(lam, lam_min: float, alpha: float, tol: float, ranks, mode="pcg"):
    """Predicted iterations against r (the analysis behind Fig. 1b): for each r
    in `ranks`, lambda_{r+1} is taken from the descending spectrum `lam`."""
    rows = []
    for r in ranks:
        lam_next = 1.0 if r == 0 else float(lam[r])
        kap, ia, ir = cg_bound(mode if r > 0 else "paper", alpha, lam_next, lam_min, tol)
        rows.append({"r": int(r), "lambda_next": lam_next, "kappa": kap, "iters_anorm": ia, "iters_resid": ir})
    return rows


def filter_poly(ctx: Context, g: Graph, eig, y_ptr, y_idx, y_val, coeffs, X=None, ldx=None):
    """x = h(W) y for h(A) = sum_i coeffs[i] A^i via Theorem 2 (Eq. 32);
    X defaults to a new (n x B) device tensor."""
    import torch
    B = len(y_ptr) - 1
    co = np.ascontiguousarray(coeffs, dtype=np.float64)
    yp, yi, yv = (_typed(y_ptr, np.int32, "int32"), _typed(y_idx, np.int32, "int32"),
                  _typed(y_val, np.float32, "float32"))
    if X is None:
        X = torch.empty((g.n, B), dtype=torch.float32, device="cuda")
    ld = ldx if ldx is not None else (X.shape[1] if hasattr(X, "shape") else B)
    ctx.check(lib().hd_filter_poly(ctx.handle, g.handle, eig.handle if eig is not None else None, B, _ptr(yp),
                                   _ptr(yi), _ptr(yv), _ptr(co), len(co), _ptr(X), ld), "hd_filter_poly")
    return X


def query_batch(ctx: Context, g: Graph, eig, mode, y_ptr, y_idx, y_val, alpha: float, tol, max_iter: int,
                X=None, ldx=None, iters=None, relres=None, status=None):
    """Solve B ranking vectors; X defaults to a new (n x B) device tensor.

    Returns (X, iters, relres, status); the per-column arrays are numpy unless
    device tensors were passed in.
    """
    import torch
    B = len(y_ptr) - 1
    y_ptr = _typed(y_ptr, np.int32, "int32")
    y_idx = _typed(y_idx, np.int32, "int32")
    y_val = _typed(y_val, np.float32, "float32")
    if isinstance(mode, str):
        mode = MODES[mode]
    if np.isscalar(tol):
        tol = np.full(B, tol, np.float32)
    if isinstance(tol, np.ndarray):
        tol = np.ascontiguousarray(tol, dtype=np.float32)
    if X is None:
        X = torch.empty((g.n, B), dtype=torch.float32, device=f"cuda:{ctx.device}")
    if ldx is None:
        ldx = X.shape[1] if X.ndim == 2 else B
    iters = np.zeros(B, np.int32) if iters is None else iters
    relres = np.zeros(B, np.float32) if relres is None else relres
    status = np.zeros(B, np.int32) if status is None else status
    rc = lib().hd_query_batch(ctx.handle, g.handle, eig.handle if eig is not None else None, mode, B, _ptr(y_ptr),
                              _ptr(y_idx), _ptr(y_val), alpha, _ptr(tol), max_iter, _ptr(X), ldx, _ptr(iters),
                              _ptr(relres), _ptr(status))
    ctx.check(rc, "hd_query_batch")
    return X, iters, relres, status


def temporal_truncated(ctx: Context, g: Graph, sl_ptr, sl_idx, y_ptr, y_idx, y_val, alpha: float, tol,
                       max_iter: int, X=None):
    """Temporal† (Sec. 3.1): CG on each query's shortlist subgraph.  Returns
    (X, iters, relres, status) with X (s_max x B) holding shortlist-position
    scores: X[t, j] belongs to sl_idx[sl_ptr[j] + t]."""
    import torch
    B = len(sl_ptr) - 1
    slp = np.ascontiguousarray(sl_ptr, np.int32)
    smax = int(np.max(np.diff(slp)))
    if np.isscalar(tol):
        tol = np.full(B, tol, np.float32)
    tol = np.ascontiguousarray(tol, dtype=np.float32)
    if X is None:
        X = torch.empty((smax, B), dtype=torch.float32, device=f"cuda:{ctx.device}")
    iters = np.zeros(B, np.int32)
    relres = np.zeros(B, np.float32)
    status = np.zeros(B, np.int32)
    sli = _typed(sl_idx, np.int32, "int32")
    y_ptr = _typed(y_ptr, np.int32, "int32")
    y_idx = _typed(y_idx, np.int32, "int32")
    y_val = _typed(y_val, np.float32, "float32")
    ctx.check(lib().hd_temporal_truncated(ctx.handle, g.handle, B, _ptr(slp), _ptr(sli), _ptr(y_ptr), _ptr(y_idx),
                                          _ptr(y_val), alpha, _ptr(tol), max_iter, _ptr(X), X.shape[1], _ptr(iters),
                                          _ptr(relres), _ptr(status)), "hd_temporal_truncated")
    return X, iters, relres, status


def rank_shortlists(ctx: Context, X, sl_ptr, sl_idx, K: int):
    """Top-K of truncated scores (s_max x B), mapped back to database ids:
    (ids, scores), each B x K; ids are -1 past a shortlist's end."""
    slp = np.asarray(sl_ptr, np.int64)
    sli = np.asarray(sl_idx)
    pos, sc = rank(ctx, X, K)
    ids = np.full(pos.shape, -1, np.int64)
    for j in range(pos.shape[0]):
        s = slp[j + 1] - slp[j]
        ok = (pos[j] >= 0) & (pos[j] < s)
        ids[j, ok] = sli[slp[j] + pos[j, ok]]
    return ids, sc


def rank(ctx: Context, X, K, Kmax: int | None = None, pool: int = 0, n: int | None = None, idx=None, score=None):
    """Per-column top-K of device scores X (n x B): (idx, score), each B x Kmax."""
    B = X.shape[1]
    ldx = X.stride(0)
    n = X.shape[0] if n is None else n
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.int32), (B,)))
    Kmax = int(K.max()) if Kmax is None else Kmax
    if idx is None:
        idx = np.empty((B, Kmax), np.int32)
        score = np.empty((B, Kmax), np.float32)
    size = (lambda a: a.size if isinstance(a, np.ndarray) else a.numel())
    if size(idx) < B * Kmax or size(score) < B * Kmax:
        raise ValueError("idx/score buffers must hold B x Kmax entries")
    ctx.check(lib().hd_rank(ctx.handle, _ptr(X), n, B, ldx, _ptr(K), Kmax, pool, _ptr(idx), _ptr(score)), "hd_rank")
    return idx, score


class ReqStats(C.Structure):
    _fields_ = [("submit_s", C.c_double), ("admit_s", C.c_double), ("done_s", C.c_double),
                ("iters", C.c_int32), ("status", C.c_int32), ("relres", C.c_float), ("slot", C.c_int32)]


class Server:
    """Continuous-batching server (hd_serve_*): submit requests, step, poll."""

    def __init__(self, ctx: Context, g: Graph, eig=None, mode="pcg", alpha: float = 0.99, max_slots: int = 64,
                 mem_budget: int = 0, max_iter: int = 1000, Kmax: int = 1000):
        self.ctx = ctx
        self.Kmax = Kmax
        self._h = vp()
        m = MODES[mode] if isinstance(mode, str) else mode
        ctx.check(lib().hd_serve_open(ctx.handle, g.handle, eig.handle if eig is not None else None, m, alpha,
                                      max_slots, mem_budget, max_iter, Kmax, C.byref(self._h)), "hd_serve_open")
        ctx._servers.add(self)
        self.slots = int(lib().hd_serve_slots(self._h))

    def submit(self, idx, val, tol: float, K: int) -> int:
        idx = np.ascontiguousarray(idx, np.int32)
        val = np.ascontiguousarray(val, np.float32)
        t = u64()
        self.ctx.check(lib().hd_serve_submit(self._h, idx.size, _ptr(idx), _ptr(val), tol, K, C.byref(t)),
                       "hd_serve_submit")
        return t.value

    def step(self, iters: int = 1) -> int:
        busy = i32()
        self.ctx.check(lib().hd_serve_step(self._h, iters, C.byref(busy)), "hd_serve_step")
        return busy.value

    def poll(self, ticket: int, K: int):
        """None while pending, else (ids, scores, stats dict)."""
        ids = np.empty(max(K, 1), np.int32)
        sc = np.empty(max(K, 1), np.float32)
        st = ReqStats()
        rc = lib().hd_serve_poll(self._h, ticket, _ptr(ids), _ptr(sc), C.byref(st))
        if rc == PENDING:
            return None
        self.ctx.check(rc, "hd_serve_poll")
        stats = {f: getattr(st, f) for f, _ in ReqStats._fields_}
        return ids[:K], sc[:K], stats

    def cancel(self, ticket: int):
        """Withdraw a queued or running request (it then polls with status 4, no ranking)."""
        self.ctx.check(lib().hd_serve_cancel(self._h, ticket), "hd_serve_cancel")

    def completed(self, max_tickets: int = 4096):
        """Tickets retired since the last call (poll them for their results)."""
        buf = np.empty(max_tickets, np.uint64)
        cnt = i32()
        self.ctx.check(lib().hd_serve_completed(self._h, _ptr(buf), max_tickets, C.byref(cnt)), "hd_serve_completed")
        return [int(t) for t in buf[:cnt.value]]

    def close(self):
        if self._h:
            lib().hd_serve_close(self._h)
            self._h = vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
