"""Python binding of the C ABI in include/mlbicgstab.h (ctypes).

Argument marshalling only: every step of a solve runs in the CUDA library
``libmlbicgstab.so``.  The functions keep the C names
(``mlbicgstab_create``, ``mlbicgstab_solve``, ...).  Arrays may be NumPy
arrays (host memory) or CUDA tensors of PyTorch (device memory; the tensor
only supplies memory and its pointer).  There is no CPU fallback: if the
library has not been built, ``load`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmlbicgstab.so")

MLB_OK, MLB_ERR_ARG, MLB_ERR_CUDA, MLB_ERR_OOM, MLB_ERR_TIMEOUT, MLB_ERR_UNSUPPORTED = range(6)
MLB_F64, MLB_F32, MLB_C128, MLB_C64 = 0, 1, 2, 3
MLB_PREC_FP64, MLB_PREC_FP32_REFINED = 0, 1
MLB_PRECOND_NONE, MLB_PRECOND_JACOBI, MLB_PRECOND_ILU0, MLB_PRECOND_ILU0_MC = 0, 1, 2, 3

# Every symbol the header declares (checked against the header by a test).
EXPORTS = (
    "mlbicgstab_default_options", "mlbicgstab_create", "mlbicgstab_solve",
    "mlbicgstab_solve_batch", "mlbicgstab_spmv_qdot", "mlbicgstab_get_Q",
    "mlbicgstab_info", "mlbicgstab_destroy", "mlbicgstab_strerror",
    "mlbicgstab_selftest_barrier_timeout", "mlbicgstab_spmv_qdot_noalloc",
    "mlbicgstab_set_n", "mlbicgstab_next_n", "mlbicgstab_solve_sequence",
    "mlbicgstab_autotune", "mlbicgstab_spmv_qdot_async", "mlbicgstab_get_perm",
    "mlbicgstab_autotune_batch", "mlbicgstab_get_tuning", "mlbicgstab_set_tuning",
    "mlbicgstab_batch_plan",
)


class mlb_matrix(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("values", C.c_void_p), ("dtype", C.c_int32),
                ("block", C.c_int32)]


class mlb_options(C.Structure):
    _fields_ = [("n", C.c_int32), ("precision", C.c_int32),
                ("q_seed", C.c_uint64), ("Q", C.c_void_p),
                ("kappa", C.c_double), ("max_outer", C.c_int32),
                ("grid", C.c_int32), ("inner_tol", C.c_double),
                ("inner_maxit", C.c_int64), ("stream", C.c_void_p),
                ("timeout_ns", C.c_int64), ("precond", C.c_int32),
                ("reserved0", C.c_int32)]


class mlb_result(C.Structure):
    _fields_ = [("flag", C.c_int32), ("j", C.c_int32), ("i", C.c_int32),
                ("status", C.c_int32), ("iter", C.c_int64),
                ("spmv", C.c_int64), ("outer", C.c_int64),
                ("err", C.c_double), ("true_relres", C.c_double),
                ("kernel_ms", C.c_double), ("bytes", C.c_double),
                ("ops", C.c_int64 * 5), ("flops", C.c_double),
                ("ctas", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("ops", "reserved")}
        d["ops"] = dict(zip(("matvec", "dot", "saxpy", "scale", "norm"),
                            [int(v) for v in self.ops]))
        return d


class mlb_info(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("nnz", C.c_int64), ("n", C.c_int32),
                ("dtype", C.c_int32), ("precision", C.c_int32),
                ("grid", C.c_int32), ("block", C.c_int32),
                ("precond", C.c_int32), ("nnz_padded", C.c_int64),
                ("device_bytes", C.c_int64), ("n_active", C.c_int32),
                ("ilu_levels", C.c_int32), ("qd_kernel_ms", C.c_double),
                ("entry_values", C.c_int32), ("reserved2", C.c_int32)]


class mlb_tune_result(C.Structure):
    _fields_ = [("grid", C.c_int32), ("spt_cap", C.c_int32), ("us_per_iter", C.c_double),
                ("default_us_per_iter", C.c_double), ("trials", C.c_int32), ("from_cache", C.c_int32),
                ("qd_fused", C.c_int32), ("reserved", C.c_int32), ("qd_us", C.c_double),
                ("qd_default_us", C.c_double)]


class mlb_tuning(C.Structure):
    _fields_ = [("grid", C.c_int32), ("spt_cap", C.c_int32), ("batch_spt_cap", C.c_int32),
                ("batch_team", C.c_int32), ("qd_fused", C.c_int32)]


class mlb_batch_tune_result(C.Structure):
    _fields_ = [("classes", C.c_int32), ("trials", C.c_int32), ("from_cache", C.c_int32),
                ("team", C.c_int32), ("default_ms", C.c_double), ("tuned_ms", C.c_double)]


class mlb_sequence_options(C.Structure):
    _fields_ = [("n0", C.c_int32), ("step", C.c_int32), ("n_min", C.c_int32),
                ("n_max", C.c_int32)]


class MlbError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (status {code})")


_LIB = None


def load(path: str | None = None):
    """Load the CUDA library.  Raises if it has not been built."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(
            f"{p} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(p)
    P = C.c_void_p
    lib.mlbicgstab_default_options.restype = None
    lib.mlbicgstab_default_options.argtypes = [C.POINTER(mlb_options)]
    lib.mlbicgstab_create.restype = C.c_int
    lib.mlbicgstab_create.argtypes = [C.POINTER(P), C.POINTER(mlb_matrix),
                                      C.POINTER(mlb_matrix), C.POINTER(mlb_options)]
    lib.mlbicgstab_solve.restype = C.c_int
    lib.mlbicgstab_solve.argtypes = [P, P, P, C.c_int32, C.c_double, C.c_int64,
                                     C.POINTER(mlb_result), P, C.c_int64]
    lib.mlbicgstab_solve_batch.restype = C.c_int
    lib.mlbicgstab_solve_batch.argtypes = [P, C.c_int32, P, P, C.c_int32, P, P,
                                           C.POINTER(mlb_result)]
    lib.mlbicgstab_spmv_qdot.restype = C.c_int
    lib.mlbicgstab_spmv_qdot.argtypes = [P, P, P, P]
    lib.mlbicgstab_get_perm.restype = C.c_int
    lib.mlbicgstab_get_perm.argtypes = [P, P]
    lib.mlbicgstab_spmv_qdot_async.restype = C.c_int
    lib.mlbicgstab_spmv_qdot_async.argtypes = [P, C.c_int32, P, P, P]
    lib.mlbicgstab_get_Q.restype = C.c_int
    lib.mlbicgstab_get_Q.argtypes = [P, P]
    lib.mlbicgstab_info.restype = C.c_int
    lib.mlbicgstab_info.argtypes = [P, C.POINTER(mlb_info)]
    lib.mlbicgstab_destroy.restype = None
    lib.mlbicgstab_destroy.argtypes = [P]
    lib.mlbicgstab_strerror.restype = C.c_char_p
    lib.mlbicgstab_strerror.argtypes = [C.c_int]
    lib.mlbicgstab_selftest_barrier_timeout.restype = C.c_int
    lib.mlbicgstab_selftest_barrier_timeout.argtypes = [C.c_int32, C.c_int64]
    lib.mlbicgstab_set_n.restype = C.c_int
    lib.mlbicgstab_set_n.argtypes = [P, C.c_int32]
    lib.mlbicgstab_next_n.restype = C.c_int32
    lib.mlbicgstab_next_n.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_int32,
                                      C.c_int32, C.c_int32]
    lib.mlbicgstab_solve_sequence.restype = C.c_int
    lib.mlbicgstab_solve_sequence.argtypes = [P, C.c_int32, P, P, C.c_int32, P, P,
                                              C.POINTER(mlb_sequence_options),
                                              C.POINTER(mlb_result), P]
    lib.mlbicgstab_autotune.restype = C.c_int
    lib.mlbicgstab_autotune.argtypes = [P, C.c_int32, C.c_int32, C.POINTER(mlb_tune_result)]
    lib.mlbicgstab_batch_plan.restype = C.c_int
    lib.mlbicgstab_batch_plan.argtypes = [P, P, P, C.c_int32, C.c_int32, C.c_int32, P, P,
                                          C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.mlbicgstab_get_tuning.restype = C.c_int
    lib.mlbicgstab_get_tuning.argtypes = [P, C.POINTER(mlb_tuning)]
    lib.mlbicgstab_set_tuning.restype = C.c_int
    lib.mlbicgstab_set_tuning.argtypes = [P, C.POINTER(mlb_tuning)]
    lib.mlbicgstab_autotune_batch.restype = C.c_int
    lib.mlbicgstab_autotune_batch.argtypes = [P, C.c_int32, C.c_double, C.c_int64, C.c_int32,
                                              C.POINTER(mlb_batch_tune_result)]
    lib.mlbicgstab_spmv_qdot_noalloc.restype = C.c_int
    lib.mlbicgstab_spmv_qdot_noalloc.argtypes = [C.c_int64, C.c_int64, P, P, P, C.c_int32,
                                                 P, P, C.c_int64, C.c_int32, P, P, P]
    if path is None:
        _LIB = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().mlbicgstab_strerror(code).decode()
    except ImportError:
        return f"status {code}"


def _check(rc: int, what: str):
    if rc != MLB_OK:
        raise MlbError(rc, what)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, on_device) of a NumPy array or a torch tensor."""
    if a is None:
        return None, 0
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data), 0


class Matrix:
    """Keeps the host arrays of an mlb_matrix alive while it is used.  A
    CSR matrix (row_ptr, col, val, n_rows), or a BSR matrix of 3x3 blocks
    (val of shape (nblocks, 3, 3), row_ptr and col over block rows and
    columns), passed with block = 3."""

    def __init__(self, A):
        cplx = np.iscomplexobj(A.val)
        dt = np.complex128 if cplx else np.float64
        self.rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(A.col, dtype=np.int32)
        block = 3 if np.ndim(A.val) == 3 else 0
        self.val = np.ascontiguousarray(np.asarray(A.val, dtype=dt).reshape(-1))
        self.c = mlb_matrix(int(A.n_rows), int(self.rp[-1]),
                            self.rp.ctypes.data, self.ci.ctypes.data,
                            self.val.ctypes.data, MLB_C128 if cplx else MLB_F64, block)
        self.dtype = self.val.dtype


def mlbicgstab_default_options() -> mlb_options:
    o = mlb_options()
    load().mlbicgstab_default_options(C.byref(o))
    return o


def mlbicgstab_strerror(code: int) -> str:
    return strerror(code)


class Handle:
    """An mlb_handle plus the dtype and size needed to marshal its calls."""

    def __init__(self, ptr, N: int, n: int, dtype):
        self.ptr = ptr
        self.N = N
        self.n = n
        self.dtype = dtype

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self):
        if self.ptr is not None and self.ptr.value:
            load().mlbicgstab_destroy(self.ptr)
        self.ptr = None


def mlbicgstab_create(A, AH=None, n: int = 4, q_seed: int = 0, Q=None,
                      kappa: float = 0.0, precision: int = MLB_PREC_FP64,
                      max_outer: int | None = None, grid: int = 0,
                      inner_tol: float | None = None,
                      inner_maxit: int | None = None, stream=None,
                      timeout_ns: int | None = None,
                      precond: int = MLB_PRECOND_NONE) -> Handle:
    """Create a solver for CSR matrix ``A`` (see mlbicgstab_create in C).
    ``stream``: a torch.cuda.Stream, a raw cudaStream_t integer, or None.
    ``precond``: MLB_PRECOND_NONE, MLB_PRECOND_JACOBI (M = diag(A)),
    MLB_PRECOND_ILU0 (M = the ILU(0) factors of A) or MLB_PRECOND_ILU0_MC
    (the ILU(0) factors of A in a multicolour order)."""
    lib = load()
    M = Matrix(A)
    MH = Matrix(AH) if AH is not None else None
    o = mlbicgstab_default_options()
    o.n = n
    o.precision = precision
    o.q_seed = q_seed
    o.kappa = kappa
    o.grid = grid
    o.precond = precond
    if max_outer is not None:
        o.max_outer = max_outer
    if inner_tol is not None:
        o.inner_tol = inner_tol
    if inner_maxit is not None:
        o.inner_maxit = inner_maxit
    if timeout_ns is not None:
        o.timeout_ns = int(timeout_ns)
    Qh = None
    if Q is not None:
        Qh = np.asfortranarray(Q, dtype=M.dtype)
        if Qh.shape != (A.n_rows, n):
            raise ValueError("Q must be N x n")
        o.Q = Qh.ctypes.data
    if stream is not None:
        o.stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    h = C.c_void_p()
    rc = lib.mlbicgstab_create(C.byref(h), C.byref(M.c),
                               C.byref(MH.c) if MH is not None else None, C.byref(o))
    _check(rc, "mlbicgstab_create")
    return Handle(h, int(A.n_rows), n, M.dtype)


def mlbicgstab_solve(h: Handle, b, x, tol: float, maxit: int,
                     hist_cap: int = 0):
    """Solve in place: ``x`` holds x_0 and receives the solution.  Returns
    (mlb_result, err_hist or None)."""
    pb, db = _ptr(b)
    px, dx = _ptr(x)
    if db != dx:
        raise ValueError("b and x must both be host or both device arrays")
    res = mlb_result()
    hist = np.full(hist_cap, np.nan) if hist_cap else None
    rc = load().mlbicgstab_solve(h.ptr, pb, px, db, float(tol), int(maxit),
                                 C.byref(res),
                                 hist.ctypes.data if hist is not None else None,
                                 int(hist_cap))
    if rc not in (MLB_OK, MLB_ERR_TIMEOUT):
        _check(rc, "mlbicgstab_solve")
    if rc == MLB_ERR_TIMEOUT:
        raise MlbError(rc, "mlbicgstab_solve")
    return res, hist


def mlbicgstab_solve_batch(hs, bs, xs, tols, maxits):
    """Solve several systems in one launch; returns a list of mlb_result."""
    count = len(hs)
    ptrs = (C.c_void_p * count)(*[h.ptr.value for h in hs])
    pb = [_ptr(b) for b in bs]
    px = [_ptr(x) for x in xs]
    on_dev = pb[0][1]
    if any(p[1] != on_dev for p in pb + px):
        raise ValueError("all b and x must be host arrays, or all device arrays")
    bp = (C.c_void_p * count)(*[p[0].value for p in pb])
    xp = (C.c_void_p * count)(*[p[0].value for p in px])
    t = np.ascontiguousarray(tols, dtype=np.float64)
    m = np.ascontiguousarray(maxits, dtype=np.int64)
    res = (mlb_result * count)()
    rc = load().mlbicgstab_solve_batch(ptrs, count, bp, xp, on_dev,
                                       t.ctypes.data, m.ctypes.data, res)
    _check(rc, "mlbicgstab_solve_batch")
    return list(res)


def mlbicgstab_set_n(h: Handle, n: int) -> None:
    """Use the first n shadow vectors in later solves (n <= created n)."""
    _check(load().mlbicgstab_set_n(h.ptr, int(n)), "mlbicgstab_set_n")


def mlbicgstab_next_n(n: int, t_prev: float, t_cur: float, step: int, n_min: int, n_max: int) -> int:
    """The paper's rule for the next n in a sequence of systems (§5)."""
    return int(load().mlbicgstab_next_n(int(n), float(t_prev), float(t_cur), int(step),
                                        int(n_min), int(n_max)))


def mlbicgstab_solve_sequence(hs, bs, xs, tols, maxits, n0: int, step: int, n_min: int, n_max: int):
    """Solve systems one after another with n chosen automatically;
    returns (list of mlb_result, list of the n each system used)."""
    count = len(hs)
    ptrs = (C.c_void_p * count)(*[h.ptr.value for h in hs])
    pb = [_ptr(b) for b in bs]
    px = [_ptr(x) for x in xs]
    on_dev = pb[0][1]
    if any(p[1] != on_dev for p in pb + px):
        raise ValueError("all b and x must be host arrays, or all device arrays")
    bp = (C.c_void_p * count)(*[p[0].value for p in pb])
    xp = (C.c_void_p * count)(*[p[0].value for p in px])
    t = np.ascontiguousarray(tols, dtype=np.float64)
    m = np.ascontiguousarray(maxits, dtype=np.int64)
    so = mlb_sequence_options(int(n0), int(step), int(n_min), int(n_max))
    res = (mlb_result * count)()
    used = np.zeros(count, dtype=np.int32)
    rc = load().mlbicgstab_solve_sequence(ptrs, count, bp, xp, on_dev, t.ctypes.data, m.ctypes.data,
                                          C.byref(so), res, used.ctypes.data)
    _check(rc, "mlbicgstab_solve_sequence")
    return list(res), [int(v) for v in used]


def mlbicgstab_autotune(h: Handle, iters: int = 20, use_cache: bool = True) -> dict:
    """Choose the CTA count and SpMV tile size of a handle, and the columns
    fused into its product's epilogue, by timing."""
    r = mlb_tune_result()
    _check(load().mlbicgstab_autotune(h.ptr, int(iters), 1 if use_cache else 0, C.byref(r)),
           "mlbicgstab_autotune")
    return {f: getattr(r, f) for f, _ in r._fields_ if f != "reserved"}


def mlbicgstab_batch_plan(N, nnz, precond, team: int = 4, slots: int = 152) -> dict:
    """The batch work plan for systems of the given sizes (host only):
    ctas per system, processing order, team count and grid."""
    n = np.ascontiguousarray(N, dtype=np.int64)
    z = np.ascontiguousarray(nnz, dtype=np.int64)
    p = np.ascontiguousarray(precond, dtype=np.int32)
    count = len(n)
    ctas = np.zeros(count, dtype=np.int32)
    order = np.zeros(count, dtype=np.int32)
    nbig, teams, grid = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().mlbicgstab_batch_plan(n.ctypes.data, z.ctypes.data, p.ctypes.data, count, int(team),
                                        int(slots), ctas.ctypes.data, order.ctypes.data, C.byref(nbig),
                                        C.byref(teams), C.byref(grid)), "mlbicgstab_batch_plan")
    return {"ctas": ctas, "order": order, "nbig": nbig.value, "teams": teams.value, "grid": grid.value}


def mlbicgstab_get_tuning(h: Handle) -> dict:
    """The handle's launch configuration (grid, spt_cap, batch_spt_cap, qd_fused)."""
    t = mlb_tuning()
    _check(load().mlbicgstab_get_tuning(h.ptr, C.byref(t)), "mlbicgstab_get_tuning")
    return {f: getattr(t, f) for f, _ in t._fields_}


def mlbicgstab_set_tuning(h: Handle, **kw) -> None:
    """Set fields of the handle's launch configuration (the others kept)."""
    cur = mlbicgstab_get_tuning(h)
    unknown = set(kw) - set(cur)
    if unknown:
        raise TypeError(f"unknown tuning fields {sorted(unknown)}")
    cur.update(kw)
    t = mlb_tuning(**{k: int(v) for k, v in cur.items()})
    _check(load().mlbicgstab_set_tuning(h.ptr, C.byref(t)), "mlbicgstab_set_tuning")


def mlbicgstab_autotune_batch(hs, tol: float = 1e-10, maxit: int = 20000, use_cache: bool = True) -> dict:
    """Choose the batch's team size and the tile cap of each size class of
    handles by timing trial batches (A x = 1 solved to tol)."""
    count = len(hs)
    ptrs = (C.c_void_p * count)(*[h.ptr for h in hs])
    r = mlb_batch_tune_result()
    _check(load().mlbicgstab_autotune_batch(ptrs, count, float(tol), int(maxit), 1 if use_cache else 0,
                                            C.byref(r)), "mlbicgstab_autotune_batch")
    return {f: getattr(r, f) for f, _ in r._fields_}


def mlbicgstab_spmv_qdot(h: Handle, x, y) -> np.ndarray:
    """y = A x and d = Q^H y (x, y CUDA tensors); returns d (host), one
    value per active shadow vector (mlbicgstab_set_n)."""
    px, dx = _ptr(x)
    py, dy = _ptr(y)
    if not (dx and dy):
        raise ValueError("x and y must be CUDA tensors")
    d = np.empty(mlbicgstab_info(h)["n_active"], dtype=h.dtype)
    _check(load().mlbicgstab_spmv_qdot(h.ptr, px, py, d.ctypes.data),
           "mlbicgstab_spmv_qdot")
    return d


def mlbicgstab_spmv_qdot_async(h: Handle, x, y, d) -> None:
    """Enqueue y = A x, d = Q^H y on the handle's stream (no wait).  x, y,
    d are CUDA tensors: x, y float64/complex128 (the handle's FP64 data) or
    float32/complex64 (a refined handle's FP32 copies); d float64 with
    n_active * (2 if complex else 1) + 1 entries (the last one is the
    status word)."""
    import torch
    ptrs = [_ptr(a) for a in (x, y, d)]
    if not all(dv for _, dv in ptrs):
        raise ValueError("x, y, d must be CUDA tensors")
    vt = {torch.float64: MLB_F64, torch.float32: MLB_F32, torch.complex128: MLB_C128,
          torch.complex64: MLB_C64}[x.dtype]
    _check(load().mlbicgstab_spmv_qdot_async(h.ptr, vt, ptrs[0][0], ptrs[1][0], ptrs[2][0]),
           "mlbicgstab_spmv_qdot_async")


def mlbicgstab_spmv_qdot_noalloc(row_ptr, col_idx, values, x, Q, y, d,
                                 stream=None) -> None:
    """Allocation-free y = A x, d = Q^H y.  Every argument is a CUDA tensor:
    CSR arrays (int64, int32, float64/complex128), x and y (N), Q (n x ldq
    row-major, i.e. column q of the shadow matrix is Q[q]), d (n).  Only
    enqueues the work on `stream` (torch.cuda.Stream, raw handle or None)."""
    N = int(row_ptr.numel()) - 1
    nnz = int(col_idx.numel())
    cplx = values.is_complex()
    n, ldq = int(Q.shape[0]), int(Q.shape[1])
    ptrs = [_ptr(a) for a in (row_ptr, col_idx, values, x, Q, y, d)]
    if not all(dv for _, dv in ptrs):
        raise ValueError("all arrays must be CUDA tensors")
    st = None
    if stream is not None:
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = load().mlbicgstab_spmv_qdot_noalloc(
        N, nnz, ptrs[0][0], ptrs[1][0], ptrs[2][0], MLB_C128 if cplx else MLB_F64,
        ptrs[3][0], ptrs[4][0], ldq, n, ptrs[5][0], ptrs[6][0], st)
    _check(rc, "mlbicgstab_spmv_qdot_noalloc")


def mlbicgstab_get_Q(h: Handle) -> np.ndarray:
    out = np.empty((h.N, h.n), dtype=h.dtype, order="F")
    _check(load().mlbicgstab_get_Q(h.ptr, out.ctypes.data), "mlbicgstab_get_Q")
    return out


def mlbicgstab_get_perm(h: Handle) -> np.ndarray:
    """Row order of the handle's system (new row r = caller's row out[r])."""
    out = np.empty(h.N, dtype=np.int32)
    _check(load().mlbicgstab_get_perm(h.ptr, out.ctypes.data), "mlbicgstab_get_perm")
    return out


def mlbicgstab_info(h: Handle) -> dict:
    info = mlb_info()
    _check(load().mlbicgstab_info(h.ptr, C.byref(info)), "mlbicgstab_info")
    return {f: getattr(info, f) for f, _ in info._fields_}


def mlbicgstab_destroy(h: Handle):
    h.destroy()


def mlbicgstab_selftest_barrier_timeout(grid: int, timeout_ns: int) -> int:
    return int(load().mlbicgstab_selftest_barrier_timeout(grid, int(timeout_ns)))
