"""CPU oracle for ML(n)BiCGStab — TEST INFRASTRUCTURE ONLY.

A ctypes front end to the plain C oracle in ``mlb_oracle.c`` (FP64 and
complex128, sequential loops).  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import this package; the CUDA
library and its Python binding never do.

Matrices are passed duck-typed: any object with ``row_ptr`` (int64),
``col`` (int32), ``val`` (float64 or complex128) and ``n_rows``.

Functions
    gn, rn              §2 index functions
    spmv                y = A x
    ahq                 F = A^H Q(:, :m)                (Algorithm 4.1, step 2)
    q_gauss             shadow vectors from the library's documented
                        SplitMix64 + Box–Muller generator
    mlbicgstabt         one call of Algorithm 7.1 (M = I, a diagonal M, or
                        ILU(0) factors)
    ilu0                ILU(0) factors of A in A's pattern
    minv, minv_h        M^{-1} v and M^{-H} v
    solve               repeated calls from the current x until the true
                        residual meets tol (restart wrapper, not in the paper)
    load_par            the multi-core build (pass as ``lib=``)
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

_LIB = None
OP_NAMES = ("matvec", "dot", "saxpy", "scale", "norm")


class _Result(C.Structure):
    _fields_ = [("iter", C.c_int64), ("flag", C.c_int32), ("j", C.c_int32),
                ("i", C.c_int32), ("pad", C.c_int32), ("err", C.c_double),
                ("ops", C.c_int64 * 5)]


def load(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` selects an
    alternative build, e.g. a deliberately broken one in a test."""
    global _LIB
    if path is None and _LIB is not None:
        return _LIB
    lib = C.CDLL(path or _build.build())
    P = C.c_void_p
    lib.orc_gn.restype = C.c_int64
    lib.orc_gn.argtypes = [C.c_int64, C.c_int64]
    lib.orc_rn.restype = C.c_int64
    lib.orc_rn.argtypes = [C.c_int64, C.c_int64]
    lib.orc_normal_at.restype = C.c_double
    lib.orc_normal_at.argtypes = [C.c_uint64, C.c_uint64]
    lib.orc_qgauss.restype = None
    lib.orc_qgauss.argtypes = [C.c_uint64, C.c_int64, C.c_int32, C.c_int32, P]
    for sfx in ("d", "z"):
        f = getattr(lib, f"orc_spmv_{sfx}")
        f.restype = None
        f.argtypes = [C.c_int64, P, P, P, P, P]
        f = getattr(lib, f"orc_ahq_{sfx}")
        f.restype = None
        f.argtypes = [C.c_int64, P, P, P, C.c_int32, P, P]
        f = getattr(lib, f"orc_mlbicgstabt_{sfx}")
        f.restype = C.c_int
        f.argtypes = [C.c_int64, P, P, P, C.c_int32, P, P, P, C.c_int64,
                      C.c_double, C.c_double, P, P, P, C.POINTER(_Result),
                      P, C.c_int64, P, C.c_int64, P, C.c_int64, P, C.c_int64]
        f = getattr(lib, f"orc_ilu0_{sfx}")
        f.restype = C.c_int
        f.argtypes = [C.c_int64, P, P, P, P, P]
        f = getattr(lib, f"orc_minv_{sfx}")
        f.restype = None
        f.argtypes = [C.c_int64, P, P, P, P, P, P, P]
        f = getattr(lib, f"orc_minv_h_{sfx}")
        f.restype = None
        f.argtypes = [C.c_int64, P, P, P, P, P, P]
    if path is None:
        _LIB = lib
    return lib


_LIB_PAR = None


def load_par():
    """The multi-core build of the oracle (OpenMP; inner products and norms
    over fixed 1024-entry blocks, so results do not depend on the thread
    count).  Pass it as ``lib=`` to any function here; ``par_threads``
    sets its thread count."""
    global _LIB_PAR
    if _LIB_PAR is None:
        _build.build()
        lib = load(_build.OUT_PAR)
        lib.orc_par_set_threads.restype = None
        lib.orc_par_set_threads.argtypes = [C.c_int32]
        lib.orc_par_max_threads.restype = C.c_int32
        lib.orc_par_max_threads.argtypes = []
        _LIB_PAR = lib
    return _LIB_PAR


def par_threads(t: int | None = None) -> int:
    """Set (when t is given) and return the multi-core oracle's threads."""
    lib = load_par()
    if t is not None:
        lib.orc_par_set_threads(int(t))
    return int(lib.orc_par_max_threads())


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _mat(A, complex_: bool):
    dt = np.complex128 if complex_ else np.float64
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    av = np.ascontiguousarray(A.val, dtype=dt)
    return rp, ci, av


def gn(n: int, k: int, lib=None) -> int:
    return int((lib or load()).orc_gn(n, k))


def rn(n: int, k: int, lib=None) -> int:
    return int((lib or load()).orc_rn(n, k))


def normal_at(seed: int, t: int, lib=None) -> float:
    return float((lib or load()).orc_normal_at(seed, t))


def q_gauss(seed: int, N: int, n: int, complex_: bool = False,
            lib=None) -> np.ndarray:
    """N x n shadow matrix (Fortran order) from the documented generator."""
    lib = lib or load()
    if complex_:
        buf = np.empty(2 * N * n, dtype=np.float64)
        lib.orc_qgauss(seed, N, n, 1, _ptr(buf))
        return buf.view(np.complex128).reshape((N, n), order="F")
    buf = np.empty(N * n, dtype=np.float64)
    lib.orc_qgauss(seed, N, n, 0, _ptr(buf))
    return buf.reshape((N, n), order="F")


class Bound:
    """The functions of this package bound to one loaded build (used to run
    the pins against deliberately broken copies of the oracle)."""

    def __init__(self, lib):
        self.lib = lib

    def __getattr__(self, name):
        fn = globals()[name]
        return lambda *a, **k: fn(*a, lib=self.lib, **k)


def spmv(A, x, lib=None) -> np.ndarray:
    cplx = np.iscomplexobj(A.val) or np.iscomplexobj(x)
    dt = np.complex128 if cplx else np.float64
    rp, ci, av = _mat(A, cplx)
    x = np.ascontiguousarray(x, dtype=dt)
    y = np.empty(A.n_rows, dtype=dt)
    fn = (lib or load()).orc_spmv_z if cplx else (lib or load()).orc_spmv_d
    fn(A.n_rows, _ptr(rp), _ptr(ci), _ptr(av), _ptr(x), _ptr(y))
    return y


def ahq(A, Q, m: int | None = None, lib=None) -> np.ndarray:
    """F = A^H Q(:, :m) (column-major N x m)."""
    cplx = np.iscomplexobj(A.val) or np.iscomplexobj(Q)
    dt = np.complex128 if cplx else np.float64
    N = A.n_rows
    m = Q.shape[1] if m is None else m
    rp, ci, av = _mat(A, cplx)
    Qf = np.asfortranarray(Q, dtype=dt)
    F = np.empty((N, m), dtype=dt, order="F")
    fn = (lib or load()).orc_ahq_z if cplx else (lib or load()).orc_ahq_d
    fn(N, _ptr(rp), _ptr(ci), _ptr(av), m, _ptr(Qf), _ptr(F))
    return F


@dataclasses.dataclass
class Result:
    x: np.ndarray
    iter: int
    flag: int
    err: float
    j: int
    i: int
    ops: dict
    err_hist: np.ndarray | None = None
    x_hist: np.ndarray | None = None
    blk_ops: np.ndarray | None = None
    trace: np.ndarray | None = None
    outer: int = 0
    true_relres: float | None = None


class IluError(ValueError):
    """ILU(0) does not exist for this input (code -1: a row unsorted or
    without a diagonal entry; -3: a zero pivot)."""


@dataclasses.dataclass
class Ilu:
    """ILU(0) factors in the pattern of A: ``lu`` holds L's strictly lower
    entries (unit diagonal implied) and U's entries, ``dpos[r]`` the
    position of row r's diagonal."""
    lu: np.ndarray
    dpos: np.ndarray


def ilu0(A, lib=None) -> Ilu:
    """ILU(0) of A (Saad, Algorithm 10.4; the paper's experiments use ILU(0),
    §5).  Column indices must increase within each row."""
    lib = lib or load()
    cplx = np.iscomplexobj(A.val)
    rp, ci, av = _mat(A, cplx)
    lu = np.empty_like(av)
    dpos = np.empty(A.n_rows, dtype=np.int64)
    fn = lib.orc_ilu0_z if cplx else lib.orc_ilu0_d
    rc = fn(A.n_rows, _ptr(rp), _ptr(ci), _ptr(av), _ptr(lu), _ptr(dpos))
    if rc == -2:
        raise MemoryError("oracle allocation failed")
    if rc != 0:
        raise IluError(rc)
    return Ilu(lu=lu, dpos=dpos)


def _pc_args(A, cplx, mdiag, ilu):
    dt = np.complex128 if cplx else np.float64
    md = None if mdiag is None else np.ascontiguousarray(mdiag, dtype=dt)
    if md is not None and md.shape != (A.n_rows,):
        raise ValueError("mdiag must hold N entries")
    if md is not None and ilu is not None:
        raise ValueError("give mdiag or ilu, not both")
    lu = None if ilu is None else np.ascontiguousarray(ilu.lu, dtype=dt)
    dp = None if ilu is None else np.ascontiguousarray(ilu.dpos, dtype=np.int64)
    return md, lu, dp


def minv(A, v, mdiag=None, ilu=None, lib=None) -> np.ndarray:
    """M^{-1} v for M = diag(mdiag) or M = L U from ``ilu``."""
    lib = lib or load()
    cplx = np.iscomplexobj(A.val) or np.iscomplexobj(v)
    dt = np.complex128 if cplx else np.float64
    rp, ci, _ = _mat(A, cplx)
    md, lu, dp = _pc_args(A, cplx, mdiag, ilu)
    src = np.ascontiguousarray(v, dtype=dt)
    dst = np.empty_like(src)
    fn = lib.orc_minv_z if cplx else lib.orc_minv_d
    fn(A.n_rows, _ptr(rp), _ptr(ci), _ptr(md), _ptr(lu), _ptr(dp), _ptr(src), _ptr(dst))
    return dst


def minv_h(A, v, mdiag=None, ilu=None, lib=None) -> np.ndarray:
    """M^{-H} v for M = diag(mdiag) or M = L U from ``ilu``."""
    lib = lib or load()
    cplx = np.iscomplexobj(A.val) or np.iscomplexobj(v)
    dt = np.complex128 if cplx else np.float64
    rp, ci, _ = _mat(A, cplx)
    md, lu, dp = _pc_args(A, cplx, mdiag, ilu)
    w = np.array(v, dtype=dt, copy=True)
    fn = lib.orc_minv_h_z if cplx else lib.orc_minv_h_d
    fn(A.n_rows, _ptr(rp), _ptr(ci), _ptr(md), _ptr(lu), _ptr(dp), _ptr(w))
    return w


def mlbicgstabt(A, b, x0, Q, maxit: int, tol: float, kappa: float = 0.0,
                err_hist: bool = False, x_hist: int = 0, blk_ops: int = 0,
                trace: bool = False, lib=None, mdiag=None, ilu=None) -> Result:
    """One call of ML(n)BiCGStabt (Algorithm 7.1) from x0; ``mdiag`` is the
    diagonal of the preconditioner M, ``ilu`` its ILU(0) factors (from
    ``ilu0``); neither: M = I."""
    lib = lib or load()
    cplx = (np.iscomplexobj(A.val) or np.iscomplexobj(b)
            or np.iscomplexobj(Q) or np.iscomplexobj(x0))
    dt = np.complex128 if cplx else np.float64
    N = A.n_rows
    n = Q.shape[1]
    rp, ci, av = _mat(A, cplx)
    Qf = np.asfortranarray(Q, dtype=dt)
    b = np.ascontiguousarray(b, dtype=dt)
    x = np.array(x0, dtype=dt, copy=True)
    md, lu, dp = _pc_args(A, cplx, mdiag, ilu)
    cap = int(maxit) + 1
    eh = np.full(cap, np.nan) if err_hist else None
    xh = np.zeros((x_hist, N), dtype=dt) if x_hist else None
    bo = np.zeros((blk_ops, 5), dtype=np.int64) if blk_ops else None
    tr = np.zeros((cap, 2), dtype=np.int32) if trace else None
    res = _Result()
    fn = lib.orc_mlbicgstabt_z if cplx else lib.orc_mlbicgstabt_d
    rc = fn(N, _ptr(rp), _ptr(ci), _ptr(av), n, _ptr(Qf), _ptr(b), _ptr(x),
            int(maxit), float(tol), float(kappa), _ptr(md), _ptr(lu), _ptr(dp), C.byref(res),
            _ptr(eh), cap if eh is not None else 0,
            _ptr(xh), x_hist, _ptr(bo), blk_ops,
            _ptr(tr), cap if tr is not None else 0)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    it = int(res.iter)
    return Result(
        x=x, iter=it, flag=int(res.flag), err=float(res.err), j=int(res.j),
        i=int(res.i), ops=dict(zip(OP_NAMES, [int(v) for v in res.ops])),
        err_hist=None if eh is None else eh[:it + 1],
        x_hist=None if xh is None else xh[:min(it, x_hist)],
        blk_ops=bo, trace=None if tr is None else tr[:it])


def jacobi_diag(A, lib=None):
    """diag(A) as a vector: the Jacobi preconditioner M = diag(A)
    (duplicate entries of a row are summed, as in the product A x)."""
    d = np.zeros(A.n_rows, dtype=A.val.dtype)
    for r in range(A.n_rows):
        for k in range(A.row_ptr[r], A.row_ptr[r + 1]):
            if A.col[k] == r:
                d[r] += A.val[k]
    return d


def true_relres(A, b, x, lib=None) -> float:
    """||b - A x||_2 / ||b||_2 with ||b|| replaced by 1 when b = 0."""
    r = np.asarray(b) - spmv(A, x, lib=lib)
    bn = float(np.sqrt(np.sum(np.abs(np.asarray(b)) ** 2)))
    return float(np.sqrt(np.sum(np.abs(r) ** 2))) / (bn if bn != 0.0 else 1.0)


def solve(A, b, x0, Q, maxit: int, tol: float, kappa: float = 0.0,
          max_outer: int = 10, lib=None, mdiag=None, ilu=None) -> Result:
    """Call ``mlbicgstabt`` again from the current x while its recursive
    residual met ``tol`` but the true residual ||b - A x||/||b|| did not;
    each new call recomputes r = b - A x and returns at once (iter 0) when
    the true residual already meets ``tol``.  Iterations accumulate against
    one ``maxit`` budget.  This restart rule is the library's, not the
    paper's: the paper stops on the recursive residual (§5)."""
    x = np.array(x0, copy=True)
    total = 0
    outer = 0
    res = None
    while True:
        res = mlbicgstabt(A, b, x, Q, maxit - total, tol, kappa, lib=lib, mdiag=mdiag, ilu=ilu)
        x = res.x
        total += res.iter
        if res.flag != 0 or res.iter == 0 or total >= maxit:
            break
        if outer >= max_outer:
            break
        outer += 1
    res.iter = total
    res.outer = outer
    res.x = x
    res.true_relres = true_relres(A, b, x, lib=lib)
    return res
