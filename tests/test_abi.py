"""The C-ABI library builds, loads and exports every symbol the header
declares; struct layouts of the binding match the C compiler's; argument
validation answers before any GPU work (no compute calls here)."""
from __future__ import annotations

import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1106_3678_gb300 import build as B
from paper_1106_3678_gb300 import mlbicgstab as M
from paper_1106_3678_gb300 import workloads as W

HEADER = os.path.join(B.ROOT, "include", "mlbicgstab.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(mlbicgstab_\w+)\s*\(", text))


def test_header_and_binding_agree():
    assert _declared() == set(M.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], check=True,
                         capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if l.strip()}
    for name in _declared():
        assert name in syms, name
        assert hasattr(lib, name)


def test_struct_layout_matches_c_compiler(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(f'''
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mlb_matrix), sizeof(mlb_options),
         sizeof(mlb_result), sizeof(mlb_info), sizeof(mlb_sequence_options), sizeof(mlb_tune_result),
         sizeof(mlb_batch_tune_result), sizeof(mlb_tuning));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", offsetof(mlb_options, stream),
         offsetof(mlb_options, timeout_ns), offsetof(mlb_result, ops),
         offsetof(mlb_options, precond), offsetof(mlb_info, precond),
         offsetof(mlb_info, n_active), offsetof(mlb_info, qd_kernel_ms),
         offsetof(mlb_result, flops), offsetof(mlb_result, ctas), offsetof(mlb_tune_result, qd_us),
         offsetof(mlb_batch_tune_result, tuned_ms));
  return 0;
}}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(prog), "-o", str(exe)], check=True)
    sizes, offs = subprocess.run([str(exe)], check=True, capture_output=True,
                                 text=True).stdout.split("\n")[:2]
    assert [int(v) for v in sizes.split()] == [
        C.sizeof(M.mlb_matrix), C.sizeof(M.mlb_options),
        C.sizeof(M.mlb_result), C.sizeof(M.mlb_info), C.sizeof(M.mlb_sequence_options),
        C.sizeof(M.mlb_tune_result), C.sizeof(M.mlb_batch_tune_result), C.sizeof(M.mlb_tuning)]
    assert [int(v) for v in offs.split()] == [
        M.mlb_options.stream.offset, M.mlb_options.timeout_ns.offset,
        M.mlb_result.ops.offset, M.mlb_options.precond.offset,
        M.mlb_info.precond.offset, M.mlb_info.n_active.offset, M.mlb_info.qd_kernel_ms.offset,
        M.mlb_result.flops.offset, M.mlb_result.ctas.offset, M.mlb_tune_result.qd_us.offset,
        M.mlb_batch_tune_result.tuned_ms.offset]


def test_strerror_and_defaults(lib):
    assert M.strerror(M.MLB_OK) == "success"
    assert "timed out" in M.strerror(M.MLB_ERR_TIMEOUT)
    assert M.strerror(99) == "unknown status code"
    o = M.mlbicgstab_default_options()
    assert (o.n, o.precision, o.max_outer, o.grid) == (4, 0, 10, 0)
    assert o.timeout_ns == 2_000_000_000 and o.Q is None


def _raw_create(lib, A, **kw):
    Mx = M.Matrix(A)
    o = M.mlbicgstab_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    h = C.c_void_p()
    rc = lib.mlbicgstab_create(C.byref(h), C.byref(Mx.c), None, C.byref(o))
    return rc, h


def test_invalid_arguments_are_rejected_before_gpu_work(lib):
    A = W.cd2d(4)
    h = C.c_void_p()
    assert lib.mlbicgstab_create(C.byref(h), None, None, None) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_create(None, None, None, None) == M.MLB_ERR_ARG
    assert _raw_create(lib, A, n=0)[0] == M.MLB_ERR_ARG
    assert _raw_create(lib, A, n=65)[0] == M.MLB_ERR_ARG
    assert _raw_create(lib, A, kappa=-1.0)[0] == M.MLB_ERR_ARG
    assert _raw_create(lib, A, precision=7)[0] == M.MLB_ERR_ARG
    assert _raw_create(lib, A, precond=5)[0] == M.MLB_ERR_ARG
    assert _raw_create(lib, A, precond=4)[0] == M.MLB_ERR_ARG
    # refined mode: the reliable-update factor lies in (0, 1), the inner
    # iteration cap is positive
    assert _raw_create(lib, A, precision=1, inner_tol=0.0)[0] == M.MLB_ERR_ARG
    assert _raw_create(lib, A, precision=1, inner_tol=1.0)[0] == M.MLB_ERR_ARG
    assert _raw_create(lib, A, precision=1, inner_maxit=0)[0] == M.MLB_ERR_ARG
    assert _raw_create(lib, A, reserved0=1)[0] == M.MLB_ERR_ARG
    # storage: CSR (block 0 or 1) or BSR(3); BSR needs nrows divisible by 3
    # and block columns below nrows / 3
    Mx = M.Matrix(A)
    Mx.c.block = 2
    assert lib.mlbicgstab_create(C.byref(C.c_void_p()), C.byref(Mx.c), None, None) == M.MLB_ERR_ARG
    Bk = W.reservoir_bsr3(2, 2, 2)
    Mb = M.Matrix(Bk)
    assert Mb.c.block == 3 and Mb.c.nnz == Bk.nblocks
    Mb.c.nrows = Bk.n_rows + 1
    assert lib.mlbicgstab_create(C.byref(C.c_void_p()), C.byref(Mb.c), None, None) == M.MLB_ERR_ARG
    Mb = M.Matrix(Bk)
    Mb.ci[0] = Bk.n_cells
    assert lib.mlbicgstab_create(C.byref(C.c_void_p()), C.byref(Mb.c), None, None) == M.MLB_ERR_ARG
    bad = W.CSR(A.row_ptr.copy(), A.col.copy(), A.val.copy(), A.n_rows)
    bad.col[3] = A.n_rows          # column out of range
    assert _raw_create(lib, bad)[0] == M.MLB_ERR_ARG
    bad = W.CSR(A.row_ptr.copy(), A.col.copy(), A.val.copy(), A.n_rows)
    bad.row_ptr[5], bad.row_ptr[6] = bad.row_ptr[6], bad.row_ptr[5]  # not monotone
    assert _raw_create(lib, bad)[0] == M.MLB_ERR_ARG
    Mx = M.Matrix(A)
    Mx.c.nnz = A.nnz + 1           # nnz disagrees with row_ptr[N]
    assert lib.mlbicgstab_create(C.byref(h), C.byref(Mx.c), None, None) == M.MLB_ERR_ARG
    res = M.mlb_result()
    assert lib.mlbicgstab_solve(None, None, None, 0, 1e-10, 10, C.byref(res),
                                None, 0) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_solve_batch(None, 0, None, None, 0, None, None,
                                      None) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_selftest_barrier_timeout(0, 1000) == M.MLB_ERR_ARG
    lib.mlbicgstab_destroy(None)   # accepted


def test_no_cpu_fallback_without_a_device(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    rc, _ = _raw_create(lib, W.cd2d(4))
    assert rc == M.MLB_ERR_CUDA
    with pytest.raises(M.MlbError):
        M.mlbicgstab_create(W.cd2d(4))


def test_binding_refuses_to_run_without_library(tmp_path):
    with pytest.raises(ImportError):
        M.load(str(tmp_path / "missing.so"))
    x = np.zeros(3)
    assert M._ptr(x)[1] == 0


def test_next_n_rule_of_section_5(lib):
    """§5 ("Choice of n"): a faster current solve (t_prev > t_cur) moves n
    up by `step`, otherwise down, clamped to [n_min, n_max]; invalid
    arguments give -1.  A host function: no device involved."""
    nn = M.mlbicgstab_next_n
    assert nn(4, 2.0, 1.0, 2, 1, 16) == 6      # faster -> increase
    assert nn(4, 1.0, 2.0, 2, 1, 16) == 2      # slower -> decrease
    assert nn(4, 1.0, 1.0, 2, 1, 16) == 2      # equal counts as "otherwise"
    assert nn(15, 2.0, 1.0, 4, 1, 16) == 16    # clamped above
    assert nn(2, 1.0, 2.0, 4, 1, 16) == 1      # clamped below
    assert nn(4, 2.0, 1.0, 0, 1, 16) == 4      # step 0 keeps n
    assert nn(4, 2.0, 1.0, -1, 1, 16) == -1
    assert nn(0, 2.0, 1.0, 1, 1, 16) == -1
    assert nn(20, 2.0, 1.0, 1, 1, 16) == -1
    assert nn(4, 2.0, 1.0, 1, 5, 3) == -1
    # a sequence of times drives n as the rule says
    n, seq = 4, []
    times = [5.0, 4.0, 3.0, 3.5, 2.0, 2.5]
    for k in range(1, len(times)):
        n = nn(n, times[k - 1], times[k], 2, 2, 8)
        seq.append(n)
    assert seq == [6, 8, 6, 8, 6]


def test_sequence_and_set_n_validate_before_gpu(lib):
    """Invalid sequence arguments are rejected before any device work."""
    so = M.mlb_sequence_options(4, 1, 1, 8)
    res = (M.mlb_result * 1)()
    used = (C.c_int32 * 1)()
    assert lib.mlbicgstab_solve_sequence(None, 1, None, None, 0, None, None, C.byref(so), res, used) == M.MLB_ERR_ARG
    bad = M.mlb_sequence_options(9, 1, 1, 8)   # n0 > n_max
    hs = (C.c_void_p * 1)(1)
    t = (C.c_double * 1)(1e-10)
    m = (C.c_int64 * 1)(10)
    p = (C.c_void_p * 1)(1)
    assert lib.mlbicgstab_solve_sequence(hs, 1, p, p, 0, t, m, C.byref(bad), res, used) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_set_n(None, 2) == M.MLB_ERR_ARG


def test_autotune_validates_before_gpu(lib):
    r = M.mlb_tune_result()
    assert lib.mlbicgstab_autotune(None, 20, 1, C.byref(r)) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_autotune(C.c_void_p(1), 0, 1, C.byref(r)) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_autotune(C.c_void_p(1), 20, 2, C.byref(r)) == M.MLB_ERR_ARG
    rb = M.mlb_batch_tune_result()
    hs = (C.c_void_p * 1)(1)
    assert lib.mlbicgstab_autotune_batch(None, 1, 1e-8, 20, 1, C.byref(rb)) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_autotune_batch(hs, 0, 1e-8, 20, 1, C.byref(rb)) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_autotune_batch(hs, 1, -1.0, 20, 1, C.byref(rb)) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_autotune_batch(hs, 1, float("nan"), 20, 1, C.byref(rb)) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_autotune_batch(hs, 1, 1e-8, 0, 1, C.byref(rb)) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_autotune_batch(hs, 1, 1e-8, 10000001, 1, C.byref(rb)) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_autotune_batch(hs, 1, 1e-8, 20, 2, C.byref(rb)) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_autotune_batch(hs, 1, 1e-8, 20, 1, None) == M.MLB_ERR_ARG
    t = M.mlb_tuning()
    assert lib.mlbicgstab_get_tuning(None, C.byref(t)) == M.MLB_ERR_ARG
    assert lib.mlbicgstab_set_tuning(None, C.byref(t)) == M.MLB_ERR_ARG
