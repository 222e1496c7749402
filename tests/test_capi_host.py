"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every symbol include/*.h declares, and rejects bad arguments on the
host before any launch (no compute call is made)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tk():
    from paper_2203_07329_gb300 import build
    build.build()
    from paper_2203_07329_gb300 import tikhonov
    tikhonov.lib()
    return tikhonov


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"TK_API\s+[\w\s\*]+?\b(tk_\w+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(tk):
    syms = declared_symbols()
    assert len(syms) >= 15
    L = C.CDLL(tk.LIB_PATH)
    for name in syms:
        assert hasattr(L, name), name


def test_status_strings_and_defaults(tk):
    L = tk.lib()
    for s in range(8):
        assert len(L.tk_status_str(s)) > 0
    o = tk.opts_default()
    assert o.tol == 1e-14 and o.maxiter == 500 and o.sketch == tk.TK_SKETCH_SRHT and o.seed == 1
    # the mixed form's float64 products and large LSQR products from exact digits by default
    assert o.emulate_fp64 == 1 and o.lsqr_tc == 2


def test_workspace_counts_the_digit_planes(tk):
    # 32 bytes per element of A for the two sets of digit planes (rows and columns) of the mixed form
    m, n = 8192, 256
    p = _prob(tk, m, n)
    lam = np.array([1e-3, 1.0])
    o_em = tk.opts_default(precision=tk.TK_PREC_MIXED, s=1024)
    o_no = tk.opts_default(precision=tk.TK_PREC_MIXED, s=1024, emulate_fp64=0, lsqr_tc=0)
    w_em = tk.workspace_size(p, len(lam), o_em)
    w_no = tk.workspace_size(p, len(lam), o_no)
    assert w_em - w_no >= 32 * m * n


def _prob(tk, m, n, lda=None):
    # fake non-null device addresses: validation must reject before touching them
    return tk.tk_problem(m, n, lda if lda is not None else n, tk.TK_F64, 0x1000, 0x2000)


@pytest.mark.parametrize("lams,field", [([1.0, 0.0], "zero"), ([1.0, -2.0], "negative"),
                                        ([float("nan")], "nan"), ([float("inf")], "inf")])
def test_bad_lambda_rejected_on_host(tk, lams, field):
    p = _prob(tk, 100, 10)
    o = tk.opts_default()
    lam = np.array(lams, dtype=np.float64)
    st = tk.lib().tk_solve(C.byref(p), lam.ctypes.data_as(C.c_void_p), len(lams), C.byref(o), None, 0, None,
                           C.c_void_p(0x3000), None)
    assert st == tk.TK_EINVAL, field
    assert "lambda" in tk.last_error()


def test_bad_shapes_and_options_rejected(tk):
    L = tk.lib()
    o = tk.opts_default()
    out = C.c_size_t(0)
    assert L.tk_workspace_size(C.byref(_prob(tk, 100, 10, lda=5)), 2, C.byref(o), C.byref(out)) == tk.TK_EINVAL
    assert L.tk_workspace_size(C.byref(_prob(tk, 0, 10)), 2, C.byref(o), C.byref(out)) == tk.TK_EINVAL
    o2 = tk.opts_default(tol=-1.0)
    assert L.tk_workspace_size(C.byref(_prob(tk, 100, 10)), 2, C.byref(o2), C.byref(out)) == tk.TK_EINVAL
    o3 = tk.opts_default(s=1000)  # SRHT sketch larger than the padded length 128
    assert L.tk_workspace_size(C.byref(_prob(tk, 100, 10)), 2, C.byref(o3), C.byref(out)) == tk.TK_EINVAL
    o4 = tk.opts_default(precond=tk.TK_PRECOND_LOWRANK, precision=tk.TK_PREC_MIXED)  # mixed: m >= n only
    assert L.tk_workspace_size(C.byref(_prob(tk, 10, 100)), 2, C.byref(o4), C.byref(out)) == tk.TK_EINVAL
    o5 = tk.opts_default(precond=tk.TK_PRECOND_LOWRANK)  # Algorithm 4
    assert L.tk_workspace_size(C.byref(_prob(tk, 10, 100)), 2, C.byref(o5), C.byref(out)) == tk.TK_OK
    assert L.tk_workspace_size(C.byref(_prob(tk, 100, 10)), 2, C.byref(o), C.byref(out)) == tk.TK_OK
    assert out.value > 100 * 10 * 8


def test_workspace_too_small_is_enomem(tk):
    p = _prob(tk, 100, 10)
    o = tk.opts_default()
    lam = np.array([1.0])
    st = tk.lib().tk_solve(C.byref(p), lam.ctypes.data_as(C.c_void_p), 1, C.byref(o), C.c_void_p(0x4000), 16, None,
                           C.c_void_p(0x3000), None)
    assert st == tk.TK_ENOMEM


def test_workspace_grows_with_lambda_count(tk):
    o = tk.opts_default()
    sizes = []
    for N in (1, 8, 32):
        out = C.c_size_t(0)
        assert tk.lib().tk_workspace_size(C.byref(_prob(tk, 4096, 256)), N, C.byref(o), C.byref(out)) == 0
        sizes.append(out.value)
    assert sizes[0] < sizes[1] < sizes[2]


def test_emulated_entry_points_validate_on_host(tk):
    # the float64-accurate tensor-core entry points reject bad arguments and short workspaces
    # before any launch (fake device addresses are never touched)
    L = tk.lib()
    fake = C.c_void_p(0x1000)
    assert L.tk_gram_emulated(None, 10, 4, fake, fake, 1 << 20, None) == tk.TK_EINVAL
    assert L.tk_gram_emulated(fake, 0, 4, fake, fake, 1 << 20, None) == tk.TK_EINVAL
    need = L.tk_gram_emulated_workspace(300, 70)
    assert need >= 8 * 2 * 70 * 320  # 8 BF16 digit planes of Y^T (rows padded to 64)
    assert L.tk_gram_emulated(fake, 300, 70, fake, fake, need - 1, None) == tk.TK_ENOMEM
    lam = np.array([1e-3, 1.0])
    brk = (C.c_int * 2)()
    need_c = L.tk_cholesky_emulated_workspace(200, 2)
    assert need_c > L.tk_cholesky_workspace(200, 2)
    st = L.tk_cholesky_shifted_emulated(fake, 200, lam.ctypes.data_as(C.c_void_p), 2, fake, brk, fake, need_c - 1,
                                        None)
    assert st == tk.TK_ENOMEM
    bad = np.array([1.0, float("nan")])
    st = L.tk_cholesky_shifted_emulated(fake, 200, bad.ctypes.data_as(C.c_void_p), 2, fake, brk, fake, need_c,
                                        None)
    assert st == tk.TK_EINVAL
    p = _prob(tk, 1000, 100)
    need_r = L.tk_residual_workspace(1000, 100, 4)
    # two sets of 8 BF16 digit planes of A: rows (1000 x 128, n padded to 64), columns (100 x 1024)
    assert need_r >= 8 * 2 * (1000 * 128 + 100 * 1024)
    assert L.tk_residual(C.byref(p), fake, 4, 99, 1, fake, None, fake, need_r, None) == tk.TK_EINVAL  # ldx < n
    assert L.tk_residual(C.byref(p), fake, 4, 100, 1, fake, None, fake, need_r - 1, None) == tk.TK_ENOMEM
    # rows of more than 2^27 values: beyond what the int64 level sums of one split hold exactly (the
    # plain float64 form takes them)
    wide = (1 << 27) + 1
    pw = _prob(tk, 2, wide)
    assert L.tk_residual(C.byref(pw), fake, 1, wide, 1, fake, None, fake, 1 << 40, None) == tk.TK_EINVAL
    assert "2^27" in tk.last_error()


def test_warm_start_arguments_checked_on_host(tk):
    L = tk.lib()
    out = C.c_size_t(0)
    o = tk.opts_default()
    o.x0 = 0x5000  # a fake device address: validation and sizing never touch it
    # Algorithm 2 / 4 (m < n) take no warm start
    assert L.tk_workspace_size(C.byref(_prob(tk, 10, 100)), 2, C.byref(o), C.byref(out)) == tk.TK_EINVAL
    assert "x0" in tk.last_error()
    # the float64 form keeps r0 = b - A x0 and -lambda x0 per lambda: a larger workspace
    cold = tk.opts_default()
    assert L.tk_workspace_size(C.byref(_prob(tk, 4096, 64)), 4, C.byref(cold), C.byref(out)) == tk.TK_OK
    w_cold = out.value
    assert L.tk_workspace_size(C.byref(_prob(tk, 4096, 64)), 4, C.byref(o), C.byref(out)) == tk.TK_OK
    assert out.value >= w_cold + 8 * 4 * (4096 + 2 * 64)
    # one warm start cannot serve several problems
    probs = (tk.tk_problem * 2)(_prob(tk, 500, 20), _prob(tk, 600, 30))
    assert L.tk_workspace_size_batched(probs, 2, 3, C.byref(o), 1, C.byref(out)) == tk.TK_EINVAL


def test_handle_calls_validate_on_host(tk):
    L = tk.lib()
    assert L.tk_create(None, None) == tk.TK_EINVAL
    assert L.tk_destroy(None) == tk.TK_OK
    assert L.tk_handle_workspace_bytes(None) == 0
    p = _prob(tk, 100, 10)
    o = tk.opts_default()
    lam = np.array([1.0])
    assert L.tk_handle_solve(None, C.byref(p), lam.ctypes.data_as(C.c_void_p), 1, C.byref(o), C.c_void_p(0x3000),
                             None) == tk.TK_EINVAL
    assert L.tk_handle_solve_batched(None, C.byref(p), 1, lam.ctypes.data_as(C.c_void_p), 1, C.byref(o), 1, None,
                                     None) == tk.TK_EINVAL


def test_wait_selftest_validates_on_host(tk):
    L = tk.lib()
    fake = C.c_void_p(0x1000)
    assert L.tk_wait_selftest(0, fake, 16, None) == tk.TK_EINVAL
    assert L.tk_wait_selftest(3000000, fake, 16, None) == tk.TK_EINVAL
    assert L.tk_wait_selftest(1000, None, 0, None) == tk.TK_ENOMEM
    assert L.tk_wait_selftest(1000, fake, 8, None) == tk.TK_ENOMEM
    assert tk.STATUS_NAMES[tk.TK_ETIMEOUT] == "TK_ETIMEOUT"
    assert "timed out" in L.tk_status_str(tk.TK_ETIMEOUT).decode()


def test_profiler_reports_implementation_bytes_beside_algorithmic(tk):
    # the stats struct carries both counts; a collect with nothing recorded gives zeros
    arr = (tk.tk_phase_stats * tk.TK_PHASE_COUNT)()
    assert tk.lib().tk_profile_collect(arr) == tk.TK_OK
    assert all(arr[i].bytes == 0.0 and arr[i].impl_bytes == 0.0 for i in range(tk.TK_PHASE_COUNT))
    assert C.sizeof(tk.tk_phase_stats) == 40


def test_lcurve_validates_on_host(tk):
    L = tk.lib()
    out = C.c_size_t(0)
    o = tk.opts_default()
    p = _prob(tk, 1000, 20)
    assert L.tk_lcurve_workspace_size(C.byref(p), 2, 4, C.byref(o), C.byref(out)) == tk.TK_EINVAL  # N < 3
    assert L.tk_lcurve_workspace_size(C.byref(p), 5, -1, C.byref(o), C.byref(out)) == tk.TK_EINVAL
    assert L.tk_lcurve_workspace_size(C.byref(p), 5, 4, C.byref(o), C.byref(out)) == tk.TK_OK
    big = out.value
    assert L.tk_lcurve_workspace_size(C.byref(p), 5, 0, C.byref(o), C.byref(out)) == tk.TK_OK
    assert out.value < big  # planned for N + N_refine lambdas
    ow = tk.opts_default()
    ow.x0 = 0x5000
    assert L.tk_lcurve_workspace_size(C.byref(p), 5, 4, C.byref(ow), C.byref(out)) == tk.TK_EINVAL
    lam = np.array([1e-3, 1e-2, -1.0])
    pts = (tk.tk_lcurve_point * 3)()
    k = C.c_int(0)
    fake = C.c_void_p(0x4000)
    st = L.tk_lcurve(C.byref(p), lam.ctypes.data_as(C.c_void_p), 3, 0, C.byref(o), fake, 1 << 40, None, fake, pts,
                     C.byref(k))
    assert st == tk.TK_EINVAL and "lambda" in tk.last_error()
    lam = np.array([1e-3, 1e-2, 1e-1])
    st = L.tk_lcurve(C.byref(p), lam.ctypes.data_as(C.c_void_p), 3, 0, C.byref(o), fake, 16, None, fake, pts,
                     C.byref(k))
    assert st == tk.TK_ENOMEM


def test_sparse_sketch_arguments_checked_on_host(tk):
    L = tk.lib()
    fake = C.c_void_p(0x1000)
    assert L.tk_sketch_draw_sparse(1, 0, 4, None, None, None, None, fake, 1 << 20, None) == tk.TK_EINVAL
    assert L.tk_sketch_draw_sparse(1, 100, 0, None, None, None, None, fake, 1 << 20, None) == tk.TK_EINVAL
    assert L.tk_sketch_draw_sparse(1, 100, (1 << 22) + 1, None, None, None, None, fake, 1 << 30, None) == tk.TK_EINVAL
    need = L.tk_sketch_draw_sparse_workspace(100000, 5000)
    assert need >= 17 * 100000  # keys and indices twice, the signs
    assert L.tk_sketch_draw_sparse(1, 100000, 5000, None, None, None, None, fake, need - 1, None) == tk.TK_ENOMEM
    out = C.c_size_t(0)
    o = tk.opts_default(sketch=tk.TK_SKETCH_SPARSE)
    assert L.tk_workspace_size(C.byref(_prob(tk, 5000, 50)), 2, C.byref(o), C.byref(out)) == tk.TK_OK
    o.s = (1 << 22) + 1
    assert L.tk_workspace_size(C.byref(_prob(tk, 1 << 23, 50)), 2, C.byref(o), C.byref(out)) == tk.TK_EINVAL
    o.sketch = 7
    assert L.tk_workspace_size(C.byref(_prob(tk, 5000, 50)), 2, C.byref(o), C.byref(out)) == tk.TK_EINVAL


def test_bp2_arguments_checked_on_host(tk):
    L = tk.lib()
    fake = C.c_void_p(0x1000)
    lam = np.array([1e-3, 1.0])
    brk = (C.c_int * 2)()
    need = L.tk_bp2_factor_workspace(300, 70, 2)
    assert need >= 8 * 2 * 370 * 70  # the two (s + n) x n stacks
    assert L.tk_bp2_factor(fake, 300, 70, lam.ctypes.data_as(C.c_void_p), 2, fake, brk, fake, need - 1,
                           None) == tk.TK_ENOMEM
    bad = np.array([1e-3, 0.0])
    assert L.tk_bp2_factor(fake, 300, 70, bad.ctypes.data_as(C.c_void_p), 2, fake, brk, fake, need,
                           None) == tk.TK_EINVAL
    out = C.c_size_t(0)
    o = tk.opts_default(precond=tk.TK_PRECOND_QR)
    assert L.tk_workspace_size(C.byref(_prob(tk, 10, 100)), 2, C.byref(o), C.byref(out)) == tk.TK_EINVAL  # m < n
    assert L.tk_workspace_size(C.byref(_prob(tk, 1000, 50)), 3, C.byref(o), C.byref(out)) == tk.TK_OK
    o.s = 800
    assert L.tk_workspace_size(C.byref(_prob(tk, 1000, 50)), 3, C.byref(o), C.byref(out)) == tk.TK_OK
    assert out.value >= 8 * 3 * 50 * (800 + 50)  # the three (s + n) x n QR stacks
