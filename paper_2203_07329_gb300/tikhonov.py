"""ctypes binding of libtikhonov (include/tikhonov.h).  Argument marshalling only.

Every function here forwards to the C ABI of the same name; torch is used for
device buffers (inputs, outputs, the workspace) and streams.  There is no CPU
fallback: if the shared library is missing this module raises on load.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtikhonov.so")

TK_OK, TK_EINVAL, TK_ENOMEM, TK_ENOTSPD, TK_ENOCONV, TK_ENUMERIC, TK_ETIMEOUT, TK_ECUDA = range(8)
TK_F64, TK_F32 = 0, 1
TK_SKETCH_SRHT, TK_SKETCH_GAUSS, TK_SKETCH_SPARSE, TK_SKETCH_SRDCT = 0, 1, 2, 3
TK_PRECOND_CHOL, TK_PRECOND_LOWRANK, TK_PRECOND_QR = 0, 1, 2
TK_PREC_FP64, TK_PREC_MIXED = 0, 1
TK_SCHED_BATCHED, TK_SCHED_ONE_AT_A_TIME = 0, 1

STATUS_NAMES = {0: "TK_OK", 1: "TK_EINVAL", 2: "TK_ENOMEM", 3: "TK_ENOTSPD", 4: "TK_ENOCONV", 5: "TK_ENUMERIC",
                6: "TK_ETIMEOUT", 7: "TK_ECUDA"}


class tk_problem(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("lda", C.c_int64), ("dtype", C.c_int),
                ("A", C.c_void_p), ("b", C.c_void_p)]


class tk_opts(C.Structure):
    _fields_ = [("sketch", C.c_int), ("s", C.c_int64), ("precond", C.c_int), ("alpha", C.c_double),
                ("precision", C.c_int), ("tol", C.c_double), ("maxiter", C.c_int), ("max_refine", C.c_int),
                ("inner_tol", C.c_double), ("refine_tol", C.c_double), ("seed", C.c_uint64),
                ("schedule", C.c_int), ("lsqr_tc", C.c_int), ("group", C.c_int), ("emulate_fp64", C.c_int),
                ("x0", C.c_void_p)]


class tk_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("refine_steps", C.c_int), ("istop", C.c_int), ("rank", C.c_int64),
                ("rnorm", C.c_double), ("arnorm", C.c_double), ("ne_norm", C.c_double), ("status", C.c_int)]


TK_PHASE_COUNT = 15


class tk_phase_stats(C.Structure):
    _fields_ = [("ms", C.c_double), ("flops", C.c_double), ("bytes", C.c_double), ("launches", C.c_int),
                ("impl_bytes", C.c_double)]


class tk_lcurve_point(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("rnorm", C.c_double), ("xnorm", C.c_double), ("curvature", C.c_double),
                ("iters", C.c_int), ("status", C.c_int)]


class TikhonovError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """Load libtikhonov.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
        L = C.CDLL(LIB_PATH)
        P, I64, D, INT, SZ, U64 = C.c_void_p, C.c_int64, C.c_double, C.c_int, C.c_size_t, C.c_uint64
        sigs = {
            "tk_opts_default": (INT, [P]),
            "tk_status_str": (C.c_char_p, [INT]),
            "tk_last_error": (C.c_char_p, []),
            "tk_workspace_size": (INT, [P, INT, P, P]),
            "tk_solve": (INT, [P, P, INT, P, P, SZ, P, P, P]),
            "tk_workspace_size_batched": (INT, [P, INT, INT, P, INT, P]),
            "tk_solve_batched": (INT, [P, INT, P, INT, P, INT, P, SZ, P, P, P]),
            "tk_sketch_draw_workspace": (SZ, [I64]),
            "tk_sketch_draw": (INT, [U64, I64, I64, P, P, P, SZ, P]),
            "tk_sketch_apply_workspace": (INT, [P, P, P]),
            "tk_sketch_apply": (INT, [P, P, P, P, SZ, P]),
            "tk_gram": (INT, [P, I64, I64, INT, P, P]),
            "tk_cholesky_workspace": (SZ, [I64, INT]),
            "tk_cholesky_shifted": (INT, [P, I64, P, INT, P, P, P, SZ, P]),
            "tk_cholesky_emulated_workspace": (SZ, [I64, INT]),
            "tk_cholesky_shifted_emulated": (INT, [P, I64, P, INT, P, P, P, SZ, P]),
            "tk_bp2_factor_workspace": (SZ, [I64, I64, INT]),
            "tk_bp2_factor": (INT, [P, I64, I64, P, INT, P, P, P, SZ, P]),
            "tk_sketch_svd_workspace": (SZ, [I64, I64]),
            "tk_sketch_svd": (INT, [P, I64, I64, P, P, P, P, SZ, P]),
            "tk_lowrank_ranks_workspace": (SZ, [INT]),
            "tk_lowrank_ranks": (INT, [P, I64, P, INT, D, P, P, P, SZ, P]),
            "tk_sketch_draw_static": (INT, [U64, I64, I64, P, P, P]),
            "tk_sketch_draw_sparse_workspace": (SZ, [I64, I64]),
            "tk_sketch_draw_sparse": (INT, [U64, I64, I64, P, P, P, P, P, SZ, P]),
            "tk_phase_name": (C.c_char_p, [INT]),
            "tk_launch_count": (C.c_ulonglong, []),
            "tk_profile_enable": (INT, [INT]),
            "tk_profile_collect": (INT, [P]),
            "tk_autotune": (INT, [P, INT, P, P, SZ, P]),
            "tk_autotune_entries": (SZ, []),
            "tk_gram_emulated_workspace": (SZ, [I64, I64]),
            "tk_gram_emulated": (INT, [P, I64, I64, P, P, SZ, P]),
            "tk_residual_workspace": (SZ, [I64, I64, INT]),
            "tk_residual": (INT, [P, P, INT, I64, INT, P, P, P, SZ, P]),
            "tk_autotune_clear": (None, []),
            "tk_wait_selftest": (INT, [I64, P, SZ, P]),
            "tk_lsqr_step_products_workspace": (SZ, [I64, I64, INT]),
            "tk_lsqr_step_products": (INT, [P, P, INT, P, P, P, INT, P, SZ, P]),
            "tk_lcurve_workspace_size": (INT, [P, INT, INT, P, P]),
            "tk_lcurve": (INT, [P, P, INT, INT, P, P, SZ, P, P, P, P]),
            "tk_create": (INT, [P, P]),
            "tk_destroy": (INT, [P]),
            "tk_handle_workspace_bytes": (SZ, [P]),
            "tk_handle_solve": (INT, [P, P, P, INT, P, P, P]),
            "tk_handle_solve_batched": (INT, [P, P, INT, P, INT, P, INT, P, P]),
            "tk_autotune_describe": (SZ, [C.c_char_p, SZ]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().tk_last_error().decode()


def _check(status: int, ok=(TK_OK,)) -> int:
    if status not in ok:
        raise TikhonovError(status, last_error())
    return status


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return TK_F64
    if t.dtype == torch.float32:
        return TK_F32
    raise TypeError("A must be float64 or float32")


def make_problem(A: torch.Tensor, b: torch.Tensor) -> tk_problem:
    if not (A.is_cuda and b.is_cuda):
        raise ValueError("A and b must be CUDA tensors")
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a row-major matrix (unit column stride)")
    if b.dtype != torch.float64 or not b.is_contiguous() or b.numel() != A.shape[0]:
        raise ValueError("b must be a contiguous float64 vector of length m")
    return tk_problem(A.shape[0], A.shape[1], A.stride(0), _dtype_code(A), A.data_ptr(), b.data_ptr())


def opts_default(**kw) -> tk_opts:
    o = tk_opts()
    lib().tk_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def workspace_size(prob: tk_problem, N: int, opts: tk_opts) -> int:
    out = C.c_size_t(0)
    _check(lib().tk_workspace_size(C.byref(prob), N, C.byref(opts), C.byref(out)))
    return int(out.value)


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


@dataclass
class SolveResult:
    X: torch.Tensor          # N x n float64 on the device
    info: list               # per-lambda dicts
    status: int


def _info_dicts(arr, N):
    return [dict(iters=arr[i].iters, refine_steps=arr[i].refine_steps, istop=arr[i].istop, rank=arr[i].rank,
                 rnorm=arr[i].rnorm, arnorm=arr[i].arnorm, ne_norm=arr[i].ne_norm, status=arr[i].status)
            for i in range(N)]


def tk_solve(A: torch.Tensor, b: torch.Tensor, lambdas, opts: tk_opts | None = None, *, work=None, stream=None,
             X: torch.Tensor | None = None, allow=(TK_OK, TK_ENOCONV, TK_ENOTSPD),
             x0: torch.Tensor | None = None) -> SolveResult:
    """x_{lambda_i} for all lambda_i (problem (1.2)); see tk_solve in include/tikhonov.h.
    x0: optional N x n float64 CUDA warm start (sets opts.x0 for this call)."""
    opts = opts or opts_default()
    if x0 is not None:
        if not (x0.is_cuda and x0.dtype == torch.float64 and x0.is_contiguous()):
            raise ValueError("x0 must be a contiguous float64 CUDA tensor (N x n)")
        if tuple(x0.shape) != (len(lambdas), A.shape[1]):
            raise ValueError("x0 must be N x n")
        o2 = tk_opts.from_buffer_copy(opts)
        o2.x0 = x0.data_ptr()
        opts = o2
    prob = make_problem(A, b)
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
    N = int(lam.shape[0])
    n = A.shape[1]
    if X is None:
        X = torch.empty((N, n), dtype=torch.float64, device=A.device)
    nbytes = workspace_size(prob, N, opts)
    if work is None or work.numel() < nbytes:
        work = _workspace(nbytes, A.device)
    info = (tk_info * max(N, 1))()
    st = lib().tk_solve(C.byref(prob), lam.ctypes.data_as(C.c_void_p), N, C.byref(opts), _ptr(work),
                        work.numel(), _stream(stream), _ptr(X), info)
    _check(st, allow)
    return SolveResult(X=X, info=_info_dicts(info, N), status=st)


def tk_solve_batched(problems, lambdas, opts=None, *, work=None, stream=None,
                     allow=(TK_OK, TK_ENOCONV, TK_ENOTSPD)):
    """problems: list of (A, b) CUDA tensors; lambdas: P x N host array; opts: one tk_opts or a list of P."""
    P = len(problems)
    if opts is None:
        opts = opts_default()
    olist = list(opts) if isinstance(opts, (list, tuple)) else [opts]
    n_opts = len(olist)
    oarr = (tk_opts * n_opts)(*olist)
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
    N = lam.shape[1]
    probs = (tk_problem * P)(*[make_problem(A, b) for A, b in problems])
    out = C.c_size_t(0)
    _check(lib().tk_workspace_size_batched(probs, P, N, oarr, n_opts, C.byref(out)))
    dev = problems[0][0].device
    if work is None or work.numel() < out.value:
        work = _workspace(out.value, dev)
    Xs = [torch.empty((N, A.shape[1]), dtype=torch.float64, device=dev) for A, _ in problems]
    xp = (C.c_void_p * P)(*[x.data_ptr() for x in Xs])
    info = (tk_info * (P * N))()
    st = lib().tk_solve_batched(probs, P, lam.ctypes.data_as(C.c_void_p), N, oarr, n_opts, _ptr(work),
                                work.numel(), _stream(stream), xp, info)
    _check(st, allow)
    infos = _info_dicts(info, P * N)
    return Xs, [infos[p * N:(p + 1) * N] for p in range(P)], st


def workspace_size_batched(problems, N, opts) -> int:
    olist = list(opts) if isinstance(opts, (list, tuple)) else [opts]
    oarr = (tk_opts * len(olist))(*olist)
    probs = (tk_problem * len(problems))(*[make_problem(A, b) for A, b in problems])
    out = C.c_size_t(0)
    _check(lib().tk_workspace_size_batched(probs, len(problems), N, oarr, len(olist), C.byref(out)))
    return int(out.value)


def tk_sketch_draw(seed: int, mp: int, s: int, device="cuda", stream=None):
    """SRHT integer draws: (signs int8[mp], rows int64[s]) on the device."""
    signs = torch.empty(mp, dtype=torch.int8, device=device)
    rows = torch.empty(max(s, 1), dtype=torch.int64, device=device)
    ws = int(lib().tk_sketch_draw_workspace(mp))
    work = _workspace(ws, device)
    _check(lib().tk_sketch_draw(seed, mp, s, _ptr(signs), _ptr(rows), _ptr(work), work.numel(), _stream(stream)))
    return signs, rows[:s]


def tk_sketch_draw_static(seed: int, mp: int, s: int, device="cuda", stream=None):
    """The same draws as tk_sketch_draw with no workspace (library-held scratch, mp <= 2^20)."""
    signs = torch.empty(mp, dtype=torch.int8, device=device)
    rows = torch.empty(max(s, 1), dtype=torch.int64, device=device)
    _check(lib().tk_sketch_draw_static(seed, mp, s, _ptr(signs), _ptr(rows), _stream(stream)))
    return signs, rows[:s]


def tk_sketch_draw_sparse(seed: int, L: int, s: int, device="cuda", stream=None):
    """Sparse embedding draws: (h int32[L], sign int8[L], order int32[L], start int32[s+1]) on the device."""
    h = torch.empty(L, dtype=torch.int32, device=device)
    sign = torch.empty(L, dtype=torch.int8, device=device)
    order = torch.empty(L, dtype=torch.int32, device=device)
    start = torch.empty(s + 1, dtype=torch.int32, device=device)
    work = _workspace(int(lib().tk_sketch_draw_sparse_workspace(L, s)), device)
    _check(lib().tk_sketch_draw_sparse(seed, L, s, _ptr(h), _ptr(sign), _ptr(order), _ptr(start), _ptr(work),
                                       work.numel(), _stream(stream)))
    return h, sign, order, start


def tk_sketch_apply(A: torch.Tensor, opts: tk_opts, stream=None) -> torch.Tensor:
    """Y = X A (m >= n, s x n) or Y = A X (m < n, m x s), float64."""
    b = torch.zeros(A.shape[0], dtype=torch.float64, device=A.device)
    prob = make_problem(A, b)
    out = C.c_size_t(0)
    _check(lib().tk_sketch_apply_workspace(C.byref(prob), C.byref(opts), C.byref(out)))
    m, n = A.shape
    s = opts.s if opts.s > 0 else min((16 if opts.sketch == TK_SKETCH_SPARSE else 4) * min(m, n), max(m, n))
    Y = torch.empty((s, n) if m >= n else (m, s), dtype=torch.float64, device=A.device)
    work = _workspace(out.value, A.device)
    _check(lib().tk_sketch_apply(C.byref(prob), C.byref(opts), _ptr(Y), _ptr(work), work.numel(), _stream(stream)))
    return Y


def tk_gram(Y: torch.Tensor, transpose_first: bool = True, stream=None, emulate: bool = False) -> torch.Tensor:
    """C = Y^T Y (transpose_first) or Y Y^T; emulate: Y^T Y on the BF16 tensor cores with
    float64 accuracy, only the upper triangle defined."""
    r, c = Y.shape
    Cm = torch.empty((c, c) if transpose_first else (r, r), dtype=torch.float64, device=Y.device)
    if emulate:
        if not transpose_first:
            raise ValueError("the emulated Gram matrix is Y^T Y")
        work = _workspace(int(lib().tk_gram_emulated_workspace(r, c)), Y.device)
        _check(lib().tk_gram_emulated(_ptr(Y.contiguous()), r, c, _ptr(Cm), _ptr(work), work.numel(),
                                      _stream(stream)))
        return Cm
    _check(lib().tk_gram(_ptr(Y.contiguous()), r, c, 1 if transpose_first else 0, _ptr(Cm), _stream(stream)))
    return Cm


def tk_cholesky_shifted(Cm: torch.Tensor, lambdas, stream=None, emulate: bool = False):
    """R_i = chol(C + lambda_i I): returns (R N x n x n, breakdown list); emulate: the trailing
    updates on the BF16 tensor cores with float64 accuracy."""
    n = Cm.shape[0]
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
    N = lam.shape[0]
    R = torch.empty((N, n, n), dtype=torch.float64, device=Cm.device)
    brk = (C.c_int * N)()
    if emulate:
        work = _workspace(lib().tk_cholesky_emulated_workspace(n, N), Cm.device)
        fn = lib().tk_cholesky_shifted_emulated
    else:
        work = _workspace(lib().tk_cholesky_workspace(n, N), Cm.device)
        fn = lib().tk_cholesky_shifted
    st = fn(_ptr(Cm.contiguous()), n, lam.ctypes.data_as(C.c_void_p), N, _ptr(R), brk, _ptr(work), work.numel(),
            _stream(stream))
    _check(st, (TK_OK, TK_ENOTSPD))
    return R, list(brk)


def tk_bp2_factor(Y: torch.Tensor, lambdas, stream=None):
    """BP2 factors R_i from a QR of [Y; sqrt(l_i) I] (Section 4.1): (R N x n x n, breakdown list)."""
    s, n = Y.shape
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
    N = lam.shape[0]
    R = torch.empty((N, n, n), dtype=torch.float64, device=Y.device)
    brk = (C.c_int * N)()
    work = _workspace(lib().tk_bp2_factor_workspace(s, n, N), Y.device)
    st = lib().tk_bp2_factor(_ptr(Y.contiguous()), s, n, lam.ctypes.data_as(C.c_void_p), N, _ptr(R), brk, _ptr(work),
                             work.numel(), _stream(stream))
    _check(st, (TK_OK, TK_ENOTSPD))
    return R, list(brk)


def tk_sketch_svd(Y: torch.Tensor, stream=None):
    """[~, Sigma, V] = svd(Y, 'econ') by one-sided Jacobi: (sigma s, V n x s, sweeps)."""
    s, n = Y.shape
    sig = torch.empty(s, dtype=torch.float64, device=Y.device)
    V = torch.empty((n, s), dtype=torch.float64, device=Y.device)
    sw = C.c_int(0)
    work = _workspace(lib().tk_sketch_svd_workspace(s, n), Y.device)
    _check(lib().tk_sketch_svd(_ptr(Y.contiguous()), s, n, _ptr(sig), _ptr(V), C.byref(sw), _ptr(work),
                               work.numel(), _stream(stream)))
    return sig, V, sw.value


def tk_lowrank_ranks(sigma: torch.Tensor, lambdas, alpha: float, stream=None):
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
    N = lam.shape[0]
    sd = np.zeros(N)
    rk = np.zeros(N, dtype=np.int64)
    work = _workspace(lib().tk_lowrank_ranks_workspace(N), sigma.device)
    _check(lib().tk_lowrank_ranks(_ptr(sigma.contiguous()), sigma.numel(), lam.ctypes.data_as(C.c_void_p), N,
                                  alpha, sd.ctypes.data_as(C.c_void_p), rk.ctypes.data_as(C.c_void_p), _ptr(work),
                                  work.numel(), _stream(stream)))
    return sd, rk


def tk_profile_enable(on: bool = True) -> None:
    _check(lib().tk_profile_enable(1 if on else 0))


def tk_profile_collect() -> dict:
    """Per-phase totals since the last collect: {name: dict(ms, flops, bytes, launches)}."""
    arr = (tk_phase_stats * TK_PHASE_COUNT)()
    _check(lib().tk_profile_collect(arr))
    return {lib().tk_phase_name(i).decode(): dict(ms=arr[i].ms, flops=arr[i].flops, bytes=arr[i].bytes,
                                                   impl_bytes=arr[i].impl_bytes, launches=arr[i].launches)
            for i in range(TK_PHASE_COUNT)}


def tk_launch_count() -> int:
    return int(lib().tk_launch_count())


def tk_autotune(A: torch.Tensor, b: torch.Tensor, N: int, opts: tk_opts, work=None, stream=None) -> int:
    """Measure the tile shapes and split counts of this problem's LSQR / refinement
    products (the table is process-wide); returns the number of table entries."""
    prob = make_problem(A, b)
    need = workspace_size(prob, N, opts)
    if work is None or work.numel() < need:
        work = _workspace(need, A.device)
    _check(lib().tk_autotune(C.byref(prob), N, C.byref(opts), _ptr(work), work.numel(), _stream(stream)))
    return int(lib().tk_autotune_entries())


def tk_autotune_clear() -> None:
    lib().tk_autotune_clear()


def tk_autotune_describe() -> str:
    n = int(lib().tk_autotune_describe(None, 0))
    buf = C.create_string_buffer(n)
    lib().tk_autotune_describe(buf, n)
    return buf.value.decode()


def tk_lcurve(A: torch.Tensor, b: torch.Tensor, lambdas, N_refine: int, opts: tk_opts | None = None, *,
              work=None, stream=None, allow=(TK_OK, TK_ENOCONV, TK_ENOTSPD)):
    """The L-curve of Section 4.3 (include/tikhonov.h tk_lcurve): returns (X, points, corner) with X
    (N + N_refine) x n on the device and points a list of dicts in ascending lambda."""
    opts = opts or opts_default()
    prob = make_problem(A, b)
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
    N = int(lam.shape[0])
    Np = N + int(N_refine)
    out = C.c_size_t(0)
    _check(lib().tk_lcurve_workspace_size(C.byref(prob), N, int(N_refine), C.byref(opts), C.byref(out)))
    if work is None or work.numel() < out.value:
        work = _workspace(out.value, A.device)
    X = torch.empty((Np, A.shape[1]), dtype=torch.float64, device=A.device)
    pts = (tk_lcurve_point * Np)()
    corner = C.c_int(-1)
    st = lib().tk_lcurve(C.byref(prob), lam.ctypes.data_as(C.c_void_p), N, int(N_refine), C.byref(opts), _ptr(work),
                         work.numel(), _stream(stream), _ptr(X), pts, C.byref(corner))
    _check(st, allow)
    points = [dict(lam=pts[i].lambda_, rnorm=pts[i].rnorm, xnorm=pts[i].xnorm, curvature=pts[i].curvature,
                   iters=pts[i].iters, status=pts[i].status) for i in range(Np)]
    return X, points, corner.value


def lcurve_workspace_size(A, b, N: int, N_refine: int, opts: tk_opts) -> int:
    out = C.c_size_t(0)
    prob = make_problem(A, b)
    _check(lib().tk_lcurve_workspace_size(C.byref(prob), N, N_refine, C.byref(opts), C.byref(out)))
    return int(out.value)


def tk_lsqr_step_products(A: torch.Tensor, W: torch.Tensor, U: torch.Tensor, coef: torch.Tensor | None, mode: int,
                          stream=None) -> torch.Tensor:
    """U <- W A^T + coef .* U (in place) and G = U A; returns G (count x n).  mode 0: the two digit
    products; 1: both in one kernel; 2: the float32 products of at most 16 lambda."""
    b = torch.zeros(A.shape[0], dtype=torch.float64, device=A.device)
    prob = make_problem(A, b)
    count = W.shape[0]
    G = torch.empty((count, A.shape[1]), dtype=torch.float64, device=A.device)
    work = _workspace(int(lib().tk_lsqr_step_products_workspace(A.shape[0], A.shape[1], count)), A.device)
    _check(lib().tk_lsqr_step_products(C.byref(prob), _ptr(W.contiguous()), count, _ptr(U), _ptr(coef), _ptr(G),
                                       int(mode), _ptr(work), work.numel(), _stream(stream)))
    return G


def tk_wait_selftest(budget_us: int, device="cuda", stream=None) -> int:
    """Status of the bounded-wait self-test (TK_ETIMEOUT when the wait gave up, as it should)."""
    work = _workspace(16, device)
    return int(lib().tk_wait_selftest(int(budget_us), _ptr(work), work.numel(), _stream(stream)))


def tk_residual(A: torch.Tensor, b: torch.Tensor, X: torch.Tensor, emulate: bool, with_g: bool = False,
                stream=None):
    """R = b - X A^T (M x m) and, with with_g, G = R A (M x n), float64, for the M rows
    of X: float64 FMA (emulate=False) or the BF16 tensor cores with float64 accuracy."""
    prob = make_problem(A, b)
    X = X.contiguous()
    M = X.shape[0]
    R = torch.empty((M, A.shape[0]), dtype=torch.float64, device=A.device)
    G = torch.empty((M, A.shape[1]), dtype=torch.float64, device=A.device) if with_g else None
    need = int(lib().tk_residual_workspace(A.shape[0], A.shape[1], M))
    work = _workspace(need, A.device)
    _check(lib().tk_residual(C.byref(prob), _ptr(X), M, X.shape[1], 1 if emulate else 0, _ptr(R), _ptr(G),
                             _ptr(work), work.numel(), _stream(stream)))
    return (R, G) if with_g else R


class Handle:
    """tk_create / tk_destroy: a stream and a library-owned workspace (include/tikhonov.h)."""

    def __init__(self, stream=None):
        self._h = C.c_void_p(None)
        _check(lib().tk_create(C.byref(self._h), _stream(stream)))

    def close(self):
        if self._h:
            _check(lib().tk_destroy(self._h))
            self._h = C.c_void_p(None)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self) -> int:
        return int(lib().tk_handle_workspace_bytes(self._h))

    def solve(self, A, b, lambdas, opts=None, X=None, allow=(TK_OK, TK_ENOCONV, TK_ENOTSPD)) -> SolveResult:
        opts = opts or opts_default()
        prob = make_problem(A, b)
        lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
        N = int(lam.shape[0])
        if X is None:
            X = torch.empty((N, A.shape[1]), dtype=torch.float64, device=A.device)
        info = (tk_info * max(N, 1))()
        st = lib().tk_handle_solve(self._h, C.byref(prob), lam.ctypes.data_as(C.c_void_p), N, C.byref(opts),
                                   _ptr(X), info)
        _check(st, allow)
        return SolveResult(X=X, info=_info_dicts(info, N), status=st)

    def solve_batched(self, problems, lambdas, opts=None, allow=(TK_OK, TK_ENOCONV, TK_ENOTSPD)):
        P = len(problems)
        olist = list(opts) if isinstance(opts, (list, tuple)) else [opts or opts_default()]
        oarr = (tk_opts * len(olist))(*olist)
        lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
        N = lam.shape[1]
        probs = (tk_problem * P)(*[make_problem(A, b) for A, b in problems])
        dev = problems[0][0].device
        Xs = [torch.empty((N, A.shape[1]), dtype=torch.float64, device=dev) for A, _ in problems]
        xp = (C.c_void_p * P)(*[x.data_ptr() for x in Xs])
        info = (tk_info * (P * N))()
        st = lib().tk_handle_solve_batched(self._h, probs, P, lam.ctypes.data_as(C.c_void_p), N, oarr, len(olist),
                                           xp, info)
        _check(st, allow)
        infos = _info_dicts(info, P * N)
        return Xs, [infos[p * N:(p + 1) * N] for p in range(P)], st
