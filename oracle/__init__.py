"""Plain FP64 CPU oracle for randomized Tikhonov regularization (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The product (``paper_2203_07329_gb300``
and its CUDA library) never imports it and shares no code with it.

The arithmetic lives in ``tk_oracle.c`` (plain loops, double precision, built
with ``-ffp-contract=off``).  This module only compiles it and marshals numpy
arrays through ctypes.  Every function names the passage of the paper it
follows; see the C source for the formulas.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = C.c_double
_i64 = C.c_int64
_u64 = C.c_uint64
_int = C.c_int
_p = C.c_void_p


def build(force: bool = False) -> str:
    """Compile tk_oracle.c into liboracle.so next to it (gcc, OpenMP, no contraction)."""
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            sig = {
                "orc_philox4x32_10": (None, [_p, _p, _p]),
                "orc_draw_signs": (None, [_u64, _i64, _p]),
                "orc_draw_keys": (None, [_u64, _i64, _p]),
                "orc_draw_rows": (_int, [_u64, _i64, _i64, _p]),
                "orc_gauss_entry": (_d, [_u64, _u64, _d]),
                "orc_draw_gauss": (None, [_u64, _i64, _i64, _p]),
                "orc_next_pow2": (_i64, [_i64]),
                "orc_fwht": (None, [_p, _i64]),
                "orc_srht_over": (None, [_p, _i64, _i64, _i64, _u64, _i64, _p]),
                "orc_srht_under": (None, [_p, _i64, _i64, _i64, _u64, _i64, _p]),
                "orc_gauss_over": (None, [_p, _i64, _i64, _i64, _u64, _i64, _p]),
                "orc_gauss_under": (None, [_p, _i64, _i64, _i64, _u64, _i64, _p]),
                "orc_gram_tn": (None, [_p, _i64, _i64, _p]),
                "orc_gram_nt": (None, [_p, _i64, _i64, _p]),
                "orc_cholesky_shifted": (_int, [_p, _i64, _d, _p]),
                "orc_trsv_upper": (None, [_p, _i64, _p, _p]),
                "orc_trsv_upper_t": (None, [_p, _i64, _p, _p]),
                "orc_lsqr_plain": (_int, [_p, _i64, _i64, _i64, _p, _d, _int, _p, _p]),
                "orc_lsqr_over_chol": (_int, [_p, _i64, _i64, _i64, _p, _d, _p, _d, _int, _p, _p]),
                "orc_lsqr_over_lr": (_int, [_p, _i64, _i64, _i64, _p, _d, _p, _i64, _p, _i64, _d, _int, _p, _p]),
                "orc_lsqr_under_chol": (_int, [_p, _i64, _i64, _i64, _p, _d, _p, _d, _int, _p, _p]),
                "orc_lsqr_under_lr": (_int, [_p, _i64, _i64, _i64, _p, _d, _p, _i64, _p, _i64, _d, _int, _p, _p]),
                "orc_jacobi_svd": (_int, [_p, _i64, _i64, _d, _int, _p, _p]),
                "orc_sd_estimate": (_d, [_p, _i64, _d]),
                "orc_truncation": (_i64, [_d, _d, _i64]),
                "orc_lr_diag": (None, [_p, _i64, _d, _p]),
                "orc_draw_sparse": (None, [_u64, _i64, _i64, _p, _p]),
                "orc_sparse_over": (None, [_p, _i64, _i64, _i64, _u64, _i64, _p]),
                "orc_sparse_under": (None, [_p, _i64, _i64, _i64, _u64, _i64, _p]),
                "orc_dct2_rows": (None, [_p, _i64, _p, _i64, _p]),
                "orc_srdct_over": (None, [_p, _i64, _i64, _i64, _u64, _i64, _p]),
                "orc_srdct_under": (None, [_p, _i64, _i64, _i64, _u64, _i64, _p]),
                "orc_bp2_r": (_int, [_p, _i64, _i64, _d, _p]),
                "orc_lcurve_norms": (None, [_p, _i64, _i64, _i64, _p, _p, _int, _p, _p]),
                "orc_lcurve_curvature": (_int, [_p, _p, _p, _int, _p]),
                "orc_lcurve_refine_grid": (None, [_p, _int, _int, _int, _p]),
                "orc_alg1": (_int, [_p, _i64, _i64, _i64, _p, _p, _int, _int, _i64, _u64, _d, _int, _p, _p, _p]),
                "orc_alg2": (_int, [_p, _i64, _i64, _i64, _p, _p, _int, _int, _i64, _u64, _d, _int, _p, _p, _p]),
                "orc_alg3": (_int, [_p, _i64, _i64, _i64, _p, _p, _int, _int, _i64, _d, _u64, _d, _int, _p, _p, _p,
                                    _p, _p]),
                "orc_alg4": (_int, [_p, _i64, _i64, _i64, _p, _p, _int, _int, _i64, _d, _u64, _d, _int, _p, _p, _p,
                                    _p, _p]),
                "orc_two_prod": (None, [_d, _d, _p, _p]),
                "orc_two_sum": (None, [_d, _d, _p, _p]),
                "orc_ridge_residual_dd": (None, [_p, _i64, _i64, _i64, _p, _d, _p, _p, _p]),
                "orc_ref_ridge_qr": (_int, [_p, _i64, _i64, _i64, _p, _d, _int, _p]),
                "orc_ref_ridge_refine": (None, [_p, _i64, _i64, _i64, _p, _d, _p, _i64, _p, _int, _p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


SKETCH_SRHT = 0
SKETCH_GAUSS = 1
SKETCH_SPARSE = 2
SKETCH_SRDCT = 3


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dims(A: np.ndarray):
    A = _f64(A)
    m, n = A.shape
    return A, m, n, n


# ---------------------------------------------------------------- draws ----
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw_signs(seed: int, mp: int) -> np.ndarray:
    """Section 2.1.1, the diagonal D of random signs (stream 0)."""
    d = np.zeros(mp, dtype=np.int8)
    lib().orc_draw_signs(seed, mp, _ptr(d))
    return d


def draw_keys(seed: int, mp: int) -> np.ndarray:
    k = np.zeros(mp, dtype=np.uint64)
    lib().orc_draw_keys(seed, mp, _ptr(k))
    return k


def draw_rows(seed: int, mp: int, s: int) -> np.ndarray:
    """Section 2.1.1, the row subset of S: s smallest (key, row), ascending."""
    rows = np.zeros(max(s, 1), dtype=np.int64)
    rc = lib().orc_draw_rows(seed, mp, s, _ptr(rows))
    if rc != 0:
        raise ValueError("s out of range")
    return rows[:s]


def draw_gauss(seed: int, s: int, L: int) -> np.ndarray:
    """Section 2.1.1, Gaussian embedding G (s x L) with N(0, 1/s) entries."""
    G = np.zeros((s, L), dtype=np.float64)
    lib().orc_draw_gauss(seed, s, L, _ptr(G))
    return G


def next_pow2(m: int) -> int:
    return int(lib().orc_next_pow2(m))


# -------------------------------------------------------------- sketches ---
def fwht(z) -> np.ndarray:
    z = _f64(z).copy()
    lib().orc_fwht(_ptr(z), z.shape[0])
    return z


def srht_over(A, seed: int, s: int) -> np.ndarray:
    A, m, n, lda = _dims(A)
    Y = np.zeros((s, n))
    lib().orc_srht_over(_ptr(A), m, n, lda, seed, s, _ptr(Y))
    return Y


def srht_under(A, seed: int, s: int) -> np.ndarray:
    A, m, n, lda = _dims(A)
    Y = np.zeros((m, s))
    lib().orc_srht_under(_ptr(A), m, n, lda, seed, s, _ptr(Y))
    return Y


def gauss_over(A, seed: int, s: int) -> np.ndarray:
    A, m, n, lda = _dims(A)
    Y = np.zeros((s, n))
    lib().orc_gauss_over(_ptr(A), m, n, lda, seed, s, _ptr(Y))
    return Y


def gauss_under(A, seed: int, s: int) -> np.ndarray:
    A, m, n, lda = _dims(A)
    Y = np.zeros((m, s))
    lib().orc_gauss_under(_ptr(A), m, n, lda, seed, s, _ptr(Y))
    return Y


def draw_sparse(seed: int, L: int, s: int):
    """Sparse embedding draws (Section 2.1.1, one nonzero per column): rows h (int32[L]) and signs
    (int8[L]) of Philox stream 4."""
    h = np.zeros(L, dtype=np.int32)
    d = np.zeros(L, dtype=np.int8)
    lib().orc_draw_sparse(seed, L, s, _ptr(h), _ptr(d))
    return h, d


def sparse_over(A, seed: int, s: int) -> np.ndarray:
    """Y = X A with the sparse embedding X (s x m): Y[h_i] += sign_i A[i], rows in ascending order."""
    A, m, n, lda = _dims(A)
    Y = np.zeros((s, n))
    lib().orc_sparse_over(_ptr(A), m, n, lda, seed, s, _ptr(Y))
    return Y


def sparse_under(A, seed: int, s: int) -> np.ndarray:
    """Y = A X^T with the sparse embedding on the columns (m x s)."""
    A, m, n, lda = _dims(A)
    Y = np.zeros((m, s))
    lib().orc_sparse_under(_ptr(A), m, n, lda, seed, s, _ptr(Y))
    return Y


def dct2_rows(z, rows) -> np.ndarray:
    """Rows `rows` of the orthonormal DCT-II of z, each by its defining sum."""
    z = _f64(z)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(r.shape[0])
    lib().orc_dct2_rows(_ptr(z), z.shape[0], _ptr(r), r.shape[0], _ptr(out))
    return out


def srdct_over(A, seed: int, s: int) -> np.ndarray:
    """Y = sqrt(mp/s) S C D [A; 0] (s x n), C the orthonormal DCT-II of length mp."""
    A, m, n, lda = _dims(A)
    Y = np.zeros((s, n))
    lib().orc_srdct_over(_ptr(A), m, n, lda, seed, s, _ptr(Y))
    return Y


def srdct_under(A, seed: int, s: int) -> np.ndarray:
    """Y = sqrt(np/s) [A 0] D C^T S^T (m x s)."""
    A, m, n, lda = _dims(A)
    Y = np.zeros((m, s))
    lib().orc_srdct_under(_ptr(A), m, n, lda, seed, s, _ptr(Y))
    return Y


def sketch_over(A, kind: int, seed: int, s: int) -> np.ndarray:
    if kind == SKETCH_SRDCT:
        return srdct_over(A, seed, s)
    if kind == SKETCH_SPARSE:
        return sparse_over(A, seed, s)
    return srht_over(A, seed, s) if kind == SKETCH_SRHT else gauss_over(A, seed, s)


def sketch_under(A, kind: int, seed: int, s: int) -> np.ndarray:
    if kind == SKETCH_SRDCT:
        return srdct_under(A, seed, s)
    if kind == SKETCH_SPARSE:
        return sparse_under(A, seed, s)
    return srht_under(A, seed, s) if kind == SKETCH_SRHT else gauss_under(A, seed, s)


# ------------------------------------------------------ Gram / Cholesky ----
def gram_tn(Y) -> np.ndarray:
    Y = _f64(Y)
    r, c = Y.shape
    G = np.zeros((c, c))
    lib().orc_gram_tn(_ptr(Y), r, c, _ptr(G))
    return G


def gram_nt(Y) -> np.ndarray:
    Y = _f64(Y)
    r, c = Y.shape
    G = np.zeros((r, r))
    lib().orc_gram_nt(_ptr(Y), r, c, _ptr(G))
    return G


def cholesky_shifted(Cm, lam: float):
    """Algorithm 1 step 4: R = chol(C + lambda I), upper.  Returns (R, info)."""
    Cm = _f64(Cm)
    n = Cm.shape[0]
    R = np.zeros((n, n))
    info = lib().orc_cholesky_shifted(_ptr(Cm), n, lam, _ptr(R))
    return R, int(info)


def trsv_upper(R, v) -> np.ndarray:
    R, v = _f64(R), _f64(v)
    x = np.zeros_like(v)
    lib().orc_trsv_upper(_ptr(R), R.shape[0], _ptr(v), _ptr(x))
    return x


def trsv_upper_t(R, v) -> np.ndarray:
    R, v = _f64(R), _f64(v)
    x = np.zeros_like(v)
    lib().orc_trsv_upper_t(_ptr(R), R.shape[0], _ptr(v), _ptr(x))
    return x


# ----------------------------------------------------------------- LSQR ----
def lsqr_plain(A, b, tol: float, maxiter: int):
    A, m, n, lda = _dims(A)
    b = _f64(b)
    x = np.zeros(n)
    ist = C.c_int(0)
    it = lib().orc_lsqr_plain(_ptr(A), m, n, lda, _ptr(b), tol, maxiter, _ptr(x), C.byref(ist))
    return x, int(it), ist.value


def lsqr_over_chol(A, b, lam: float, R, tol: float, maxiter: int):
    A, m, n, lda = _dims(A)
    b, R = _f64(b), _f64(R)
    x = np.zeros(n)
    ist = C.c_int(0)
    it = lib().orc_lsqr_over_chol(_ptr(A), m, n, lda, _ptr(b), lam, _ptr(R), tol, maxiter, _ptr(x), C.byref(ist))
    return x, int(it), ist.value


def lsqr_over_lr(A, b, lam: float, V, S, si: int, tol: float, maxiter: int):
    A, m, n, lda = _dims(A)
    b, V, S = _f64(b), _f64(V), _f64(S)
    x = np.zeros(n)
    ist = C.c_int(0)
    it = lib().orc_lsqr_over_lr(_ptr(A), m, n, lda, _ptr(b), lam, _ptr(V), V.shape[1], _ptr(S), si, tol, maxiter,
                                _ptr(x), C.byref(ist))
    return x, int(it), ist.value


def lsqr_under_chol(A, b, lam: float, R, tol: float, maxiter: int):
    A, m, n, lda = _dims(A)
    b, R = _f64(b), _f64(R)
    x = np.zeros(n)
    ist = C.c_int(0)
    it = lib().orc_lsqr_under_chol(_ptr(A), m, n, lda, _ptr(b), lam, _ptr(R), tol, maxiter, _ptr(x), C.byref(ist))
    return x, int(it), ist.value


# ------------------------------------------------------------ low rank -----
def jacobi_svd(Y, tol: float = 1e-15, max_sweeps: int = 80):
    """Algorithm 3 step 4 ([~, Sigma, V] = svd(Y, 'econ')) by one-sided Jacobi."""
    Y = _f64(Y)
    s, n = Y.shape
    sig = np.zeros(s)
    V = np.zeros((n, s))
    sweeps = lib().orc_jacobi_svd(_ptr(Y), s, n, tol, max_sweeps, _ptr(sig), _ptr(V))
    return sig, V, int(sweeps)


def sd_estimate(sigma, lam: float) -> float:
    """Section 3.1.2: sd estimate from the singular values of the sketch."""
    sigma = _f64(sigma)
    return float(lib().orc_sd_estimate(_ptr(sigma), sigma.shape[0], lam))


def truncation(sd: float, alpha: float, s: int) -> int:
    return int(lib().orc_truncation(sd, alpha, s))


def lr_diag(sigma, si: int, lam: float) -> np.ndarray:
    sigma = _f64(sigma)
    S = np.zeros(max(si, 1))
    lib().orc_lr_diag(_ptr(sigma), si, lam, _ptr(S))
    return S[:si]


def lsqr_under_lr(A, b, lam: float, U, S, tol: float, maxiter: int):
    """Section 3.2 / Algorithm 4 step 8: min-norm LSQR with R^-T = l^{-1/2}(I - U S U^T)."""
    A, m, n, lda = _dims(A)
    b = _f64(b)
    U = _f64(U)
    S = _f64(S)
    x = np.zeros(n)
    ist = C.c_int(0)
    it = lib().orc_lsqr_under_lr(_ptr(A), m, n, lda, _ptr(b), lam, _ptr(U), U.shape[1], _ptr(S), S.shape[0], tol,
                                 maxiter, _ptr(x), C.byref(ist))
    return x, int(it), int(ist.value)


# ------------------------------------------------------- whole algorithms --
def alg1(A, b, lambdas, sketch_kind: int, s: int, seed: int, tol: float, maxiter: int):
    """Algorithm 1 (overdetermined, Cholesky).  Returns (X n x N, iters, istops, rc)."""
    A, m, n, lda = _dims(A)
    b = _f64(b)
    lam = _f64(lambdas)
    N = lam.shape[0]
    X = np.zeros((n, N))
    it = np.zeros(N, dtype=np.int32)
    st = np.zeros(N, dtype=np.int32)
    rc = lib().orc_alg1(_ptr(A), m, n, lda, _ptr(b), _ptr(lam), N, sketch_kind, s, seed, tol, maxiter, _ptr(X),
                        _ptr(it), _ptr(st))
    return X, it, st, int(rc)


def alg2(A, b, lambdas, sketch_kind: int, s: int, seed: int, tol: float, maxiter: int):
    """Algorithm 2 (underdetermined, Cholesky, min-norm LSQR)."""
    A, m, n, lda = _dims(A)
    b = _f64(b)
    lam = _f64(lambdas)
    N = lam.shape[0]
    X = np.zeros((n, N))
    it = np.zeros(N, dtype=np.int32)
    st = np.zeros(N, dtype=np.int32)
    rc = lib().orc_alg2(_ptr(A), m, n, lda, _ptr(b), _ptr(lam), N, sketch_kind, s, seed, tol, maxiter, _ptr(X),
                        _ptr(it), _ptr(st))
    return X, it, st, int(rc)


def alg3(A, b, lambdas, sketch_kind: int, s: int, alpha: float, seed: int, tol: float, maxiter: int):
    """Algorithm 3 (overdetermined, low rank).  Returns (X, iters, istops, s_i, sigma(Y))."""
    A, m, n, lda = _dims(A)
    b = _f64(b)
    lam = _f64(lambdas)
    N = lam.shape[0]
    X = np.zeros((n, N))
    it = np.zeros(N, dtype=np.int32)
    st = np.zeros(N, dtype=np.int32)
    si = np.zeros(N, dtype=np.int64)
    sig = np.zeros(s)
    lib().orc_alg3(_ptr(A), m, n, lda, _ptr(b), _ptr(lam), N, sketch_kind, s, alpha, seed, tol, maxiter, _ptr(X),
                   _ptr(it), _ptr(st), _ptr(si), _ptr(sig))
    return X, it, st, si, sig


# ------------------------------------------------------------ reference ----
def two_prod(a: float, b: float):
    p, e = C.c_double(), C.c_double()
    lib().orc_two_prod(a, b, C.byref(p), C.byref(e))
    return p.value, e.value


def two_sum(a: float, b: float):
    s, e = C.c_double(), C.c_double()
    lib().orc_two_sum(a, b, C.byref(s), C.byref(e))
    return s.value, e.value


def ridge_residual_dd(A, b, lam: float, x):
    """g = A^T (b - A x) - lambda x accumulated in double-double; returns (g, r)."""
    A, m, n, lda = _dims(A)
    b, x = _f64(b), _f64(x)
    g = np.zeros(n)
    r = np.zeros(m)
    lib().orc_ridge_residual_dd(_ptr(A), m, n, lda, _ptr(b), lam, _ptr(x), _ptr(g), _ptr(r))
    return g, r


def ref_ridge_qr(A, b, lam: float, refine: int = 2) -> np.ndarray:
    """Unique ridge solution (1.2) by Householder QR of [A; sqrt(l) I] + dd refinement."""
    A, m, n, lda = _dims(A)
    b = _f64(b)
    x = np.zeros(n)
    rc = lib().orc_ref_ridge_qr(_ptr(A), m, n, lda, _ptr(b), lam, refine, _ptr(x))
    if rc != 0:
        raise ArithmeticError("singular QR factor")
    return x


def ref_ridge_refine(A, b, lam: float, V, sigma, x0, steps: int = 2) -> np.ndarray:
    """Refine x0 against the stored A with the approximate inverse built from (V, sigma)."""
    A, m, n, lda = _dims(A)
    b, V, sigma = _f64(b), _f64(V), _f64(sigma)
    x = _f64(x0).copy()
    lib().orc_ref_ridge_refine(_ptr(A), m, n, lda, _ptr(b), lam, _ptr(V), V.shape[1], _ptr(sigma), steps, _ptr(x))
    return x


def ref_ridge_under(A, b, lam: float, refine: int = 2) -> np.ndarray:
    """Ridge solution for m < n (the unique minimiser of (1.2), equal to the top
    block of the min-norm solution of (1.4)): the closed form
    x = V diag(sigma/(sigma^2+l)) U^T b from a library SVD of A, then refinement
    against A with the double-double normal-equation residual."""
    A, m, n, lda = _dims(A)
    b = _f64(b)
    U, sig, Vt = np.linalg.svd(A, full_matrices=False)
    x0 = Vt.T @ ((sig / (sig * sig + lam)) * (U.T @ b))
    return ref_ridge_refine(A, b, lam, Vt.T, sig, x0, steps=refine)


def alg4(A, b, lambdas, sketch_kind: int, s: int, alpha: float, seed: int, tol: float, maxiter: int):
    """Algorithm 4 (underdetermined, low rank).  Returns (X n x N, iters, istops, s_i, sigma(Y))."""
    A, m, n, lda = _dims(A)
    b = _f64(b)
    lam = _f64(lambdas)
    N = lam.shape[0]
    X = np.zeros((n, N))
    it = np.zeros(N, dtype=np.int32)
    st = np.zeros(N, dtype=np.int32)
    si = np.zeros(N, dtype=np.int64)
    sig = np.zeros(s)
    lib().orc_alg4(_ptr(A), m, n, lda, _ptr(b), _ptr(lam), N, sketch_kind, s, alpha, seed, tol, maxiter, _ptr(X),
                   _ptr(it), _ptr(st), _ptr(si), _ptr(sig))
    return X, it, st, si, sig


# ------------------------------------------------------------- L-curve ----
def lcurve_norms(A, b, X):
    """(||b - A x_i||, ||x_i||) for the rows x_i of X (Section 4.3)."""
    A, m, n, lda = _dims(A)
    b = _f64(b)
    X = _f64(np.atleast_2d(X))
    N = X.shape[0]
    rn, xn = np.zeros(N), np.zeros(N)
    lib().orc_lcurve_norms(_ptr(A), m, n, lda, _ptr(b), _ptr(X), N, _ptr(rn), _ptr(xn))
    return rn, xn


def lcurve_curvature(lambdas, rn, xn):
    """Curvature of (ln ||Ax-b||, ln ||x||) in t = ln lambda on an ascending grid, and the corner
    index (largest interior curvature; Section 4.3 read as Hansen's maximum-curvature corner)."""
    lam, rn, xn = _f64(lambdas), _f64(rn), _f64(xn)
    N = lam.shape[0]
    kap = np.zeros(N)
    k = lib().orc_lcurve_curvature(_ptr(lam), _ptr(rn), _ptr(xn), N, _ptr(kap))
    return kap, int(k)


def lcurve_refine_grid(lambdas, k, nr):
    """nr parameters log-spaced strictly between the corner's neighbours."""
    lam = _f64(lambdas)
    out = np.zeros(nr)
    lib().orc_lcurve_refine_grid(_ptr(lam), lam.shape[0], int(k), int(nr), _ptr(out))
    return out


def lcurve(A, b, lambdas, nr, refine=3):
    """The two-sweep L-curve of Section 4.3 from the dense reference solutions: coarse sweep over the
    ascending `lambdas`, corner, `nr` parameters between the corner's neighbours, the corner of the
    merged grid.  Returns (lambdas merged ascending, rn, xn, kappa, corner index, X merged)."""
    lam = np.sort(_f64(lambdas))
    X1 = np.stack([ref_ridge_qr(A, b, float(l), refine=refine) for l in lam])
    rn1, xn1 = lcurve_norms(A, b, X1)
    _, k = lcurve_curvature(lam, rn1, xn1)
    lam2 = lcurve_refine_grid(lam, k, nr)
    X2 = np.stack([ref_ridge_qr(A, b, float(l), refine=refine) for l in lam2])
    rn2, xn2 = lcurve_norms(A, b, X2)
    allm = np.concatenate([lam, lam2])
    order = np.argsort(allm, kind="stable")
    lamm = allm[order]
    rnm = np.concatenate([rn1, rn2])[order]
    xnm = np.concatenate([xn1, xn2])[order]
    Xm = np.concatenate([X1, X2])[order]
    kap, km = lcurve_curvature(lamm, rnm, xnm)
    return lamm, rnm, xnm, kap, km, Xm


# ------------------------------------------------------------------ BP2 ----
def bp2_r(Y, lam: float) -> np.ndarray:
    """R_BP2 from a Householder QR of [Y; sqrt(lambda) I] (Section 4.1), diag(R) > 0."""
    Y = _f64(Y)
    s, n = Y.shape
    R = np.zeros((n, n))
    rc = lib().orc_bp2_r(_ptr(Y), s, n, float(lam), _ptr(R))
    if rc:
        raise ValueError("zero column in the BP2 factorization")
    return R


def alg1_bp2(A, b, lambdas, sketch_kind: int, s: int, seed: int, tol: float, maxiter: int):
    """Algorithm 1 with the BP2 preconditioner (Section 4.1): the same sketch Y = XA, then for each
    lambda R from a QR of [Y; sqrt(l) I] in place of chol(Y^T Y + l I), LSQR, x = R^-1 y.
    Returns (X n x N, iterations, istop)."""
    A = _f64(A)
    Y = sketch_over(A, sketch_kind, seed, s)
    N = len(lambdas)
    X = np.zeros((A.shape[1], N))
    its, ist = np.zeros(N, dtype=int), np.zeros(N, dtype=int)
    for i, lam in enumerate(lambdas):
        R = bp2_r(Y, float(lam))
        X[:, i], its[i], ist[i] = lsqr_over_chol(A, b, float(lam), R, tol, maxiter)
    return X, its, ist
