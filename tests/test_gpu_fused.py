"""GPU parity of the fused LSQR step of the mixed form (lsqr_tc = 3): the two
products with A of one LSQR step (Algorithm 1 step 5 run by LSQR: u' = A R^-1 v
- alpha u and then A^T u'), computed in one kernel over one read of the 4-digit
slices of A, through the C ABI.

The products are checked against float64 products on the CPU of the same float32
inputs.  What bounds the error: A is rounded to its first 4 base-128 digits (28
bits below each row's maximum), W and u' to 4 digits below each lambda's
maximum, the level sums are exact, and the float32 sums over the bands of rows a
cluster of CTAs walks add one float32 rounding per band.  So every element is
within 2^-20 (u') and 2^-16 (A^T u') of |W| |A|^T + |c U| and |u'| |A| -- a
dropped leading digit level, a wrong row exponent or a lost band changes results
by orders of magnitude more.  Solves with the fused step reach the oracle's reference
x to 1e-10 like the other forms.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_07329_gb300 import datagen

pytestmark = pytest.mark.gpu

TOL_X = 1e-10


@pytest.fixture(scope="module")
def tk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_07329_gb300 import build
    build.build()
    from paper_2203_07329_gb300 import tikhonov
    tikhonov.lib()
    return tikhonov


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def inputs(m, n, count, seed, scale_rows=False, dtype=torch.float64):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(m, n, dtype=torch.float64, generator=g)
    if scale_rows:  # rows spread over 2^-20 .. 2^20: the row exponents differ inside a band
        A *= torch.pow(2.0, torch.randint(-20, 21, (m, 1), generator=g).double())
    A = A.to(dtype)
    W = torch.randn(count, n, dtype=torch.float32, generator=g)
    U = torch.randn(count, m, dtype=torch.float32, generator=g)
    coef = torch.randn(count, dtype=torch.float64, generator=g)
    return A, W, U, coef


# n covers clusters of 1 CTA (<= 256 columns), 2, 4 and 8 CTAs, CTAs wholly beyond the last column
# (n = 700: 4 x 256 columns; n = 1500: 8 x 256), a ragged last 64-column box, and 1 .. 32 lambda;
# m spans several bands and a ragged one
@pytest.mark.parametrize("m,n,count", [(129, 64, 1), (1000, 200, 5), (5000, 300, 8), (777, 700, 32),
                                       (3001, 1000, 32), (20000, 2048, 17), (4096, 1500, 31)])
@pytest.mark.parametrize("mode", [1, 0])
def test_step_products_match_float64(tk, m, n, count, mode):
    A, W, U, coef = inputs(m, n, count, seed=m + n + count)
    Ad, Wd, Ud, cd = A.numpy(), W.double().numpy(), U.double().numpy(), coef.numpy()
    Uc = U.cuda()
    G = tk.tk_lsqr_step_products(A.cuda(), W.cuda(), Uc, coef.cuda(), mode=mode).cpu().numpy()
    Ug = Uc.cpu().double().numpy()
    U_ref = Wd @ Ad.T + cd[:, None] * Ud
    U_mag = np.abs(Wd) @ np.abs(Ad).T + np.abs(cd[:, None] * Ud)
    assert np.all(np.abs(Ug - U_ref) <= 2.0 ** -20 * U_mag), np.max(np.abs(Ug - U_ref) / U_mag)
    # A^T u' of the u' the kernel wrote
    G_ref = Ug @ Ad
    G_mag = np.abs(Ug) @ np.abs(Ad)
    assert np.all(np.abs(G - G_ref) <= 2.0 ** -16 * G_mag), np.max(np.abs(G - G_ref) / G_mag)


@pytest.mark.parametrize("m,n,count", [(3000, 700, 9), (2000, 2048, 32)])
def test_step_products_rows_of_very_different_scale(tk, m, n, count):
    # the row exponent of A moves onto u' before its digits are taken: rows 2^40 apart in one band
    A, W, U, coef = inputs(m, n, count, seed=5, scale_rows=True)
    Uc = U.cuda()
    G = tk.tk_lsqr_step_products(A.cuda(), W.cuda(), Uc, None, mode=1).cpu().numpy()
    Ad, Wd = A.numpy(), W.double().numpy()
    Ug = Uc.cpu().double().numpy()
    U_ref = Wd @ Ad.T
    assert np.all(np.abs(Ug - U_ref) <= 2.0 ** -20 * (np.abs(Wd) @ np.abs(Ad).T))
    G_ref = Ug @ Ad
    # a row 2^-40 below the band's largest loses its digits: bounded normwise per lambda
    for l in range(count):
        err = np.abs(G[l] - G_ref[l]).max()
        assert err <= 2.0 ** -16 * np.abs(Ug[l]) @ np.abs(Ad).max(axis=1), (l, err)


def test_step_products_float32_input(tk):
    A, W, U, coef = inputs(2500, 640, 24, seed=8, dtype=torch.float32)
    Uc = U.cuda()
    G = tk.tk_lsqr_step_products(A.cuda(), W.cuda(), Uc, coef.cuda(), mode=1).cpu().numpy()
    Ad, Wd, Ud, cd = A.double().numpy(), W.double().numpy(), U.double().numpy(), coef.numpy()
    Ug = Uc.cpu().double().numpy()
    U_ref = Wd @ Ad.T + cd[:, None] * Ud
    assert np.all(np.abs(Ug - U_ref) <= 2.0 ** -20 * (np.abs(Wd) @ np.abs(Ad).T + np.abs(cd[:, None] * Ud)))
    G_ref = Ug @ Ad
    assert np.all(np.abs(G - G_ref) <= 2.0 ** -16 * (np.abs(Ug) @ np.abs(Ad)))


@pytest.mark.parametrize("mode", [1, 0])
def test_step_products_nan_row(tk, mode):
    # a non-finite row of A: its u' entries are NaN for every lambda, so every entry of A^T u' is NaN;
    # the other rows of u' stay finite
    A, W, U, coef = inputs(1000, 300, 6, seed=2)
    A[417, 123] = float("nan")
    Uc = U.cuda()
    G = tk.tk_lsqr_step_products(A.cuda(), W.cuda(), Uc, coef.cuda(), mode=mode).cpu().numpy()
    Ug = Uc.cpu().numpy()
    assert np.all(np.isnan(Ug[:, 417]))
    assert np.all(np.isfinite(np.delete(Ug, 417, axis=1)))
    assert np.all(np.isnan(G))


def test_step_products_rejects_wide_and_many(tk):
    import ctypes as C
    L = tk.lib()
    A = torch.zeros(100, 2049, dtype=torch.float64, device="cuda")
    b = torch.zeros(100, dtype=torch.float64, device="cuda")
    prob = tk.make_problem(A, b)
    W = torch.zeros(4, 2049, dtype=torch.float32, device="cuda")
    U = torch.zeros(4, 100, dtype=torch.float32, device="cuda")
    G = torch.zeros(4, 2049, dtype=torch.float64, device="cuda")
    nb = L.tk_lsqr_step_products_workspace(100, 2049, 4)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    st = L.tk_lsqr_step_products(C.byref(prob), tk._ptr(W), 4, tk._ptr(U), None, tk._ptr(G), 1, tk._ptr(work), nb,
                                 None)
    assert st == tk.TK_EINVAL
    st = L.tk_lsqr_step_products(C.byref(prob), tk._ptr(W), 33, tk._ptr(U), None, tk._ptr(G), 0, tk._ptr(work), nb,
                                 None)
    assert st == tk.TK_EINVAL


def problem(m, n, N, lo=1e-5, lam=(1e-6, 1.0), seed=3, dtype=torch.float64):
    sig = datagen.spectrum("log", min(m, n), hi=1.0, lo=lo)
    return datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(N, *lam), seed=seed, dtype=dtype)


# m n > 2^24 and more than 16 lambda: the digit products run; N = 40 starts above the fused step's
# 32 lambda (unfused steps) and switches to the fused step as lambda converge
@pytest.mark.parametrize("m,n,N,dtype", [(20000, 1000, 24, torch.float64), (33333, 600, 40, torch.float32),
                                         (9000, 2048, 17, torch.float64)])
def test_mixed_solve_with_fused_step(tk, m, n, N, dtype):
    p = problem(m, n, N, dtype=dtype)
    lams = p.lambdas.numpy()
    A, b = p.A.cuda(), p.b.cuda()
    o3 = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=4 * n, seed=9, precision=tk.TK_PREC_MIXED, lsqr_tc=3)
    tk.tk_profile_enable(True)
    try:
        tk.tk_profile_collect()
        res = tk.tk_solve(A, b, lams, o3)
        prof = tk.tk_profile_collect()
    finally:
        tk.tk_profile_enable(False)
    assert prof["lsqr_step_fused"]["launches"] > 0
    X = res.X.cpu().numpy()
    o2 = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=4 * n, seed=9, precision=tk.TK_PREC_MIXED, lsqr_tc=2)
    res2 = tk.tk_solve(A, b, lams, o2)
    Ad, bd = p.A.double().numpy(), p.b.numpy()
    # the oracle's reference at the smallest lambda (the hardest; the dense reference is slow at these
    # sizes), and every lambda against the unfused digit products' x (both within 1e-10 of the truth)
    xr = oracle.ref_ridge_qr(Ad, bd, float(lams[0]), refine=3)
    assert rel(X[0], xr) < TOL_X, (lams[0], rel(X[0], xr), res.info[0])
    X2 = res2.X.cpu().numpy()
    for i in range(N):
        assert res.info[i]["status"] == 0
        assert rel(X[i], X2[i]) < 2 * TOL_X, (lams[i], rel(X[i], X2[i]))
    # float32-accurate products either way: comparable iteration counts
    it3 = sum(q["iters"] for q in res.info)
    it2 = sum(q["iters"] for q in res2.info)
    assert it3 <= 1.2 * it2 + 5, (it3, it2)
