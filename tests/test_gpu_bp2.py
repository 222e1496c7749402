"""GPU parity of the BP2 preconditioner (Section 4.1: R from a QR of the partly
exact sketch [XA; sqrt(lambda) I]) through the C ABI, against the oracle's
Householder QR on the same sketch, and of solves that use it.

R is unique once its diagonal is positive, so the GPU factor is compared element
by element with the oracle's (and with the Cholesky factor of Y^T Y + lambda I,
the same factor in exact arithmetic) at the accuracy of a backward-stable QR:
||R_gpu - R_oracle|| <= 100 u kappa(B) ||B|| per row scale.  Solves reach the
oracle's reference x to 1e-10.
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


@pytest.mark.parametrize("s,n", [(64, 9), (300, 70), (130, 129), (1000, 200), (5, 1)])
def test_bp2_factor_matches_oracle(tk, s, n):
    g = torch.Generator().manual_seed(s + n)
    Y = torch.randn(s, n, dtype=torch.float64, generator=g)
    lams = [1e-8, 1e-2, 3.0]
    R, brk = tk.tk_bp2_factor(Y.cuda(), lams)
    assert brk == [0, 0, 0]
    Rg = R.cpu().numpy()
    Yn = Y.numpy()
    for i, lam in enumerate(lams):
        Ro = oracle.bp2_r(Yn, lam)
        B = np.vstack([Yn, np.sqrt(lam) * np.eye(n)])
        sv = np.linalg.svd(B, compute_uv=False)
        tol = 100 * 2.0 ** -53 * (sv[0] / sv[-1]) * sv[0]
        assert np.abs(np.tril(Rg[i], -1)).max() == 0.0 and np.all(np.diag(Rg[i]) > 0)
        assert np.abs(Rg[i] - Ro).max() <= tol, (lam, np.abs(Rg[i] - Ro).max(), tol)
        # R^T R = Y^T Y + lambda I
        G = Yn.T @ Yn + lam * np.eye(n)
        assert np.abs(Rg[i].T @ Rg[i] - G).max() <= 1e-13 * n * np.abs(G).max()


def test_bp2_nan_is_enumeric(tk):
    Y = torch.randn(50, 8, dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    Y[7, 3] = float("nan")
    import ctypes as C
    L = tk.lib()
    lam = np.array([1e-3])
    Rd = torch.empty((1, 8, 8), dtype=torch.float64, device="cuda")
    brk = (C.c_int * 1)()
    work = torch.empty(L.tk_bp2_factor_workspace(50, 8, 1), dtype=torch.uint8, device="cuda")
    st = L.tk_bp2_factor(tk._ptr(Y.cuda()), 50, 8, lam.ctypes.data_as(C.c_void_p), 1, tk._ptr(Rd), brk,
                         tk._ptr(work), work.numel(), None)
    assert st == tk.TK_ENUMERIC and brk[0] < 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_alg1_with_bp2_matches_oracle(tk, precision):
    sig = datagen.spectrum("log", 100, hi=1.0, lo=1e-5)
    p = datagen.make_ridge_problem(3000, 100, sig, datagen.log_lambdas(5, 1e-8, 1.0), seed=4)
    lams = p.lambdas.numpy()
    prec = tk.TK_PREC_FP64 if precision == "fp64" else tk.TK_PREC_MIXED
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=500, seed=8, precond=tk.TK_PRECOND_QR, precision=prec)
    res = tk.tk_solve(p.A.cuda(), p.b.cuda(), lams, o)
    X = res.X.cpu().numpy()
    Ad, bd = p.A.numpy(), p.b.numpy()
    for i, lam in enumerate(lams):
        xr = oracle.ref_ridge_qr(Ad, bd, float(lam), refine=3)
        assert rel(X[i], xr) < TOL_X, (lam, rel(X[i], xr), res.info[i])
    if precision == "fp64":
        _, it_o, _ = oracle.alg1_bp2(Ad, bd, lams, oracle.SKETCH_GAUSS, 500, 8, 1e-14, 500)
        its = np.array([q["iters"] for q in res.info])
        assert np.all(np.abs(its - it_o) <= 2), (its, it_o)
