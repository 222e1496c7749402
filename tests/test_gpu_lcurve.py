"""GPU parity of the L-curve (Section 4.3, Fig. 4) through the C ABI (tk_lcurve)
against the oracle's two-sweep L-curve on the same inputs.

The oracle solves every lambda with its dense reference (Householder QR plus
double-double refinement), forms the norms, the curvature, the corner, the
second sweep's parameters and the merged corner in plain float64.  The GPU
solves with the sketch-preconditioned LSQR (float64 or the mixed form) and
takes every decision itself.  The corner index is an argmax decided in float64
on both sides: it must agree unless the oracle's two best curvatures are
within the stated tolerance of each other.
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


@pytest.fixture(scope="module")
def lc_problem():
    m, n = 3000, 100
    sig = datagen.spectrum("log", n, hi=1.0, lo=1e-4)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(13, 1e-9, 1.0), seed=21, noise=1e-3)
    coarse = p.lambdas.numpy()
    ref = oracle.lcurve(p.A.numpy(), p.b.numpy(), coarse, nr=9)
    return p, coarse, ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lcurve_matches_oracle(tk, lc_problem, precision):
    p, coarse, (lam_o, rn_o, xn_o, kap_o, k_o, X_o) = lc_problem
    A, b = p.A.cuda(), p.b.cuda()
    if precision == "fp64":
        o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=400, seed=3)
    else:
        o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=400, seed=3, precision=tk.TK_PREC_MIXED)
    # coarse lambdas given in descending order: the call sorts them
    X, pts, k = tk.tk_lcurve(A, b, coarse[::-1].copy(), 9, o)
    lam = np.array([q["lam"] for q in pts])
    rn = np.array([q["rnorm"] for q in pts])
    xn = np.array([q["xnorm"] for q in pts])
    kap = np.array([q["curvature"] for q in pts])
    assert all(q["status"] == tk.TK_OK for q in pts), pts
    assert np.all(np.diff(lam) > 0)
    # the corner: largest interior curvature of the returned points
    assert 0 < k < len(pts) - 1 and kap[k] == kap[1:-1].max()
    tol_k = 1e-6 * np.abs(kap_o).max()
    second = np.sort(kap_o[1:-1])[-2]
    if kap_o[k_o] - second > 2 * tol_k:
        assert k == k_o, (k, k_o, kap[k], kap_o[k_o])
        # same corner, same second sweep: the parameters agree to the last bits of log/exp
        np.testing.assert_allclose(lam, lam_o, rtol=1e-13)
        np.testing.assert_allclose(rn, rn_o, rtol=1e-9)
        np.testing.assert_allclose(xn, xn_o, rtol=1e-9)
        np.testing.assert_allclose(kap, kap_o, rtol=1e-6, atol=tol_k)
        Xg = X.cpu().numpy()
        for i in range(len(lam)):
            assert rel(Xg[i], X_o[i]) < TOL_X, (lam[i], rel(Xg[i], X_o[i]))
    # the corner lies inside the grid, with its sweep-2 neighbours on both sides
    assert lam[k - 1] < lam[k] < lam[k + 1]


def test_lcurve_without_second_sweep_and_lowrank(tk, lc_problem):
    p, coarse, _ = lc_problem
    A, b = p.A.cuda(), p.b.cuda()
    X, pts, k = tk.tk_lcurve(A, b, coarse, 0, tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=400, seed=3))
    assert len(pts) == len(coarse)
    rn_o, xn_o = oracle.lcurve_norms(p.A.numpy(), p.b.numpy(), X.cpu().numpy())
    np.testing.assert_allclose([q["rnorm"] for q in pts], rn_o, rtol=1e-12)
    np.testing.assert_allclose([q["xnorm"] for q in pts], xn_o, rtol=1e-12)
    kap_o, k_o = oracle.lcurve_curvature(np.sort(coarse), rn_o, xn_o)
    np.testing.assert_allclose([q["curvature"] for q in pts], kap_o, rtol=1e-9, atol=1e-12)
    assert k == k_o
    # the low-rank preconditioner (Algorithm 3) through the same sweeps
    m, n = 3000, 120
    sig = datagen.spectrum("exp", n, tau=8.0)
    q = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(9, 1e-8, 1.0), seed=6)
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=60, seed=6, precond=tk.TK_PRECOND_LOWRANK, alpha=2.0)
    X, pts, k = tk.tk_lcurve(q.A.cuda(), q.b.cuda(), q.lambdas.numpy(), 5, o)
    Xg = X.cpu().numpy()
    for i, pt in enumerate(pts):
        xr = oracle.ref_ridge_qr(q.A.numpy(), q.b.numpy(), pt["lam"], refine=3)
        assert rel(Xg[i], xr) < TOL_X, (pt["lam"], rel(Xg[i], xr))
