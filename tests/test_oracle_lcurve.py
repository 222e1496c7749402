"""Pins for the oracle's L-curve (Section 4.3, Fig. 4), against facts that do not
come from the oracle itself.

The paper plots ||x_lambda|| against ||A x_lambda - b|| on log-log axes and picks
the corner; it does not say how the corner is found.  The reading taken is the
point of largest curvature of P(t) = ln ||A x - b||, Q(t) = ln ||x||, t = ln
lambda.  What pins the oracle:
  * the norms: the closed form of the ridge solution on an SVD-built A, and an
    independent library norm;
  * the three-point differences: exact on quadratic samples on any grid, and
    second-order convergence to the curvature of the closed-form L-curve, whose
    derivatives are taken by high-precision numerical differentiation (mpmath);
  * the corner: the maximiser of that analytic curvature, found by a
    golden-section search, lies within the second sweep's spacing of the
    oracle's two-sweep corner.
"""
import math

import mpmath
import numpy as np
import pytest

from paper_2203_07329_gb300 import datagen


def svd_problem(m=400, n=12, lo=1e-6, seed=11, noise=1e-3):
    sig = datagen.spectrum("log", n, hi=1.0, lo=lo)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(4, 1e-8, 1.0), seed=seed, noise=noise,
                                   keep_factors=True)
    return p


def closed_form_parts(p):
    """beta = U^T b, ||b_perp||^2, sigma (float64 numpy)."""
    U = p.U.numpy()
    b = p.b.numpy()
    beta = U.T @ b
    bperp2 = float(b @ b - beta @ beta)
    return p.sigma.numpy(), beta, bperp2


def closed_form_norms(sig, beta, bperp2, lam):
    f = sig * beta / (sig * sig + lam)
    g = lam * beta / (sig * sig + lam)
    return math.sqrt(float(g @ g) + bperp2), math.sqrt(float(f @ f))


def analytic_curvature(sig, beta, bperp2):
    """kappa(t) of the closed-form L-curve, derivatives by mpmath at 40 digits."""
    mpmath.mp.dps = 40
    s = [mpmath.mpf(float(v)) for v in sig]
    be = [mpmath.mpf(float(v)) for v in beta]
    bp = mpmath.mpf(bperp2)

    def P(t):
        lam = mpmath.exp(t)
        return mpmath.log(mpmath.fsum((lam * bi / (si * si + lam)) ** 2 for si, bi in zip(s, be)) + bp) / 2

    def Q(t):
        lam = mpmath.exp(t)
        return mpmath.log(mpmath.fsum((si * bi / (si * si + lam)) ** 2 for si, bi in zip(s, be))) / 2

    def kappa(t):
        t = mpmath.mpf(t)
        dP, ddP = mpmath.diff(P, t, 1), mpmath.diff(P, t, 2)
        dQ, ddQ = mpmath.diff(Q, t, 1), mpmath.diff(Q, t, 2)
        return float((dP * ddQ - ddP * dQ) / (dP * dP + dQ * dQ) ** mpmath.mpf(1.5))

    return kappa


def test_lcurve_norms_match_closed_form_and_library(orc):
    p = svd_problem()
    A, b = p.A.numpy(), p.b.numpy()
    sig, beta, bperp2 = closed_form_parts(p)
    lams = np.logspace(-8, 0, 5)
    X = np.stack([p.V.numpy() @ (sig * beta / (sig * sig + l)) for l in lams])
    rn, xn = orc.lcurve_norms(A, b, X)
    for i, l in enumerate(lams):
        r_cf, x_cf = closed_form_norms(sig, beta, bperp2, l)
        assert abs(rn[i] - r_cf) <= 1e-9 * r_cf and abs(xn[i] - x_cf) <= 1e-12 * x_cf
        assert abs(rn[i] - np.linalg.norm(b - A @ X[i])) <= 1e-12 * rn[i]


def test_curvature_is_exact_for_quadratic_samples_on_a_nonuniform_grid(orc):
    # P, Q quadratic in t: the three-point derivatives are exact at every interior sample
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(-20.0, 2.0, 15))
    aP, bP, cP = 0.03, 0.4, -1.0
    aQ, bQ, cQ = -0.05, -0.7, 2.0
    P = aP * t * t + bP * t + cP
    Q = aQ * t * t + bQ * t + cQ
    kap, k = orc.lcurve_curvature(np.exp(t), np.exp(P), np.exp(Q))
    dP, ddP = 2 * aP * t + bP, 2 * aP
    dQ, ddQ = 2 * aQ * t + bQ, 2 * aQ
    exact = (dP * ddQ - ddP * dQ) / (dP * dP + dQ * dQ) ** 1.5
    assert kap[0] == 0.0 and kap[-1] == 0.0
    np.testing.assert_allclose(kap[1:-1], exact[1:-1], rtol=1e-9, atol=1e-12)
    assert k == 1 + int(np.argmax(exact[1:-1]))


def test_curvature_converges_to_the_closed_form_lcurve(orc):
    p = svd_problem()
    sig, beta, bperp2 = closed_form_parts(p)
    kappa = analytic_curvature(sig, beta, bperp2)
    errs = []
    for h in (0.4, 0.2):
        t = np.arange(-14.0, -2.0 + 1e-9, h)
        lam = np.exp(t)
        rn = np.array([closed_form_norms(sig, beta, bperp2, l)[0] for l in lam])
        xn = np.array([closed_form_norms(sig, beta, bperp2, l)[1] for l in lam])
        kap, _ = orc.lcurve_curvature(lam, rn, xn)
        # compare at the common points t = -12, -10, ..., -4
        idx = [int(round((tt + 14.0) / h)) for tt in np.arange(-12.0, -3.9, 2.0)]
        errs.append(max(abs(kap[i] - kappa(t[i])) for i in idx))
    # second order: halving h divides the error by about 4
    assert errs[1] < errs[0] / 3.0, errs
    assert errs[1] < 0.05 * max(abs(kappa(tt)) for tt in np.arange(-12.0, -3.9, 2.0)), errs


def test_refine_grid_lies_strictly_between_the_neighbours(orc):
    lam = np.logspace(-9, 1, 11)
    for k in (1, 5, 9):
        g = orc.lcurve_refine_grid(lam, k, 7)
        assert np.all(g > lam[k - 1]) and np.all(g < lam[k + 1])
        d = np.diff(np.log(np.concatenate([[lam[k - 1]], g, [lam[k + 1]]])))
        np.testing.assert_allclose(d, d[0], rtol=1e-12)


def test_two_sweep_corner_is_the_maximum_curvature_of_the_closed_form(orc):
    p = svd_problem(m=300, n=12, lo=1e-6, noise=1e-3)
    A, b = p.A.numpy(), p.b.numpy()
    sig, beta, bperp2 = closed_form_parts(p)
    kappa = analytic_curvature(sig, beta, bperp2)
    coarse = np.logspace(-12, 0, 13)
    lamm, rnm, xnm, kap, km, Xm = orc.lcurve(A, b, coarse, nr=9)
    assert lamm.shape == (22,) and np.all(np.diff(lamm) > 0)
    # the analytic maximiser near the oracle's coarse corner: golden-section search in t
    lo, hi = math.log(lamm[max(km - 3, 0)]), math.log(lamm[min(km + 3, len(lamm) - 1)])
    g = (math.sqrt(5) - 1) / 2
    a, c = lo, hi
    x1, x2 = c - g * (c - a), a + g * (c - a)
    f1, f2 = kappa(x1), kappa(x2)
    for _ in range(40):
        if f1 > f2:
            c, x2, f2 = x2, x1, f1
            x1 = c - g * (c - a)
            f1 = kappa(x1)
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + g * (c - a)
            f2 = kappa(x2)
    t_star = (a + c) / 2
    spacing = max(math.log(lamm[km + 1]) - math.log(lamm[km]), math.log(lamm[km]) - math.log(lamm[km - 1]))
    assert abs(math.log(lamm[km]) - t_star) <= spacing, (lamm[km], math.exp(t_star), spacing)
    # the curve is L-shaped: the corner's curvature is positive and the largest of the grid
    assert kap[km] > 0 and kap[km] == kap.max()
