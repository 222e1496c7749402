"""Parity at the full workload sizes, in the launch configuration bench.py times.

The oracle cannot run Algorithms 1-2 at these sizes in test time, so it
computes the reference for sampled lambdas one by one: the closed form
x = V diag(sigma/(sigma^2 + l)) U^T b from the generator's factors, refined
against the stored A with double-double normal-equation residuals
(oracle.ref_ridge_refine).  That reference is accurate far below 1e-10.

Tolerance per lambda: 1e-10, or -- where float64 itself cannot reach it --
8x the conditioning floor of any backward-stable float64 solve,
u (kappa_B + kappa_B^2 ||r|| / (||B|| ||x||)) with kappa_B^2 = (s1^2 + l)/(sn^2 + l).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2203_07329_gb300 import datagen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def tk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_07329_gb300 import build
    build.build()
    from paper_2203_07329_gb300 import tikhonov
    tikhonov.lib()
    return tikhonov


def floor_tol(sig, lam, rnorm, xnorm):
    kB = math.sqrt((sig.max() ** 2 + lam) / (sig.min() ** 2 + lam))
    Bn = math.sqrt(sig.max() ** 2 + lam)
    return U64 * (kB + kB * kB * rnorm / (Bn * xnorm))


def reference(prob, lam, x0_dev=None):
    """Closed form from the generator's factors, then double-double refinement."""
    U, V = prob.U, prob.V
    sig = prob.sigma.to(U.device)
    c = (U.T @ prob.b) * (sig / (sig * sig + lam))
    x0 = (V @ c).cpu().numpy()
    A = prob.A.double().cpu().numpy() if prob.A.dtype != torch.float64 else prob.A.cpu().numpy()
    return oracle.ref_ridge_refine(A, prob.b.cpu().numpy(), lam, V.cpu().numpy(), prob.sigma.numpy(), x0, steps=2), A


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_over_262144x2048_srht(tk, precision):
    prob, w = datagen.workload_problem("ridge_over_262144x2048_f64", device="cuda", keep_factors=True)
    lams = prob.lambdas.numpy()
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=w["s"], seed=1, tol=1e-14,
                        precision=tk.TK_PREC_FP64 if precision == "fp64" else tk.TK_PREC_MIXED)
    res = tk.tk_solve(prob.A, prob.b, lams, o)
    X = res.X.cpu().numpy()
    assert all(q["status"] == 0 for q in res.info), res.info
    sig = prob.sigma.numpy()
    for i in (0, len(lams) // 2, len(lams) - 1):
        lam = float(lams[i])
        xr, A = reference(prob, lam)
        r = prob.b.cpu().numpy() - A @ xr
        tol = max(1e-10, 8 * floor_tol(sig, lam, np.linalg.norm(r), np.linalg.norm(xr)))
        err = np.linalg.norm(X[i] - xr) / np.linalg.norm(xr)
        print(f"{precision} lambda={lam:.1e} rel.err={err:.2e} tol={tol:.2e} iters={res.info[i]['iters']}")
        assert err < tol, (lam, err, tol)
    # iterations bounded independently of lambda (Lemma 2.1: kappa(B R^-1) <= kappa(X U_A) for
    # every lambda).  With s = 4n, kappa(X U_A) <= 3 (eps ~ sqrt(n/s) = 1/2), so the rate is
    # <= 1/2 per step and tol 1e-14 needs at most ~1.5 ln(1e14)/ln 2 + 5 = 75 steps (float64);
    # the mixed form restarts LSQR per correction, 4 corrections at most.
    its = [q["iters"] for q in res.info]
    cap = 75 if precision == "fp64" else 4 * 40
    assert max(its) <= cap, its
    # bounded uniformly in lambda (Lemma 2.1: kappa(B R^-1) <= kappa(X U_A) for every lambda): no lambda
    # needs far more iterations per LSQR run (the mixed form restarts LSQR once per refinement round)
    # than the median one -- unpreconditioned LSQR would grow like kappa_B ~ 1/sqrt(lambda) as lambda -> 0.
    # Large lambda converge faster (better conditioned), so the check is one-sided.
    per_run = np.array([q["iters"] / max(q["refine_steps"], 1) for q in res.info])
    assert per_run.max() <= 1.5 * np.median(per_run) + 5, per_run


def test_under_2048x262144_srht(tk):
    prob, w = datagen.workload_problem("ridge_under_2048x262144_f64", device="cuda", keep_factors=True)
    lams = prob.lambdas.numpy()
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=w["s"], seed=1, tol=1e-14)
    res = tk.tk_solve(prob.A, prob.b, lams, o)
    X = res.X.cpu().numpy()
    assert all(q["status"] == 0 for q in res.info), res.info
    sig = prob.sigma.numpy()
    for i in (0, len(lams) - 1):
        lam = float(lams[i])
        xr, A = reference(prob, lam)
        r = prob.b.cpu().numpy() - A @ xr
        tol = max(1e-10, 8 * floor_tol(sig, lam, np.linalg.norm(r), np.linalg.norm(xr)))
        err = np.linalg.norm(X[i] - xr) / np.linalg.norm(xr)
        print(f"under lambda={lam:.1e} rel.err={err:.2e} tol={tol:.2e} iters={res.info[i]['iters']}")
        assert err < tol, (lam, err, tol)


def refine_reference(A64, b, lam, U, V, sig, steps):
    x0 = V @ ((sig / (sig * sig + lam)) * (U.T @ b))
    return oracle.ref_ridge_refine(A64, b, lam, V, sig, x0, steps=steps)


def test_over_1048576x4096_f32_mixed_tensor_core_sketch(tk):
    prob, w = datagen.workload_problem("ridge_over_1048576x4096_f32", device="cuda", keep_factors=True)
    lams = prob.lambdas.numpy()
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=w["s"], seed=1, precision=tk.TK_PREC_MIXED)
    res = tk.tk_solve(prob.A, prob.b, lams, o)
    X = res.X.cpu().numpy()
    assert all(q["status"] == 0 for q in res.info), res.info
    A64 = prob.A.cpu().double().numpy()
    b = prob.b.cpu().numpy()
    U, V = prob.U.cpu().double().numpy(), prob.V.cpu().double().numpy()
    sig = prob.sigma.numpy()
    del prob
    for i in (0, len(lams) - 1):
        lam = float(lams[i])
        # float32 factors: the closed form is good to ~1e-7; each double-double
        # step contracts by ~||A^T A - V S^2 V^T|| / lambda, so 4 steps reach far below 1e-10
        xr = refine_reference(A64, b, lam, U, V, sig, steps=4)
        err = np.linalg.norm(X[i] - xr) / np.linalg.norm(xr)
        print(f"f32 mixed lambda={lam:.1e} rel.err={err:.2e} iters={res.info[i]['iters']} "
              f"refine={res.info[i]['refine_steps']}")
        assert err < 1e-10, (lam, err)


def test_uneven_256_problems_full_size(tk):
    import math
    probs = datagen.uneven_batch(256, device="cuda", dtype=torch.float32, keep_factors=True)
    pairs, opts = [], []
    for p in probs:
        n = p.A.shape[1]
        lam_min = float(p.lambdas.min())
        if p.meta["lowrank"]:
            sd = float(np.sum(1.0 / (1.0 + lam_min / (p.sigma.numpy() ** 2))))
            opts.append(tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=min(n, 2 * math.ceil(sd)), seed=1,
                                        precond=tk.TK_PRECOND_LOWRANK, alpha=2.0, precision=tk.TK_PREC_MIXED))
        else:
            opts.append(tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=min(4 * n, p.A.shape[0]), seed=1,
                                        precision=tk.TK_PREC_MIXED))
        pairs.append((p.A, p.b))
    lams = np.stack([p.lambdas.numpy() for p in probs])
    Xs, infos, st = tk.tk_solve_batched(pairs, lams, opts)
    assert st == tk.TK_OK
    for k in range(0, 256, 37):
        p = probs[k]
        A64 = p.A.cpu().double().numpy()
        b = p.b.cpu().numpy()
        U, V = p.U.cpu().double().numpy(), p.V.cpu().double().numpy()
        sig = p.sigma.numpy()
        X = Xs[k].cpu().numpy()
        for i in (0, lams.shape[1] - 1):
            lam = float(lams[k, i])
            # float32 factors: the double-double refinement contracts by ~1e-7/lambda per step
            xr = refine_reference(A64, b, lam, U, V, sig, steps=10)
            err = np.linalg.norm(X[i] - xr) / np.linalg.norm(xr)
            print(f"problem {k} m={A64.shape[0]} n={A64.shape[1]} lowrank={p.meta['lowrank']} "
                  f"lambda={lam:.1e} rel.err={err:.2e}")
            assert err < 1e-10, (k, lam, err)
