"""GPU tests of the boundary's solve-level behaviour: the warm start x0, the
handle calls, and the per-lambda failure statuses (iteration cap, non-finite
input, a bounded device wait that gives up), all called through the C ABI.

Warm-started solves are compared with the oracle's reference solution of the
ridge problem (1.2) (dense QR + double-double refinement), whose minimiser does
not depend on the starting point.  Failures are made on the host (a NaN written
into A or b, maxiter = 1, a wait on a barrier nothing arrives at); no test
faults or hangs the GPU.
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


def problem(m, n, lo=1e-4, N=4, lam=(1e-6, 1.0), seed=3, dtype=torch.float64):
    sig = datagen.spectrum("log", min(m, n), hi=1.0, lo=lo)
    return datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(N, *lam), seed=seed, dtype=dtype)


def reference(p, lams):
    A, b = p.A.double().numpy(), p.b.numpy()
    return np.stack([oracle.ref_ridge_qr(A, b, float(l), refine=3) for l in lams])


@pytest.fixture(scope="module")
def allow_all(tk):
    return (tk.TK_OK, tk.TK_ENOCONV, tk.TK_ENOTSPD, tk.TK_ENUMERIC)


# ------------------------------------------------------------- warm start ---
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warm_start_from_the_solution_needs_few_iterations(tk, precision):
    p = problem(3000, 128, lo=1e-4, N=4, lam=(1e-5, 1.0))
    lams = p.lambdas.numpy()
    A, b = p.A.cuda(), p.b.cuda()
    prec = tk.TK_PREC_FP64 if precision == "fp64" else tk.TK_PREC_MIXED
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=512, seed=4, precision=prec)
    cold = tk.tk_solve(A, b, lams, o)
    Xr = reference(p, lams)
    x0 = torch.from_numpy(Xr).cuda().contiguous()
    warm = tk.tk_solve(A, b, lams, o, x0=x0)
    X = warm.X.cpu().numpy()
    for i in range(len(lams)):
        assert rel(X[i], Xr[i]) < TOL_X, (lams[i], rel(X[i], Xr[i]), warm.info[i])
        assert warm.info[i]["status"] == tk.TK_OK
    it_c = np.array([q["iters"] for q in cold.info])
    it_w = np.array([q["iters"] for q in warm.info])
    # starting at the minimiser, the correction problem's right-hand side is (nearly) orthogonal to the
    # range of the preconditioned operator: far fewer iterations than from zero
    assert np.all(it_w < it_c), (it_w, it_c)
    if precision == "mixed":
        assert all(q["refine_steps"] == 1 for q in warm.info), warm.info


def test_warm_start_from_a_perturbed_point_reaches_the_same_minimiser(tk):
    # x0 far from the solution: the minimiser of (1.2) is unique, so x0 only changes the path
    p = problem(2500, 100, lo=1e-5, N=3, lam=(1e-6, 1e-1))
    lams = p.lambdas.numpy()
    A, b = p.A.cuda(), p.b.cuda()
    Xr = reference(p, lams)
    g = torch.Generator().manual_seed(1)
    x0 = (torch.from_numpy(Xr) + torch.randn(Xr.shape, dtype=torch.float64, generator=g)).cuda().contiguous()
    for prec in (tk.TK_PREC_FP64, tk.TK_PREC_MIXED):
        for sched in (tk.TK_SCHED_BATCHED, tk.TK_SCHED_ONE_AT_A_TIME):
            o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=400, seed=2, precision=prec, schedule=sched)
            X = tk.tk_solve(A, b, lams, o, x0=x0).X.cpu().numpy()
            for i in range(len(lams)):
                assert rel(X[i], Xr[i]) < TOL_X, (prec, sched, lams[i], rel(X[i], Xr[i]))


def test_warm_start_lowrank(tk):
    m, n = 3000, 120
    sig = datagen.spectrum("exp", n, tau=8.0)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(4, 1e-6, 1.0), seed=6)
    lams = p.lambdas.numpy()[::-1].copy()
    A, b = p.A.cuda(), p.b.cuda()
    Xr = reference(p, lams)
    x0 = torch.from_numpy(0.5 * Xr).cuda().contiguous()
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=60, seed=6, precond=tk.TK_PRECOND_LOWRANK, alpha=2.0)
    X = tk.tk_solve(A, b, lams, o, x0=x0).X.cpu().numpy()
    for i in range(len(lams)):
        assert rel(X[i], Xr[i]) < TOL_X, (lams[i], rel(X[i], Xr[i]))


# ---------------------------------------------------------------- handles ---
def test_handle_solves_equal_workspace_solves(tk):
    p = problem(2000, 96, N=3)
    lams = p.lambdas.numpy()
    A, b = p.A.cuda(), p.b.cuda()
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=384, seed=7)
    X_ws = tk.tk_solve(A, b, lams, o).X
    with tk.Handle() as h:
        assert h.workspace_bytes() == 0
        X_h = h.solve(A, b, lams, o).X
        grown = h.workspace_bytes()
        assert grown >= tk.workspace_size(tk.make_problem(A, b), len(lams), o)
        X_h2 = h.solve(A, b, lams, o).X  # same shapes: no growth
        assert h.workspace_bytes() == grown
        # a batch of two problems through the same handle
        q = problem(1500, 64, N=3, seed=8)
        lam2 = np.stack([lams, q.lambdas.numpy()])
        Xs, infos, st = h.solve_batched([(A, b), (q.A.cuda(), q.b.cuda())], lam2, o)
        assert st == tk.TK_OK
    assert torch.equal(X_ws, X_h) and torch.equal(X_h, X_h2)
    assert torch.allclose(Xs[0], X_ws, rtol=1e-12, atol=1e-12 * float(X_ws.abs().max()))


# --------------------------------------------------------------- failures ---
def test_iteration_cap_is_enoconv(tk):
    p = problem(2000, 80, N=3)
    lams = p.lambdas.numpy()
    A, b = p.A.cuda(), p.b.cuda()
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=320, seed=1, maxiter=1)
    r = tk.tk_solve(A, b, lams, o)
    assert r.status == tk.TK_ENOCONV
    assert all(q["status"] == tk.TK_ENOCONV and q["istop"] == 7 and q["iters"] == 1 for q in r.info), r.info


def test_refinement_cap_is_enoconv(tk):
    p = problem(2000, 80, N=3, dtype=torch.float32)
    lams = p.lambdas.numpy()
    A, b = p.A.cuda(), p.b.cuda()
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=320, seed=1, precision=tk.TK_PREC_MIXED, max_refine=1)
    r = tk.tk_solve(A, b, lams, o)
    assert r.status == tk.TK_ENOCONV
    assert all(q["status"] == tk.TK_ENOCONV and q["refine_steps"] == 1 for q in r.info), r.info


@pytest.mark.parametrize("where", ["A", "b"])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_f64pipe"])
def test_non_finite_input_is_enumeric(tk, allow_all, where, precision):
    p = problem(2000, 80, N=3)
    lams = p.lambdas.numpy()
    A, b = p.A.clone(), p.b.clone()
    if where == "A":
        A[777, 13] = float("nan")
    else:
        b[1234] = float("nan")
    A, b = A.cuda(), b.cuda()
    kw = dict(sketch=tk.TK_SKETCH_SRHT, s=320, seed=1)
    if precision != "fp64":
        kw.update(precision=tk.TK_PREC_MIXED, max_refine=8)
    if precision == "mixed_f64pipe":
        kw.update(emulate_fp64=0, lsqr_tc=0)
    r = tk.tk_solve(A, b, lams, tk.opts_default(**kw), allow=allow_all)
    assert r.status == tk.TK_ENUMERIC, (r.status, r.info)
    assert all(q["status"] == tk.TK_ENUMERIC for q in r.info), r.info
    # the refinement stops on it within its round limit
    assert all(q["refine_steps"] <= 8 for q in r.info)
    # the context is still usable: a clean solve afterwards succeeds
    q = problem(500, 20, N=2)
    assert tk.tk_solve(q.A.cuda(), q.b.cuda(), q.lambdas.numpy()).status == tk.TK_OK


def test_cholesky_reports_nan_as_enumeric(tk, allow_all):
    import ctypes as C
    n = 150
    g = torch.Generator().manual_seed(3)
    Y = torch.randn(400, n, dtype=torch.float64, generator=g)
    Cm = Y.T @ Y
    Cm[40, 40] = float("nan")
    Cd = Cm.cuda().contiguous()
    lam = np.array([1e-3, 1.0])
    L = tk.lib()
    for emulate in (False, True):
        Rd = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
        brk = (C.c_int * 2)()
        fn = L.tk_cholesky_shifted_emulated if emulate else L.tk_cholesky_shifted
        need = (L.tk_cholesky_emulated_workspace if emulate else L.tk_cholesky_workspace)(n, 2)
        work = torch.empty(need, dtype=torch.uint8, device="cuda")
        st = fn(tk._ptr(Cd), n, lam.ctypes.data_as(C.c_void_p), 2, tk._ptr(Rd), brk, tk._ptr(work), work.numel(),
                None)
        torch.cuda.synchronize()
        assert st == tk.TK_ENUMERIC, (emulate, st)
        assert all(v < 0 for v in brk), list(brk)  # NaN pivots are marked negative


def test_bounded_wait_gives_up_with_etimeout(tk):
    # the same bounded mbarrier wait every tensor-core pipeline uses, on a barrier nothing arrives at
    for budget_us in (1000, 20000):
        assert tk.tk_wait_selftest(budget_us) == tk.TK_ETIMEOUT
    # the context stays usable
    p = problem(800, 30, N=2)
    r = tk.tk_solve(p.A.cuda(), p.b.cuda(), p.lambdas.numpy(),
                    tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=120, seed=1))
    assert r.status == tk.TK_OK
