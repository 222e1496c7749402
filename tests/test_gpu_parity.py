"""GPU parity: every step of the CUDA path, called through the C ABI, against the
CPU oracle on the same seeded inputs.

Integer work (signs, sampled rows, truncation ranks) is compared bit for bit.
Floating point: x_lambda within 1e-10 relative of the oracle's reference
solution (dense QR + double-double refinement) for the float64 path and for the
mixed form after refinement; intermediate floating-point steps within the
rounding-level tolerances stated per test.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2203_07329_gb300 import datagen

pytestmark = pytest.mark.gpu

TOL_X = 1e-10  # relative error of x_lambda against the oracle (float64 and mixed)


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


def problem(m, n, lo=1e-4, kind="log", tau=50.0, N=4, lam=(1e-6, 1.0), seed=3, dtype=torch.float64):
    k = min(m, n)
    sig = datagen.spectrum("log", k, hi=1.0, lo=lo) if kind == "log" else datagen.spectrum("exp", k, tau=tau)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(N, *lam), seed=seed, dtype=dtype)
    return p


def to_dev(p):
    return p.A.cuda(), p.b.cuda()


# ------------------------------------------------------------- draws -------
@pytest.mark.parametrize("mp,s", [(1, 1), (64, 0), (64, 16), (64, 64), (1000, 333), (1 << 14, 4096),
                                  (1 << 18, 8192), (1 << 20, 5)])
def test_draws_bit_exact(tk, mp, s):
    signs, rows = tk.tk_sketch_draw(7, mp, s)
    np.testing.assert_array_equal(signs.cpu().numpy(), oracle.draw_signs(7, mp))
    np.testing.assert_array_equal(rows.cpu().numpy(), oracle.draw_rows(7, mp, s))


# ---------------------------------------------------------- sketches -------
@pytest.mark.parametrize("m,n,s", [(1000, 37, 300), (512, 16, 512), (3000, 130, 700), (700, 1, 50)])
def test_srht_over_matches_oracle(tk, m, n, s):
    A = torch.randn(m, n, dtype=torch.float64, generator=torch.Generator().manual_seed(m + n))
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=s, seed=11)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    Yo = oracle.srht_over(A.numpy(), 11, s)
    # the same butterfly tree in the same order: rounding-identical up to FMA-free adds
    np.testing.assert_allclose(Y, Yo, rtol=1e-13, atol=1e-13 * np.abs(Yo).max())


def test_srht_over_two_pass_size(tk):
    # 2^11 rows: the transform runs in two shared-memory passes (9 + 2 bits)
    m, n, s = 2000, 20, 256
    A = torch.randn(m, n, dtype=torch.float64, generator=torch.Generator().manual_seed(5))
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=s, seed=2)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    Yo = oracle.srht_over(A.numpy(), 2, s)
    np.testing.assert_allclose(Y, Yo, rtol=1e-13, atol=1e-13 * np.abs(Yo).max())


@pytest.mark.parametrize("m,n,s", [(20, 1000, 100), (3, 5000, 64)])
def test_srht_under_matches_oracle(tk, m, n, s):
    A = torch.randn(m, n, dtype=torch.float64, generator=torch.Generator().manual_seed(9))
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=s, seed=4)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    Yo = oracle.srht_under(A.numpy(), 4, s)
    np.testing.assert_allclose(Y, Yo, rtol=1e-13, atol=1e-13 * np.abs(Yo).max())


@pytest.mark.parametrize("m,n,s", [(500, 30, 120), (130, 65, 65)])
def test_gauss_over_matches_oracle(tk, m, n, s):
    A = torch.randn(m, n, dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=s, seed=8)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    Yo = oracle.gauss_over(A.numpy(), 8, s)
    # Gaussian entries agree to libm-vs-CUDA rounding (~1e-16); sums differ in order
    np.testing.assert_allclose(Y, Yo, rtol=1e-12, atol=1e-12 * np.abs(Yo).max())


def test_gauss_under_matches_oracle(tk):
    A = torch.randn(12, 300, dtype=torch.float64, generator=torch.Generator().manual_seed(2))
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=40, seed=8)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    Yo = oracle.gauss_under(A.numpy(), 8, 40)
    np.testing.assert_allclose(Y, Yo, rtol=1e-12, atol=1e-12 * np.abs(Yo).max())


# ------------------------------------------------------ Gram / Cholesky ----
@pytest.mark.parametrize("r,c", [(300, 70), (64, 64), (1000, 129)])
def test_gram_matches_oracle(tk, r, c):
    Y = torch.randn(r, c, dtype=torch.float64, generator=torch.Generator().manual_seed(r))
    G = tk.tk_gram(Y.cuda(), True).cpu().numpy()
    np.testing.assert_allclose(G, oracle.gram_tn(Y.numpy()), rtol=1e-12, atol=1e-12 * r)
    G2 = tk.tk_gram(Y.T.contiguous().cuda(), False).cpu().numpy()
    np.testing.assert_allclose(G2, oracle.gram_nt(Y.T.contiguous().numpy()), rtol=1e-12, atol=1e-12 * r)


@pytest.mark.parametrize("r,c", [(300, 70), (1000, 129), (2100, 333), (5, 1)])
def test_emulated_gram_has_float64_accuracy(tk, r, c):
    # C = Y^T Y on the BF16 tensor cores from exact column slices: every upper entry within the
    # float64 GEMM bound relative to (|Y|^T |Y|), columns of Y over 8 decades of scale
    gen = torch.Generator().manual_seed(r + c)
    Y = torch.randn(r, c, generator=gen, dtype=torch.float64) * torch.logspace(0, -8, c, dtype=torch.float64)
    G = tk.tk_gram(Y.cuda(), True, emulate=True).cpu().numpy()
    Yl = Y.numpy().astype(np.longdouble)
    Gref = Yl.T @ Yl
    scale = np.abs(Y.numpy()).T @ np.abs(Y.numpy())
    iu = np.triu_indices(c)
    err = np.abs((G[iu] - Gref[iu]).astype(np.float64)) / scale[iu]
    assert float(err.max()) < 8 * 2.0 ** -53 * math.sqrt(r), float(err.max())
    # the oracle's Gram matrix agrees on the upper triangle, relative to the same scale
    d = np.abs(G[iu] - oracle.gram_tn(Y.numpy())[iu]) / scale[iu]
    assert float(d.max()) < 16 * 2.0 ** -53 * math.sqrt(r), float(d.max())


@pytest.mark.parametrize("n", [1, 63, 64, 100, 200])
def test_cholesky_matches_oracle(tk, n):
    Y = torch.randn(3 * n + 5, n, dtype=torch.float64, generator=torch.Generator().manual_seed(n))
    Cm = (Y.T @ Y).numpy()
    lams = [1e-8, 1e-3, 1.0]
    R, brk = tk.tk_cholesky_shifted(torch.from_numpy(Cm).cuda(), lams)
    R = R.cpu().numpy()
    assert brk == [0, 0, 0]
    for i, lam in enumerate(lams):
        Ro, info = oracle.cholesky_shifted(Cm, lam)
        assert info == 0
        np.testing.assert_allclose(R[i], Ro, rtol=1e-9, atol=1e-11 * np.abs(Ro).max())
        np.testing.assert_allclose(R[i].T @ R[i], Cm + lam * np.eye(n), rtol=1e-12, atol=1e-12 * np.abs(Cm).max())


@pytest.mark.parametrize("n", [63, 64, 129, 333, 700])
def test_emulated_cholesky_matches_oracle(tk, n):
    # trailing updates on the tensor cores (exact slices, float64 accuracy): the factors agree with
    # the oracle's and with the float64 factorization to float64 rounding
    gen = torch.Generator().manual_seed(n + 1)
    Y = torch.randn(3 * n + 5, n, dtype=torch.float64, generator=gen) * torch.logspace(0, -3, n, dtype=torch.float64)
    Cm = (Y.T @ Y).numpy()
    lams = [1e-8, 1e-4, 1.0]
    Re, brk = tk.tk_cholesky_shifted(torch.from_numpy(Cm).cuda(), lams, emulate=True)
    Rn, _ = tk.tk_cholesky_shifted(torch.from_numpy(Cm).cuda(), lams)
    Re, Rn = Re.cpu().numpy(), Rn.cpu().numpy()
    assert brk == [0, 0, 0]
    for i, lam in enumerate(lams):
        Ro, info = oracle.cholesky_shifted(Cm, lam)
        assert info == 0
        np.testing.assert_allclose(Re[i], Ro, rtol=1e-9, atol=1e-11 * np.abs(Ro).max())
        np.testing.assert_allclose(Re[i], Rn[i], rtol=1e-9, atol=1e-12 * np.abs(Rn[i]).max())
        assert np.all(np.tril(Re[i], -1) == 0.0)
        np.testing.assert_allclose(Re[i].T @ Re[i], Cm + lam * np.eye(n), rtol=1e-12, atol=1e-12 * np.abs(Cm).max())


def test_emulated_cholesky_reports_breakdown(tk):
    n = 200
    Cm = np.eye(n)
    Cm[140, 140] = -3.0
    _, brk = tk.tk_cholesky_shifted(torch.from_numpy(Cm).cuda(), [0.5, 5.0], emulate=True)
    _, info = oracle.cholesky_shifted(Cm, 0.5)
    assert brk[0] == info == 141
    assert brk[1] == 0


def test_cholesky_reports_breakdown(tk):
    n = 70
    Cm = np.eye(n)
    Cm[40, 40] = -3.0
    R, brk = tk.tk_cholesky_shifted(torch.from_numpy(Cm).cuda(), [0.5, 5.0])
    _, info = oracle.cholesky_shifted(Cm, 0.5)
    assert brk[0] == info == 41
    assert brk[1] == 0


# ----------------------------------------------------- low-rank pieces -----
def test_jacobi_svd_and_ranks_match_oracle(tk):
    s, n = 30, 90
    Y = torch.randn(s, n, dtype=torch.float64, generator=torch.Generator().manual_seed(4)) @ \
        torch.diag(torch.logspace(0, -8, n, dtype=torch.float64))
    sig, V, sweeps = tk.tk_sketch_svd(Y.cuda())
    sig, V = sig.cpu().numpy(), V.cpu().numpy()
    so, Vo, _ = oracle.jacobi_svd(Y.numpy())
    np.testing.assert_allclose(sig, so, rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(sig, np.linalg.svd(Y.numpy(), compute_uv=False), rtol=1e-11, atol=1e-15)
    # same subspaces: |V^T Vo| = I (singular values are distinct here)
    np.testing.assert_allclose(np.abs(V.T @ Vo), np.eye(s), atol=1e-8)
    lams = [1e-12, 1e-8, 1e-4, 1.0, 10.0]
    sd, rk = tk.tk_lowrank_ranks(torch.from_numpy(sig).cuda(), lams, 2.0)
    for i, lam in enumerate(lams):
        sdo = oracle.sd_estimate(sig, lam)
        assert sd[i] == sdo  # same float64 operations in the same order
        assert rk[i] == oracle.truncation(sdo, 2.0, s)


# ------------------------------------------------------------ solves -------
def ref_over(p, lams):
    A, b = p.A.double().numpy(), p.b.numpy()
    return np.stack([oracle.ref_ridge_qr(A, b, lam, refine=3) for lam in lams])


@pytest.mark.parametrize("sketch", ["gauss", "srht"])
def test_alg1_fp64_matches_oracle(tk, sketch):
    p = problem(2000, 100, lo=1e-5, N=5, lam=(1e-8, 1.0))
    lams = p.lambdas.numpy()
    A, b = to_dev(p)
    kind = tk.TK_SKETCH_GAUSS if sketch == "gauss" else tk.TK_SKETCH_SRHT
    o = tk.opts_default(sketch=kind, s=400, seed=5, tol=1e-14)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    Xr = ref_over(p, lams)
    for i in range(len(lams)):
        assert rel(X[i], Xr[i]) < TOL_X, (i, rel(X[i], Xr[i]))
    # iteration counts agree with the oracle's Algorithm 1 on the same draws
    _, it_o, _, _ = oracle.alg1(p.A.numpy(), p.b.numpy(), lams, 1 if sketch == "gauss" else 0, 400, 5, 1e-14, 500)
    its = np.array([r["iters"] for r in res.info])
    assert np.all(np.abs(its - it_o) <= 2), (its, it_o)


def test_alg1_small_workload_4096x256(tk):
    prob, w = datagen.workload_problem("ridge_over_4096x256_f64")
    lams = prob.lambdas.numpy()
    A, b = to_dev(prob)
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=w["s"], seed=1, tol=1e-14)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    Xr = ref_over(prob, lams)
    errs = [rel(X[i], Xr[i]) for i in range(len(lams))]
    assert max(errs) < TOL_X, errs
    assert all(r["status"] == 0 for r in res.info)


def test_one_at_a_time_equals_batched(tk):
    p = problem(1500, 90, lo=1e-4, N=4)
    lams = p.lambdas.numpy()
    A, b = to_dev(p)
    o1 = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=360, seed=2)
    o2 = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=360, seed=2, schedule=tk.TK_SCHED_ONE_AT_A_TIME)
    X1 = tk.tk_solve(A, b, lams, o1).X.cpu().numpy()
    X2 = tk.tk_solve(A, b, lams, o2).X.cpu().numpy()
    Xr = ref_over(p, lams)
    for i in range(len(lams)):
        assert rel(X1[i], Xr[i]) < TOL_X and rel(X2[i], Xr[i]) < TOL_X


def test_alg2_underdetermined_matches_oracle(tk):
    m, n = 40, 3000
    p = problem(m, n, kind="exp", tau=10.0, N=4, lam=(1e-6, 1e-1))
    lams = p.lambdas.numpy()
    A, b = to_dev(p)
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=160, seed=3, tol=1e-14)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    for i, lam in enumerate(lams):
        xr = oracle.ref_ridge_under(p.A.numpy(), p.b.numpy(), lam, refine=3)
        assert rel(X[i], xr) < TOL_X, (lam, rel(X[i], xr))
    Xo, it_o, _, _ = oracle.alg2(p.A.numpy(), p.b.numpy(), lams, 0, 160, 3, 1e-14, 500)
    its = np.array([r["iters"] for r in res.info])
    assert np.all(np.abs(its - it_o) <= 2), (its, it_o)


@pytest.mark.parametrize("sketch", ["gauss", "srht"])
def test_alg4_lowrank_underdetermined_matches_oracle(tk, sketch):
    # Algorithm 4: Y = A X (m x s), U from its SVD, R^-T = l^-1/2 (I - U S U^T), min-norm LSQR
    m, n = 120, 3000
    p = problem(m, n, kind="exp", tau=8.0, N=5, lam=(1e-6, 1.0))
    lams = p.lambdas.numpy()[::-1].copy()
    A, b = to_dev(p)
    s = 64
    kind = tk.TK_SKETCH_GAUSS if sketch == "gauss" else tk.TK_SKETCH_SRHT
    o = tk.opts_default(sketch=kind, s=s, seed=6, precond=tk.TK_PRECOND_LOWRANK, alpha=2.0, tol=1e-14)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    Ad, bd = p.A.numpy(), p.b.numpy()
    for i, lam in enumerate(lams):
        xr = oracle.ref_ridge_under(Ad, bd, float(lam))
        assert rel(X[i], xr) < TOL_X, (lam, rel(X[i], xr), res.info[i])
    okind = 1 if sketch == "gauss" else 0
    Xo, it_o, st_o, si_o, sig_o = oracle.alg4(Ad, bd, lams, okind, s, 2.0, 6, 1e-14, 500)
    ranks = np.array([r["rank"] for r in res.info])
    assert np.all(ranks == si_o), (ranks, si_o)
    its = np.array([r["iters"] for r in res.info])
    assert np.all(np.abs(its - it_o) <= 2), (its, it_o)


def test_alg3_lowrank_matches_oracle(tk):
    m, n = 3000, 120
    p = problem(m, n, kind="exp", tau=8.0, N=5, lam=(1e-6, 1.0))
    lams = p.lambdas.numpy()[::-1].copy()
    A, b = to_dev(p)
    s = 60
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=s, seed=6, precond=tk.TK_PRECOND_LOWRANK, alpha=2.0, tol=1e-14)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    Xr = ref_over(p, lams)
    for i in range(len(lams)):
        assert rel(X[i], Xr[i]) < TOL_X, (lams[i], rel(X[i], Xr[i]))
    Xo, it_o, st_o, si_o, sig_o = oracle.alg3(p.A.numpy(), p.b.numpy(), lams, 1, s, 2.0, 6, 1e-14, 500)
    ranks = np.array([r["rank"] for r in res.info])
    # ranks are integers decided in float64 from each side's own sigma(Y); equal unless an sd
    # estimate lies within rounding of an integer
    assert np.all(np.abs(ranks - si_o) <= 0), (ranks, si_o)


def test_mixed_precision_reaches_fp64_accuracy(tk):
    p = problem(4096, 256, lo=1e-5, N=6, lam=(1e-5, 1.0), dtype=torch.float32)
    lams = p.lambdas.numpy()
    A, b = to_dev(p)
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=512, seed=9, precision=tk.TK_PREC_MIXED)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    Xr = ref_over(p, lams)
    for i in range(len(lams)):
        assert rel(X[i], Xr[i]) < TOL_X, (lams[i], rel(X[i], Xr[i]), res.info[i])
    assert all(r["refine_steps"] >= 2 for r in res.info)


def test_mixed_on_float64_input(tk):
    p = problem(3000, 128, lo=1e-4, N=3, lam=(1e-4, 1.0))
    lams = p.lambdas.numpy()
    A, b = to_dev(p)
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=512, seed=9, precision=tk.TK_PREC_MIXED)
    X = tk.tk_solve(A, b, lams, o).X.cpu().numpy()
    Xr = ref_over(p, lams)
    for i in range(len(lams)):
        assert rel(X[i], Xr[i]) < TOL_X


def test_batched_uneven_problems(tk):
    probs = datagen.uneven_batch(5, m_range=(300, 2500), n_range=(8, 120), N=3, dtype=torch.float64)
    pairs = [(p.A.cuda(), p.b.cuda()) for p in probs]
    lams = np.stack([p.lambdas.numpy() for p in probs])
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=0, seed=4)
    Xs, infos, st = tk.tk_solve_batched(pairs, lams, o)
    for p, X, lam in zip(probs, Xs, lams):
        Xr = ref_over(p, lam)
        Xc = X.cpu().numpy()
        for i in range(len(lam)):
            assert rel(Xc[i], Xr[i]) < TOL_X


def test_edge_single_column_and_single_lambda(tk):
    p = problem(257, 1, N=1, lam=(0.5, 0.5))
    A, b = to_dev(p)
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=4, seed=1)
    X = tk.tk_solve(A, b, [0.5], o).X.cpu().numpy()
    a = p.A.numpy()[:, 0]
    x_exact = a @ p.b.numpy() / (a @ a + 0.5)
    assert abs(X[0, 0] - x_exact) <= 1e-12 * abs(x_exact)


def sd_of_spectrum(sig, lam):
    return float(np.sum(1.0 / (1.0 + lam / (sig * sig))))


@pytest.mark.parametrize("group", [1, 0])
def test_uneven_batch_mixed_cholesky_and_lowrank(tk, group):
    # the 256-problem workload's structure at test size: float32 data, mixed precision,
    # half the problems with sigma_i = exp(-i/50) solved with the sd-sized low-rank form;
    # group = 1: all problems advance in one grouped LSQR, 0: each problem on its own
    probs = datagen.uneven_batch(10, m_range=(1500, 4000), n_range=(64, 200), N=4, dtype=torch.float32)
    pairs, opts = [], []
    for p in probs:
        pairs.append((p.A.cuda(), p.b.cuda()))
        n = p.A.shape[1]
        if p.meta["lowrank"]:
            s = min(n, 2 * math.ceil(sd_of_spectrum(p.sigma.numpy(), float(p.lambdas.min()))))
            opts.append(tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=s, seed=3, precond=tk.TK_PRECOND_LOWRANK,
                                        alpha=2.0, precision=tk.TK_PREC_MIXED, group=group))
        else:
            opts.append(tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=min(4 * n, p.A.shape[0]), seed=3,
                                        precision=tk.TK_PREC_MIXED, group=group))
    lams = np.stack([p.lambdas.numpy() for p in probs])
    Xs, infos, st = tk.tk_solve_batched(pairs, lams, opts)
    assert st == tk.TK_OK, infos
    for p, X, lam, inf in zip(probs, Xs, lams, infos):
        Xr = ref_over(p, lam)
        Xc = X.cpu().numpy()
        for i in range(len(lam)):
            assert rel(Xc[i], Xr[i]) < TOL_X, (p.meta, lam[i], rel(Xc[i], Xr[i]), inf[i])
            assert 1 <= inf[i]["refine_steps"] <= 8 and inf[i]["iters"] > 0
        if p.meta["lowrank"]:
            assert all(0 < q["rank"] <= p.A.shape[1] for q in inf)


def test_grouped_batch_float64_and_float32_inputs(tk):
    # grouped mixed solve over problems whose A is float64 (float32 copy for the LSQR,
    # float64 residual passes) and float32, Cholesky preconditioner, SRHT and Gaussian
    # sketches, ragged m and n (no 16-byte multiple), 12 lambda each
    shapes = [(3001, 131), (2048, 256), (5003, 77), (1777, 300), (4096, 64), (2500, 199)]
    pairs, opts, refs, lam_rows = [], [], [], []
    for i, (m, n) in enumerate(shapes):
        dt = torch.float64 if i % 2 == 0 else torch.float32
        p = datagen.make_ridge_problem(m, n, datagen.spectrum("log", n, hi=1.0, lo=1e-5),
                                       datagen.log_lambdas(12, 1e-6, 1.0), seed=900 + i, dtype=dt)
        pairs.append((p.A.cuda(), p.b.cuda()))
        sk = tk.TK_SKETCH_SRHT if i % 3 == 0 else tk.TK_SKETCH_GAUSS
        opts.append(tk.opts_default(sketch=sk, s=min(4 * n, m), seed=5, precision=tk.TK_PREC_MIXED))
        lam_rows.append(p.lambdas.numpy())
        refs.append(ref_over(p, p.lambdas.numpy()))
    lams = np.stack(lam_rows)
    Xs, infos, st = tk.tk_solve_batched(pairs, lams, opts)
    assert st == tk.TK_OK, infos
    for k in range(len(shapes)):
        Xc = Xs[k].cpu().numpy()
        for i in range(lams.shape[1]):
            assert rel(Xc[i], refs[k][i]) < TOL_X, (shapes[k], lams[k, i], rel(Xc[i], refs[k][i]), infos[k][i])


def test_mixed_gaussian_float32_scaled_workload(tk):
    # 2^20 x 4096 float32 workload structure at 2^16 x 1024: Gaussian s = 2n, 16 lambda in 1e-5..1
    prob, w = datagen.workload_problem("ridge_over_1048576x4096_f32", m=1 << 16, n=1024, N=16, keep_factors=True)
    lams = prob.lambdas.numpy()
    A, b = to_dev(prob)
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=2 * 1024, seed=1, precision=tk.TK_PREC_MIXED)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    Ad, bd = prob.A.double().numpy(), prob.b.numpy()
    U, V, sig = prob.U.double().numpy(), prob.V.double().numpy(), prob.sigma.numpy()
    for i in (0, 5, 10, 15):
        lam = float(lams[i])
        # reference: closed form from the generator's factors, refined against the stored
        # (float32, exactly widened) A in double-double
        x0 = V @ ((sig / (sig * sig + lam)) * (U.T @ bd))
        xr = oracle.ref_ridge_refine(Ad, bd, lam, V, sig, x0, steps=3)
        assert rel(X[i], xr) < TOL_X, (lams[i], rel(X[i], xr), res.info[i])
    assert all(q["status"] == 0 for q in res.info)


@pytest.mark.parametrize("m,n,s", [(1000, 300, 256), (4096, 256, 1024), (777, 513, 130), (64, 8, 16)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_tensor_core_gauss_sketch(tk, m, n, s, dtype):
    # the mixed form's sketch: G and A rounded to BF16, tcgen05 products with FP32
    # accumulation.  Each term carries two BF16 roundings (relative 2^-8 each) with
    # random signs, so ||Y - Y_oracle||_F / ||Y_oracle||_F is a few 1e-3.
    A = torch.randn(m, n, dtype=torch.float64, generator=torch.Generator().manual_seed(m * 7 + n)).to(dtype)
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=s, seed=8, precision=tk.TK_PREC_MIXED)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    Yo = oracle.gauss_over(A.double().numpy(), 8, s)
    err = np.linalg.norm(Y - Yo) / np.linalg.norm(Yo)
    assert err < 2e-2, err
    # the sketch is still an embedding: columns keep their norms to within sampling error
    assert np.all(np.isfinite(Y))


@pytest.mark.parametrize("m,n,N", [(4096, 256, 6), (3004, 164, 40), (12000, 384, 64)])
def test_mixed_tensor_core_lsqr_products(tk, m, n, N):
    # the two products with A of every LSQR step on tcgen05 (kind::tf32, 3-term split),
    # then float64 refinement: x must reach the same 1e-10 as the SIMT float32 path
    p = problem(m, n, lo=1e-5, N=N, lam=(1e-5, 1.0), dtype=torch.float32)
    lams = p.lambdas.numpy()
    A, b = to_dev(p)
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=min(4 * n, m), seed=9, precision=tk.TK_PREC_MIXED, lsqr_tc=1)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    o0 = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=min(4 * n, m), seed=9, precision=tk.TK_PREC_MIXED)
    res0 = tk.tk_solve(A, b, lams, o0)
    Ad, bd = p.A.double().numpy(), p.b.numpy()
    for i in sorted({0, N // 2, N - 1}):
        xr = oracle.ref_ridge_qr(Ad, bd, float(lams[i]), refine=3)
        assert rel(X[i], xr) < TOL_X, (lams[i], rel(X[i], xr), res.info[i])
    # same inner accuracy as the float32 SIMT products: comparable iteration counts
    it_tc = sum(q["iters"] for q in res.info)
    it_simt = sum(q["iters"] for q in res0.info)
    assert it_tc <= 1.3 * it_simt + 5, (it_tc, it_simt)


@pytest.mark.parametrize("m,n,N,dtype", [(32768, 640, 8, torch.float64), (40000, 500, 33, torch.float32)])
def test_mixed_sliced_lsqr_products(tk, m, n, N, dtype):
    # the two products with A of every LSQR step from the first 4 exact digits of the slices of A
    # (lsqr_tc = 2; m n > 2^24 so the sliced path is taken), then the float64 refinement: x must
    # reach the same 1e-10 as with the SIMT float32 products, with comparable iteration counts
    p = problem(m, n, lo=1e-5, N=N, lam=(1e-6, 1.0), dtype=dtype)
    lams = p.lambdas.numpy()
    A, b = to_dev(p)
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=4 * n, seed=9, precision=tk.TK_PREC_MIXED, lsqr_tc=2)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    o0 = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=4 * n, seed=9, precision=tk.TK_PREC_MIXED, lsqr_tc=0)
    res0 = tk.tk_solve(A, b, lams, o0)
    Ad, bd = p.A.double().numpy(), p.b.numpy()
    for i in sorted({0, N // 2, N - 1}):
        xr = oracle.ref_ridge_qr(Ad, bd, float(lams[i]), refine=3)
        assert rel(X[i], xr) < TOL_X, (lams[i], rel(X[i], xr), res.info[i])
        assert res.info[i]["status"] == 0
    it_oz = sum(q["iters"] for q in res.info)
    it_simt = sum(q["iters"] for q in res0.info)
    assert it_oz <= 1.2 * it_simt + 5, (it_oz, it_simt)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotuned_solve_matches_untuned(tk, precision):
    # the tuner only changes tile shapes and split counts: the solution stays the same
    p = problem(3000, 192, lo=1e-5, N=6, lam=(1e-6, 1.0))
    lams = p.lambdas.numpy()
    A, b = to_dev(p)
    prec = tk.TK_PREC_FP64 if precision == "fp64" else tk.TK_PREC_MIXED
    o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=768, seed=2, precision=prec, tol=1e-14)
    tk.tk_autotune_clear()
    X0 = tk.tk_solve(A, b, lams, o).X.cpu().numpy()
    try:
        entries = tk.tk_autotune(A, b, len(lams), o)
        assert entries > 0
        res = tk.tk_solve(A, b, lams, o)
    finally:
        tk.tk_autotune_clear()
    X1 = res.X.cpu().numpy()
    Xr = ref_over(p, lams)
    for i in range(len(lams)):
        assert rel(X1[i], Xr[i]) < TOL_X, (lams[i], rel(X1[i], Xr[i]))
        assert rel(X1[i], X0[i]) < 1e-11


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_emulated_residual_has_float64_accuracy(tk, dtype):
    # R = b - X A^T on the BF16 tensor cores (8 exact 7-bit slices per value) against an
    # extended-precision reference: its error must be that of the float64 FMA residual
    gen = torch.Generator().manual_seed(17)
    m, n, M = 2999, 777, 6  # ragged in every dimension (n not a multiple of 8 or of 32)
    A = torch.randn(m, n, generator=gen, dtype=torch.float64)
    A *= torch.logspace(0, -6, n, dtype=torch.float64)  # wide dynamic range along each row
    A = A.to(dtype)
    X = torch.randn(M, n, generator=gen, dtype=torch.float64) * torch.logspace(2, -3, M, dtype=torch.float64)[:, None]
    b = (X[0] @ A.double().T) + 1e-3 * torch.randn(m, generator=gen, dtype=torch.float64)  # nearly consistent
    Ad, bd, Xd = A.cuda(), b.cuda(), X.cuda()
    Re = tk.tk_residual(Ad, bd, Xd, True).cpu().numpy()
    Rn = tk.tk_residual(Ad, bd, Xd, False).cpu().numpy()
    Al = A.double().numpy().astype(np.longdouble)
    Rref = b.numpy().astype(np.longdouble)[None, :] - X.numpy().astype(np.longdouble) @ Al.T
    scale = np.abs(b.numpy())[None, :] + np.abs(X.numpy()) @ np.abs(A.double().numpy()).T
    err_e = float(np.max(np.abs((Re - Rref).astype(np.float64)) / scale))
    err_n = float(np.max(np.abs((Rn - Rref).astype(np.float64)) / scale))
    assert err_e < 8 * 2.0 ** -53 * math.sqrt(n), (err_e, err_n)
    assert err_e <= 4 * err_n + 1e-16, (err_e, err_n)


# the row exponents and row slices of A across widths (64 to 4100 columns: one to several 512-value
# column chunks of the slicing grid, ragged against the 64-value padding), rows of very different
# scale, and A as a strided view (an odd leading dimension, a base not aligned to a pair)
@pytest.mark.parametrize("m,n,dtype,offset", [(1500, 4096, torch.float64, 0), (700, 4100, torch.float64, 0),
                                              (900, 1025, torch.float32, 1), (333, 2000, torch.float64, 1),
                                              (2000, 64, torch.float32, 0), (50, 511, torch.float64, 0)])
def test_emulated_residual_row_slicing_shapes(tk, m, n, dtype, offset):
    gen = torch.Generator().manual_seed(m + n)
    full = torch.randn(m, n + 2 * offset + (1 if offset else 0), generator=gen, dtype=torch.float64)
    full *= torch.pow(2.0, torch.randint(-30, 31, (m, 1), generator=gen).double())  # row scales 2^-30 .. 2^30
    full = full.to(dtype).cuda()
    A = full[:, offset:offset + n]  # a strided view when offset = 1 (leading dimension n + 3)
    X = torch.randn(4, n, generator=gen, dtype=torch.float64)
    b = torch.randn(m, generator=gen, dtype=torch.float64)
    Re = tk.tk_residual(A, b.cuda(), X.cuda(), True).cpu().numpy()
    Ah = A.cpu().double().numpy()
    Rref = b.numpy().astype(np.longdouble)[None, :] - X.numpy().astype(np.longdouble) @ Ah.astype(np.longdouble).T
    scale = np.abs(b.numpy())[None, :] + np.abs(X.numpy()) @ np.abs(Ah).T
    err = float(np.max(np.abs((Re - Rref).astype(np.float64)) / scale))
    assert err < 8 * 2.0 ** -53 * math.sqrt(n), err


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_emulated_normal_product_has_float64_accuracy(tk, dtype):
    # G = R A (the rows A^T r_l) on the BF16 tensor cores: every column of G within the
    # float64 error of its own column, however different the scales of A's columns
    gen = torch.Generator().manual_seed(19)
    m, n, M = 4133, 333, 5  # m spans several 128-row chunks and a ragged split; n ragged
    A = torch.randn(m, n, generator=gen, dtype=torch.float64)
    A *= torch.logspace(0, -8, n, dtype=torch.float64)  # column scales over 8 decades
    A[:, 7] = 0.0  # a zero column
    A = A.to(dtype)
    X = torch.randn(M, n, generator=gen, dtype=torch.float64)
    b = torch.randn(m, generator=gen, dtype=torch.float64) * torch.logspace(0, -3, m, dtype=torch.float64)
    Ad, bd, Xd = A.cuda(), b.cuda(), X.cuda()
    Re, Ge = tk.tk_residual(Ad, bd, Xd, True, with_g=True)
    Rn, Gn = tk.tk_residual(Ad, bd, Xd, False, with_g=True)
    Al = A.double().numpy().astype(np.longdouble)
    for R, G in ((Re, Ge), (Rn, Gn)):
        assert G.shape == (M, n)
    Rl = Re.cpu().numpy().astype(np.longdouble)  # the product of the residuals actually formed
    Gref = Rl @ Al
    scale = np.abs(Re.cpu().numpy()) @ np.abs(A.double().numpy())
    scale[:, 7] = 1.0
    err_e = np.max(np.abs((Ge.cpu().numpy() - Gref).astype(np.float64)) / scale, axis=0)
    assert np.all(Ge.cpu().numpy()[:, 7] == 0.0)
    assert float(err_e.max()) < 8 * 2.0 ** -53 * math.sqrt(m), float(err_e.max())
    Rl = Rn.cpu().numpy().astype(np.longdouble)
    scale = np.abs(Rn.cpu().numpy()) @ np.abs(A.double().numpy())
    scale[:, 7] = 1.0
    err_n = np.max(np.abs((Gn.cpu().numpy() - Rl @ Al).astype(np.float64)) / scale, axis=0)
    assert float(err_n.max()) < 8 * 2.0 ** -53 * math.sqrt(m), float(err_n.max())
    # the columns of smallest scale are as accurate as the largest
    assert float(err_e[-20:].max()) <= 4 * float(err_n.max()) + 1e-16


def test_emulated_products_propagate_non_finite(tk):
    # an inf or NaN in the input reaches every output that uses it (the digits cannot hold it, so
    # the rows and columns that contain one are marked): R = b - X A^T, G = R A and the Gram matrix
    gen = torch.Generator().manual_seed(23)
    A = torch.randn(700, 150, generator=gen, dtype=torch.float64)
    A[5, 3] = float("inf")
    A[7, 2] = float("nan")
    b = torch.randn(700, generator=gen, dtype=torch.float64)
    X = torch.randn(3, 150, generator=gen, dtype=torch.float64)
    R, G = tk.tk_residual(A.cuda(), b.cuda(), X.cuda(), True, with_g=True)
    R, G = R.cpu().numpy(), G.cpu().numpy()
    bad = np.zeros(700, dtype=bool)
    bad[[5, 7]] = True
    assert not np.isfinite(R[:, bad]).any()
    assert np.isfinite(R[:, ~bad]).all()
    assert not np.isfinite(G).any()  # every residual row holds a non-finite entry
    Y = torch.randn(300, 40, generator=gen, dtype=torch.float64)
    Y[11, 4] = float("nan")
    Cm = tk.tk_gram(Y.cuda(), True, emulate=True).cpu().numpy()
    iu = np.triu_indices(40)
    touched = (iu[0] == 4) | (iu[1] == 4)
    assert not np.isfinite(Cm[iu][touched]).any()
    assert np.isfinite(Cm[iu][~touched]).all()


@pytest.mark.parametrize("emulate", [1, 0])
def test_mixed_with_emulated_residual_matches_reference(tk, emulate):
    # the mixed form with both float64 passes of its refinement on the tensor cores
    # (r = b - A x and A^T r; the default) or on the float64 pipe reaches 1e-10
    p = problem(4000, 192, lo=1e-6, N=8, lam=(1e-8, 1.0))
    lams = p.lambdas.numpy()
    A, b = to_dev(p)
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=768, seed=3, precision=tk.TK_PREC_MIXED, emulate_fp64=emulate)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    Xr = ref_over(p, lams)
    for i in range(len(lams)):
        assert rel(X[i], Xr[i]) < TOL_X, (lams[i], rel(X[i], Xr[i]), res.info[i])
        assert res.info[i]["status"] == 0
