"""Pins for the CPU oracle, against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: each check uses a closed form, a
library routine on a case that reduces to it, brute force on a tiny input, an
exact rational computation, or an inequality the paper proves.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

import torch

from paper_2203_07329_gb300 import datagen

RNG = np.random.default_rng(12345)


def small_problem(m, n, sig_lo=1e-3, seed=7, noise=1e-3):
    sig = datagen.spectrum("log", min(m, n), hi=1.0, lo=sig_lo)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(4, 1e-4, 1.0), seed=seed, noise=noise,
                                   keep_factors=True)
    return p.A.numpy(), p.b.numpy(), p


# ------------------------------------------------------------ RNG / draws --
def _kat_rows():
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = []
    with open(here) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                rows.append([int(x, 16) for x in ln.split()])
    return rows


def test_philox_known_answer_vectors(orc):
    # Salmon et al. (SC'11), Random123 known-answer vectors for philox4x32 with 10 rounds: a wrong
    # multiplier, Weyl constant, word order or round count changes every output word
    rows = _kat_rows()
    assert len(rows) == 3
    for w in rows:
        out = orc.philox4x32_10(w[0:4], w[4:6])
        assert [int(x) for x in out] == w[6:10], [hex(int(x)) for x in out]


def test_philox_words_are_balanced_and_counter_sensitive(orc):
    # bit balance over many counters: every bit of every word ~ 1/2
    words = np.array([orc.philox4x32_10([i, 0, 0, 0], [1, 0]) for i in range(4000)], dtype=np.uint64)
    bits = np.stack([(words >> k) & 1 for k in range(32)], axis=-1).astype(np.float64)
    frac = bits.mean(axis=0)
    assert np.all(np.abs(frac - 0.5) < 0.04)
    # distinct counters, keys and streams give distinct blocks
    a = orc.philox4x32_10([5, 0, 0, 0], [1, 0])
    assert not np.array_equal(a, orc.philox4x32_10([6, 0, 0, 0], [1, 0]))
    assert not np.array_equal(a, orc.philox4x32_10([5, 0, 1, 0], [1, 0]))
    assert not np.array_equal(a, orc.philox4x32_10([5, 0, 0, 0], [2, 0]))
    assert not np.array_equal(a, orc.philox4x32_10([5, 0, 0, 0], [1, 1]))


def test_signs_are_rademacher(orc):
    d = orc.draw_signs(3, 1 << 16).astype(np.float64)
    assert set(np.unique(d)) <= {-1.0, 1.0}
    assert abs(d.mean()) < 5.0 / math.sqrt(d.size)
    # lag-1 correlation ~ 0
    assert abs(np.mean(d[1:] * d[:-1])) < 5.0 / math.sqrt(d.size)


def test_row_subset_is_uniform_without_replacement(orc):
    mp, s, trials = 64, 16, 600
    counts = np.zeros(mp)
    for seed in range(trials):
        r = orc.draw_rows(seed, mp, s)
        assert r.shape == (s,)
        assert np.all(np.diff(r) > 0)  # ascending and distinct
        assert r[0] >= 0 and r[-1] < mp
        counts[r] += 1
    expected = trials * s / mp
    chi2 = np.sum((counts - expected) ** 2 / expected)
    # 63 degrees of freedom: mean 63, sd ~ 11.2; allow 5 sd
    assert chi2 < 63 + 5 * 11.3


def test_row_subset_edge_cases(orc):
    assert orc.draw_rows(1, 32, 0).shape == (0,)
    assert np.array_equal(orc.draw_rows(1, 32, 32), np.arange(32))
    with pytest.raises(ValueError):
        orc.draw_rows(1, 32, 33)


def test_row_subset_is_the_s_smallest_keys(orc):
    # brute force: sort all keys explicitly in Python
    mp, s = 200, 37
    keys = orc.draw_keys(9, mp)
    order = sorted(range(mp), key=lambda i: (int(keys[i]), i))[:s]
    assert np.array_equal(orc.draw_rows(9, mp, s), np.array(sorted(order)))


def test_gaussian_embedding_moments(orc):
    s, L = 2000, 6
    G = orc.draw_gauss(11, s, L)
    assert abs(G.mean()) < 5 / math.sqrt(G.size) / math.sqrt(s)
    assert abs(G.var() * s - 1.0) < 0.05
    # E[G^T G] = I  (scaling N(0, 1/s) is what makes the partly exact sketch consistent with lambda)
    assert np.linalg.norm(G.T @ G - np.eye(L), 2) < 0.15
    z = G.ravel() * math.sqrt(s)
    kurt = np.mean(z ** 4) / np.mean(z ** 2) ** 2
    assert abs(kurt - 3.0) < 0.3


# ----------------------------------------------------------------- FWHT ----
@pytest.mark.parametrize("L", [1, 2, 8, 64, 256])
def test_fwht_matches_sylvester_hadamard(orc, L):
    z = RNG.standard_normal(L)
    H = sla.hadamard(L).astype(np.float64)  # Sylvester order
    np.testing.assert_allclose(orc.fwht(z), H @ z, rtol=1e-13, atol=1e-13)


def explicit_srht_over(orc, m, seed, s):
    mp = orc.next_pow2(m)
    d = orc.draw_signs(seed, mp).astype(np.float64)
    rows = orc.draw_rows(seed, mp, s)
    H = sla.hadamard(mp).astype(np.float64)
    S = np.zeros((s, mp))
    S[np.arange(s), rows] = 1.0
    X = math.sqrt(mp / s) * S @ (H / math.sqrt(mp)) @ np.diag(d)
    return X[:, :m]  # the zero padding of [A; 0] drops the extra columns


@pytest.mark.parametrize("m,n,s", [(50, 7, 20), (64, 5, 64), (33, 3, 9)])
def test_srht_over_equals_explicit_embedding(orc, m, n, s):
    A = RNG.standard_normal((m, n))
    X = explicit_srht_over(orc, m, 5, s)
    np.testing.assert_allclose(orc.srht_over(A, 5, s), X @ A, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m,n,s", [(5, 50, 20), (3, 64, 16)])
def test_srht_under_equals_explicit_embedding(orc, m, n, s):
    A = RNG.standard_normal((m, n))
    X = explicit_srht_over(orc, n, 6, s).T  # n x s
    np.testing.assert_allclose(orc.srht_under(A, 6, s), A @ X, rtol=1e-12, atol=1e-12)


def test_srht_is_an_isometry_when_s_equals_mp(orc):
    # S = I: X = H D / sqrt(mp) is orthogonal, so ||XA||_F = ||A||_F
    A = RNG.standard_normal((64, 4))
    Y = orc.srht_over(A, 2, 64)
    np.testing.assert_allclose(np.linalg.norm(Y), np.linalg.norm(A), rtol=1e-13)


def test_gauss_sketches_equal_matrix_products(orc):
    A = RNG.standard_normal((40, 6))
    G = orc.draw_gauss(4, 12, 40)
    np.testing.assert_allclose(orc.gauss_over(A, 4, 12), G @ A, rtol=1e-12, atol=1e-13)
    B = RNG.standard_normal((5, 30))
    G2 = orc.draw_gauss(4, 9, 30)
    np.testing.assert_allclose(orc.gauss_under(B, 4, 9), B @ G2.T, rtol=1e-12, atol=1e-13)


# ------------------------------------------------------ Gram / Cholesky ----
def test_gram_and_cholesky_against_lapack(orc):
    Y = RNG.standard_normal((30, 9))
    Cm = orc.gram_tn(Y)
    np.testing.assert_allclose(Cm, Y.T @ Y, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(orc.gram_nt(Y.T), Y.T @ Y, rtol=1e-13, atol=1e-13)
    lam = 0.3
    R, info = orc.cholesky_shifted(Cm, lam)
    assert info == 0
    assert np.allclose(np.tril(R, -1), 0.0)
    np.testing.assert_allclose(R, np.linalg.cholesky(Cm + lam * np.eye(9)).T, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(R.T @ R, Cm + lam * np.eye(9), rtol=1e-13, atol=1e-13)


def test_cholesky_reports_breakdown_row(orc):
    Cm = np.diag([4.0, 1.0, -3.0, 2.0])
    R, info = orc.cholesky_shifted(Cm, 0.5)
    assert info == 3  # pivot of row index 2 is -2.5


def test_triangular_solves(orc):
    R = np.triu(RNG.standard_normal((8, 8))) + 4 * np.eye(8)
    v = RNG.standard_normal(8)
    np.testing.assert_allclose(orc.trsv_upper(R, v), np.linalg.solve(R, v), rtol=1e-12)
    np.testing.assert_allclose(orc.trsv_upper_t(R, v), np.linalg.solve(R.T, v), rtol=1e-12)


def test_partly_exact_cholesky_equals_qr_of_augmented_sketch(orc):
    # R_BP2 from QR([XA; sqrt(l) I]) equals the Algorithm 1 Cholesky factor up to row signs
    A = RNG.standard_normal((80, 6))
    Y = orc.gauss_over(A, 3, 24)
    lam = 0.05
    R, _ = orc.cholesky_shifted(orc.gram_tn(Y), lam)
    Rq = np.linalg.qr(np.vstack([Y, math.sqrt(lam) * np.eye(6)]), mode="r")
    Rq = np.sign(np.diag(Rq))[:, None] * Rq
    np.testing.assert_allclose(R, Rq, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------- double-double / ref --
def test_error_free_transformations_are_exact(orc):
    for _ in range(200):
        a, b = RNG.standard_normal() * 10.0 ** RNG.integers(-5, 5), RNG.standard_normal()
        p, e = orc.two_prod(a, b)
        assert Fraction(p) + Fraction(e) == Fraction(a) * Fraction(b)
        s, f = orc.two_sum(a, b)
        assert Fraction(s) + Fraction(f) == Fraction(a) + Fraction(b)


def test_dd_normal_residual_against_exact_rationals(orc):
    m, n = 7, 4
    A = RNG.standard_normal((m, n))
    b = RNG.standard_normal(m)
    x = RNG.standard_normal(n)
    lam = 0.37
    g, r = orc.ridge_residual_dd(A, b, lam, x)
    Af = [[Fraction(v) for v in row] for row in A]
    rf = [Fraction(b[i]) - sum(Af[i][j] * Fraction(x[j]) for j in range(n)) for i in range(m)]
    gf = [sum(Af[i][j] * rf[i] for i in range(m)) - Fraction(lam) * Fraction(x[j]) for j in range(n)]
    for j in range(n):
        assert abs(float(Fraction(g[j]) - gf[j])) <= 1e-30 + 4e-16 * abs(float(gf[j]))


def test_reference_qr_matches_closed_form_and_lstsq(orc):
    A, b, p = small_problem(60, 8, sig_lo=1e-2)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    for lam in [1e-6, 1e-3, 1.0]:
        x_ref = orc.ref_ridge_qr(A, b, lam)
        x_cf = Vt.T @ ((s / (s * s + lam)) * (U.T @ b))
        np.testing.assert_allclose(x_ref, x_cf, rtol=1e-10)
        B = np.vstack([A, math.sqrt(lam) * np.eye(8)])
        x_ls = np.linalg.lstsq(B, np.concatenate([b, np.zeros(8)]), rcond=None)[0]
        np.testing.assert_allclose(x_ref, x_ls, rtol=1e-9)


def test_reference_refinement_converges_from_generator_factors(orc):
    A, b, p = small_problem(200, 16, sig_lo=1e-4)
    U, sig, V = p.U.numpy(), p.sigma.numpy(), p.V.numpy()
    lam = 1e-6
    x0 = V @ ((sig / (sig * sig + lam)) * (U.T @ b))
    x = orc.ref_ridge_refine(A, b, lam, V, sig, x0, steps=3)
    x_qr = orc.ref_ridge_qr(A, b, lam, refine=3)
    assert np.linalg.norm(x - x_qr) <= 1e-13 * np.linalg.norm(x_qr)


# ---------------------------------------------------------------- LSQR -----
def test_plain_lsqr_matches_lstsq(orc):
    A = RNG.standard_normal((50, 6))
    b = RNG.standard_normal(50)
    x, it, ist = orc.lsqr_plain(A, b, 1e-14, 200)
    np.testing.assert_allclose(x, np.linalg.lstsq(A, b, rcond=None)[0], rtol=1e-10)
    assert ist in (1, 2)


def test_plain_lsqr_consistent_system_stops_on_test1(orc):
    A = RNG.standard_normal((20, 20)) + 6 * np.eye(20)
    xs = RNG.standard_normal(20)
    x, it, ist = orc.lsqr_plain(A, A @ xs, 1e-13, 200)
    np.testing.assert_allclose(x, xs, rtol=1e-9)
    assert ist == 1


def test_zero_rhs_gives_zero(orc):
    A = RNG.standard_normal((10, 3))
    x, it, ist = orc.lsqr_plain(A, np.zeros(10), 1e-10, 20)
    assert it == 0 and np.all(x == 0)


# ------------------------------------------------------- Algorithms 1-3 ----
def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("kind", [0, 1])
def test_alg1_reaches_the_unique_ridge_solution(orc, kind):
    A, b, p = small_problem(300, 24, sig_lo=1e-4)
    lams = np.array([1e-6, 1e-4, 1e-2, 1.0])
    X, it, st, rc = orc.alg1(A, b, lams, kind, 96, 1, 1e-14, 200)
    assert rc == 0
    for i, lam in enumerate(lams):
        assert rel(X[:, i], orc.ref_ridge_qr(A, b, lam)) < 1e-10, (kind, lam)
    assert np.all(it < 80)


def test_alg1_closed_form_on_known_svd(orc):
    # x_l = V diag(sigma/(sigma^2 + l)) U^T b for A built from a known SVD
    A, b, p = small_problem(512, 32, sig_lo=1e-3)
    U, sig, V = p.U.numpy(), p.sigma.numpy(), p.V.numpy()
    lams = np.array([1e-5, 1e-2])
    X, it, st, rc = orc.alg1(A, b, lams, 1, 128, 2, 1e-14, 200)
    for i, lam in enumerate(lams):
        x_cf = V @ ((sig / (sig * sig + lam)) * (U.T @ b))
        # tolerance: A is stored rounded, so the closed form is exact up to ~u*kappa_B^2
        assert rel(X[:, i], x_cf) < 1e-9


def test_alg2_equals_overdetermined_solution(orc):
    # the top block of the min-norm solution of (1.4) is the ridge solution of (1.2)
    m, n = 12, 90
    sig = datagen.spectrum("exp", m, tau=6.0)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(3, 1e-4, 1e-1), seed=3)
    A, b = p.A.numpy(), p.b.numpy()
    lams = p.lambdas.numpy()
    X, it, st, rc = orc.alg2(A, b, lams, 0, 48, 4, 1e-14, 300)
    assert rc == 0
    for i, lam in enumerate(lams):
        x_normal = np.linalg.solve(A.T @ A + lam * np.eye(n), A.T @ b)
        x_dual = A.T @ np.linalg.solve(A @ A.T + lam * np.eye(m), b)
        assert rel(X[:, i], x_dual) < 1e-10
        assert rel(x_normal, x_dual) < 1e-8


def test_alg3_lowrank_reaches_ridge_solution(orc):
    m, n = 400, 60
    sig = datagen.spectrum("exp", n, tau=5.0)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(4, 1e-6, 1.0), seed=9)
    A, b = p.A.numpy(), p.b.numpy()
    lams = p.lambdas.numpy()[::-1].copy()  # lambda_1 >= ... >= lambda_N
    s = 40
    X, it, st, si, sigY = orc.alg3(A, b, lams, 1, s, 2.0, 5, 1e-14, 300)
    for i, lam in enumerate(lams):
        assert rel(X[:, i], orc.ref_ridge_qr(A, b, lam)) < 1e-9, lam
    # truncation ranks grow as lambda shrinks, and never exceed s
    assert np.all(np.diff(si) >= 0) and si.max() <= s


def test_alg4_lowrank_underdetermined_reaches_ridge_solution(orc):
    # Algorithm 4: the top block of the min-norm solution of the low-rank-preconditioned
    # underdetermined system is the dual ridge solution A^T (A A^T + l I)^-1 b
    m, n = 60, 400
    sig = datagen.spectrum("exp", m, tau=5.0)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(4, 1e-6, 1.0), seed=19)
    A, b = p.A.numpy(), p.b.numpy()
    lams = p.lambdas.numpy()[::-1].copy()
    s = 40
    for kind in (0, 1):
        X, it, st, si, sigY = orc.alg4(A, b, lams, kind, s, 2.0, 8, 1e-14, 400)
        for i, lam in enumerate(lams):
            x_dual = A.T @ np.linalg.solve(A @ A.T + lam * np.eye(m), b)
            assert rel(X[:, i], x_dual) < 1e-9, (kind, lam, rel(X[:, i], x_dual))
        assert np.all(np.diff(si) >= 0) and si.max() <= s
        # sigma(Y) of Y = A X equals LAPACK's on the same sketch
        Y = orc.sketch_under(A, kind, 8, s)
        np.testing.assert_allclose(sigY, np.linalg.svd(Y, compute_uv=False), rtol=1e-11, atol=1e-14)


def test_lemma_3_3_and_theorem_3_4_condition_bound(orc):
    # Lemma 3.3: ||V_1||_F^2 = sd_l(A), V_1 the first n rows of the right singular vectors of
    # D = [A sqrt(l) I_m]; Theorem 3.4: kappa(R^-T D) <= sqrt((1+eps)/(1-eps)) with
    # eps = ||V_1^T X X^T V_1 - V_1^T V_1||, for R R^T = AX (AX)^T + l I_m (no truncation)
    m, n, s = 40, 300, 30
    sig = datagen.spectrum("exp", m, tau=4.0)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(2, 1e-3, 1e-1), seed=23)
    A = p.A.numpy()
    G = orc.draw_gauss(11, s, n)  # X = G^T (n x s)
    Y = orc.gauss_under(A, 11, s)
    np.testing.assert_allclose(Y, A @ G.T, atol=1e-13)
    sY, U, _ = orc.jacobi_svd(Y.T)  # right singular vectors of Y^T = left singular vectors of Y
    sA = np.linalg.svd(A, compute_uv=False)
    checked = 0
    for lam in [1e-1, 1e-2]:
        D = np.hstack([A, math.sqrt(lam) * np.eye(m)])
        V1 = np.linalg.svd(D, full_matrices=False)[2].T[:n]
        assert abs(np.linalg.norm(V1) ** 2 - np.sum(sA ** 2 / (sA ** 2 + lam))) < 1e-11
        eps = np.linalg.norm(V1.T @ G.T @ G @ V1 - V1.T @ V1, 2)
        if eps >= 1:
            continue
        S = orc.lr_diag(sY, s, lam)
        RinvT = (np.eye(m) - U @ np.diag(S) @ U.T) / math.sqrt(lam)
        # R^-T is the inverse transpose of a root of Y Y^T + l I: (R^-T)^T R^-T = (Y Y^T + l I)^-1
        np.testing.assert_allclose(RinvT.T @ RinvT, np.linalg.inv(Y @ Y.T + lam * np.eye(m)), rtol=1e-8, atol=1e-8)
        assert np.linalg.cond(RinvT @ D) <= math.sqrt((1 + eps) / (1 - eps)) * (1 + 1e-8)
        checked += 1
    assert checked >= 1


# ------------------------------------------------------------ low rank -----
def test_jacobi_svd_against_lapack(orc):
    Y = RNG.standard_normal((9, 25)) @ np.diag(np.logspace(0, -6, 25))
    sig, V, sweeps = orc.jacobi_svd(Y)
    np.testing.assert_allclose(sig, np.linalg.svd(Y, compute_uv=False), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(V.T @ V, np.eye(9), atol=1e-12)
    # Y^T Y = V Sigma^2 V^T
    np.testing.assert_allclose(Y.T @ Y, V @ np.diag(sig ** 2) @ V.T, atol=1e-12)


def test_lowrank_inverse_identity(orc):
    # (l^{-1/2} (I - V S V^T))^2 = (Y^T Y + l I)^{-1}  (Section 3.1 with the corrected F and S)
    Y = RNG.standard_normal((7, 20))
    lam = 0.01
    sig, V, _ = orc.jacobi_svd(Y)
    S = orc.lr_diag(sig, 7, lam)
    Rinv = (np.eye(20) - V @ np.diag(S) @ V.T) / math.sqrt(lam)
    np.testing.assert_allclose(Rinv @ Rinv, np.linalg.inv(Y.T @ Y + lam * np.eye(20)), rtol=1e-9, atol=1e-9)


def test_sd_definition_and_lemma_3_1(orc):
    # Lemma 3.1: ||U_1||_F^2 = sd_l(A), U_1 the first m rows of the left singular vectors of B
    A, b, p = small_problem(40, 10, sig_lo=1e-3)
    sig = np.linalg.svd(A, compute_uv=False)
    for lam in [1e-4, 1e-2, 1.0]:
        B = np.vstack([A, math.sqrt(lam) * np.eye(10)])
        Ub = np.linalg.svd(B, full_matrices=False)[0]
        lhs = np.linalg.norm(Ub[:40]) ** 2
        assert abs(lhs - orc.sd_estimate(sig, lam)) < 1e-12 * 10
        assert abs(orc.sd_estimate(sig, lam) - np.sum(sig ** 2 / (sig ** 2 + lam))) < 1e-13
    assert orc.truncation(3.2, 2.0, 100) == 8
    assert orc.truncation(60.0, 2.0, 100) == 100
    assert orc.sd_estimate(np.array([1.0, 0.0]), 1.0) == 0.5


# ------------------------------------------------- convergence theory ------
def test_lemma_2_1_condition_bound(orc):
    A, b, p = small_problem(128, 10, sig_lo=1e-5)
    U_A = np.linalg.svd(A, full_matrices=False)[0]
    X = explicit_srht_over(orc, 128, 8, 64)
    Y = X @ A
    np.testing.assert_allclose(orc.srht_over(A, 8, 64), Y, atol=1e-13)
    kX = np.linalg.cond(X @ U_A)
    for lam in [1e-8, 1e-4, 1.0]:
        R, _ = orc.cholesky_shifted(orc.gram_tn(Y), lam)
        B = np.vstack([A, math.sqrt(lam) * np.eye(10)])
        assert np.linalg.cond(B @ np.linalg.inv(R)) <= kX * (1 + 1e-6)


def test_theorem_3_2_condition_bound(orc):
    m, n = 300, 40
    sig = datagen.spectrum("exp", n, tau=4.0)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(2, 1e-3, 1e-1), seed=21)
    A = p.A.numpy()
    s = 30
    G = orc.draw_gauss(7, s, m)
    Y = G @ A
    sY, V, _ = orc.jacobi_svd(Y)
    for lam in [1e-1, 1e-2]:
        B = np.vstack([A, math.sqrt(lam) * np.eye(n)])
        U1 = np.linalg.svd(B, full_matrices=False)[0][:m]
        eps = np.linalg.norm(U1.T @ G.T @ G @ U1 - U1.T @ U1, 2)
        if eps >= 1:
            continue
        S = orc.lr_diag(sY, s, lam)
        Rinv = (np.eye(n) - V @ np.diag(S) @ V.T) / math.sqrt(lam)
        assert np.linalg.cond(B @ Rinv) <= math.sqrt((1 + eps) / (1 - eps)) * (1 + 1e-8)


def test_iterations_log_one_over_eps_and_flat_in_lambda(orc):
    # O(log 1/eps) iterations with a rate set by kappa(B R^-1) <= kappa(X U_A) (Lemma 2.1), a bound
    # that does not depend on lambda or on the decay of sigma; unpreconditioned LSQR grows with kappa.
    A, b, p = small_problem(600, 20, sig_lo=1e-6)
    G = orc.draw_gauss(3, 80, 600)
    U_A = np.linalg.svd(A, full_matrices=False)[0]
    kX = np.linalg.cond(G @ U_A)
    rho_max = (kX - 1) / (kX + 1)
    Y = orc.gauss_over(A, 3, 80)
    Cm = orc.gram_tn(Y)
    its = []
    for lam in [1e-10, 1e-6, 1e-2]:
        R, _ = orc.cholesky_shifted(Cm, lam)
        B = np.vstack([A, math.sqrt(lam) * np.eye(20)])
        kap = np.linalg.cond(B @ np.linalg.inv(R))
        assert kap <= kX * (1 + 1e-6)
        rho = (kap - 1) / (kap + 1)
        for tol in [1e-6, 1e-12]:
            x, it, ist = orc.lsqr_over_chol(A, b, lam, R, tol, 500)
            bound = 1.5 * math.log(1.0 / tol) / math.log(1.0 / rho) + 5
            assert it <= bound, (lam, tol, it, bound, kap)
            if tol == 1e-12:
                its.append(it)
    flat_bound = 1.5 * math.log(1e12) / math.log(1.0 / rho_max) + 5
    assert max(its) <= flat_bound
    # unpreconditioned LSQR needs many more iterations once kappa(B) is large (Fig. 3 caption);
    # n must exceed the preconditioned count, or Krylov finite termination hides the effect
    A2, b2, _ = small_problem(800, 120, sig_lo=1e-6, seed=5)
    lam = 1e-10
    B2 = np.vstack([A2, math.sqrt(lam) * np.eye(120)])
    _, it_plain, _ = orc.lsqr_plain(B2, np.concatenate([b2, np.zeros(120)]), 1e-12, 5000)
    R2, _ = orc.cholesky_shifted(orc.gram_tn(orc.gauss_over(A2, 3, 480)), lam)
    _, it_pre, _ = orc.lsqr_over_chol(A2, b2, lam, R2, 1e-12, 500)
    assert it_plain > 4 * it_pre, (it_plain, it_pre)


# ------------------------------------------------- sparse embedding (f3) --
def test_sparse_embedding_draws_one_signed_entry_per_column(orc):
    # Section 2.1.1: one nonzero element in each column; rows uniform, signs balanced
    L, s = 20000, 64
    h, d = orc.draw_sparse(5, L, s)
    assert h.min() >= 0 and h.max() < s
    assert set(np.unique(d)) <= {-1, 1}
    assert abs(d.astype(np.float64).mean()) < 5.0 / math.sqrt(L)
    counts = np.bincount(h, minlength=s).astype(np.float64)
    expected = L / s
    chi2 = np.sum((counts - expected) ** 2 / expected)
    assert chi2 < (s - 1) + 5 * math.sqrt(2 * (s - 1))
    # the multiply-shift row: floor(w0 s / 2^32) from word 0 of Philox stream 4, the sign from word 1
    w = orc.philox4x32_10([7, 0, 4, 0], [5, 0])
    assert h[7] == (int(w[0]) * s) >> 32 and d[7] == (-1 if int(w[1]) & 1 else 1)


def _explicit_sparse(orc, seed, L, s):
    h, d = orc.draw_sparse(seed, L, s)
    X = np.zeros((s, L))
    X[h, np.arange(L)] = d
    return X


def test_sparse_sketch_is_the_explicit_embedding(orc):
    m, n, s = 700, 9, 50
    A = RNG.standard_normal((m, n))
    X = _explicit_sparse(orc, 3, m, s)
    assert np.all(np.count_nonzero(X, axis=0) == 1)
    np.testing.assert_allclose(orc.sparse_over(A, 3, s), X @ A, rtol=1e-13, atol=1e-13)
    B = RNG.standard_normal((n, m))  # underdetermined: the embedding on the columns
    np.testing.assert_allclose(orc.sparse_under(B, 3, s), B @ X.T, rtol=1e-13, atol=1e-13)
    # integer data: every partial sum is exact, so the result is exactly X A
    Ai = RNG.integers(-1000, 1000, size=(m, n)).astype(np.float64)
    assert np.array_equal(orc.sparse_over(Ai, 3, s), X @ Ai)


def test_sparse_embedding_is_isotropic_and_embeds_a_subspace(orc):
    # E[X^T X] = I (unit columns, independent signs); and for s >> k^2 a k-dim subspace is embedded
    L, s = 40, 16
    acc = np.zeros((L, L))
    T = 400
    for seed in range(T):
        X = _explicit_sparse(orc, seed, L, s)
        acc += X.T @ X
    acc /= T
    assert np.allclose(np.diag(acc), 1.0)
    off = acc - np.diag(np.diag(acc))
    assert np.abs(off).max() < 5.0 * math.sqrt(1.0 / (s * T)) + 1e-12
    m, k, s2 = 3000, 4, 1500
    U, _ = np.linalg.qr(RNG.standard_normal((m, k)))
    Y = orc.sparse_over(U, 9, s2)
    assert np.linalg.norm(Y.T @ Y - np.eye(k), 2) < 0.5


def test_alg1_with_sparse_sketch_reaches_the_reference(orc):
    # x_lambda does not depend on the embedding; the sparse sketch only changes the iteration count
    A, b, p = small_problem(1500, 30, sig_lo=1e-3)
    lams = np.array([1e-6, 1e-3, 1.0])
    X, it, _, _ = orc.alg1(A, b, lams, orc.SKETCH_SPARSE, 600, 2, 1e-14, 500)
    for i, lam in enumerate(lams):
        xr = orc.ref_ridge_qr(A, b, lam, refine=3)
        assert np.linalg.norm(X[:, i] - xr) / np.linalg.norm(xr) < 1e-10
    assert np.all(it < 200), it


# ------------------------------------------------------------- BP2 (f4) --
def test_bp2_r_is_the_qr_factor_of_the_augmented_sketch(orc):
    # Section 4.1: Q R_BP2 = [XA; sqrt(l) I]; R^T R = Y^T Y + l I, R upper triangular with diag > 0,
    # equal to the Cholesky factor of Algorithm 1 and to LAPACK's QR factor (signs fixed)
    A = RNG.standard_normal((300, 9))
    Y = orc.srht_over(A, 4, 64)
    for lam in (1e-6, 0.3):
        R = orc.bp2_r(Y, lam)
        assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
        G = Y.T @ Y + lam * np.eye(9)
        np.testing.assert_allclose(R.T @ R, G, rtol=1e-12, atol=1e-12 * np.abs(G).max())
        Rc, _ = orc.cholesky_shifted(orc.gram_tn(Y), lam)
        np.testing.assert_allclose(R, Rc, rtol=1e-10, atol=1e-12)
        Rq = np.linalg.qr(np.vstack([Y, math.sqrt(lam) * np.eye(9)]), mode="r")
        Rq = np.sign(np.diag(Rq))[:, None] * Rq
        np.testing.assert_allclose(R, Rq, rtol=1e-11, atol=1e-13)


def test_alg1_with_bp2_reaches_the_reference(orc):
    A, b, p = small_problem(1200, 25, sig_lo=1e-4)
    lams = np.array([1e-7, 1e-3, 1.0])
    X, it, _ = orc.alg1_bp2(A, b, lams, orc.SKETCH_GAUSS, 100, 3, 1e-14, 500)
    Xc, itc, _, _ = orc.alg1(A, b, lams, orc.SKETCH_GAUSS, 100, 3, 1e-14, 500)
    for i, lam in enumerate(lams):
        xr = orc.ref_ridge_qr(A, b, lam, refine=3)
        assert np.linalg.norm(X[:, i] - xr) / np.linalg.norm(xr) < 1e-10
    # the same preconditioner in exact arithmetic: the same iteration counts to within rounding
    assert np.all(np.abs(it - itc) <= 2), (it, itc)


# ----------------------------------------------------------- SRDCT (f4) --
def test_dct_rows_are_the_orthonormal_dct2(orc):
    # the defining sums against scipy's fast DCT-II (norm="ortho"), and orthogonality of the matrix
    import scipy.fft
    N = 256
    z = RNG.standard_normal(N)
    rows = np.array([0, 1, 5, 100, 255])
    np.testing.assert_allclose(orc.dct2_rows(z, rows), scipy.fft.dct(z, type=2, norm="ortho")[rows], rtol=1e-12,
                               atol=1e-13)
    Cm = np.stack([orc.dct2_rows(e, np.arange(64)) for e in np.eye(64)], axis=1)
    np.testing.assert_allclose(Cm.T @ Cm, np.eye(64), atol=1e-13)


def test_srdct_sketch_is_the_explicit_embedding(orc):
    import scipy.fft
    m, n, s = 300, 7, 40  # mp = 512: rows 300..511 are zero padding
    A = RNG.standard_normal((m, n))
    mp = 512
    d = orc.draw_signs(6, mp).astype(np.float64)
    rows = orc.draw_rows(6, mp, s)
    Z = np.zeros((mp, n))
    Z[:m] = d[:m, None] * A
    Yx = math.sqrt(mp / s) * scipy.fft.dct(Z, type=2, norm="ortho", axis=0)[rows]
    np.testing.assert_allclose(orc.srdct_over(A, 6, s), Yx, rtol=1e-11, atol=1e-12)
    B = RNG.standard_normal((n, m))
    Yu = math.sqrt(mp / s) * scipy.fft.dct(np.hstack([d[None, :m] * B, np.zeros((n, mp - m))]), type=2,
                                          norm="ortho", axis=1)[:, rows]
    np.testing.assert_allclose(orc.srdct_under(B, 6, s), Yu, rtol=1e-11, atol=1e-12)


def test_srdct_is_isotropic_in_expectation(orc):
    # E[X^T X] = (mp/s) D C^T E[S^T S] C D = I: averaged over seeds on a small case
    m, s, T = 16, 8, 300
    acc = np.zeros((m, m))
    for seed in range(T):
        X = orc.srdct_over(np.eye(m), seed, s)  # s x m: the embedding itself
        acc += X.T @ X
    acc /= T
    assert np.abs(acc - np.eye(m)).max() < 0.25


def test_alg1_with_srdct_reaches_the_reference(orc):
    A, b, p = small_problem(900, 20, sig_lo=1e-4)
    lams = np.array([1e-7, 1e-2])
    X, it, _, _ = orc.alg1(A, b, lams, orc.SKETCH_SRDCT, 100, 2, 1e-14, 500)
    for i, lam in enumerate(lams):
        xr = orc.ref_ridge_qr(A, b, lam, refine=3)
        assert np.linalg.norm(X[:, i] - xr) / np.linalg.norm(xr) < 1e-10
