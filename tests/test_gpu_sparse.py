"""GPU parity of the sparse embedding (Section 2.1.1: one nonzero element in
each column; the sparse subspace embedding of Theorem 3.5) through the C ABI.

Integer work -- the rows h_i, the signs and the bucket lists -- is compared bit
for bit with the oracle.  The sketch itself is also bit-exact: both sides add
each bucket's rows of A in ascending row order in float64, and +-a is exact.
Solves with the sparse sketch reach the oracle's reference x to 1e-10.
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


@pytest.mark.parametrize("L,s", [(1, 1), (100, 7), (5000, 64), (1 << 18, 8192), (300001, 3000), (70000, 1 << 21),
                                 (4096, 1)])
def test_sparse_draws_and_buckets_bit_exact(tk, L, s):
    h, sign, order, start = tk.tk_sketch_draw_sparse(13, L, s)
    ho, do = oracle.draw_sparse(13, L, s)
    np.testing.assert_array_equal(h.cpu().numpy(), ho)
    np.testing.assert_array_equal(sign.cpu().numpy(), do)
    # the bucket lists: a stable sort of the columns by row (ascending column inside a bucket)
    np.testing.assert_array_equal(order.cpu().numpy(), np.argsort(ho, kind="stable"))
    np.testing.assert_array_equal(start.cpu().numpy(), np.searchsorted(np.sort(ho), np.arange(s + 1), side="left"))


@pytest.mark.parametrize("m,n,s", [(1000, 37, 300), (5000, 1, 64), (777, 130, 700), (20000, 64, 5)])
def test_sparse_over_is_bit_exact(tk, m, n, s):
    A = torch.randn(m, n, dtype=torch.float64, generator=torch.Generator().manual_seed(m + n))
    o = tk.opts_default(sketch=tk.TK_SKETCH_SPARSE, s=s, seed=11)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    assert np.array_equal(Y, oracle.sparse_over(A.numpy(), 11, s))


def test_sparse_over_float32_input_is_bit_exact(tk):
    m, n, s = 3000, 40, 256
    A = torch.randn(m, n, dtype=torch.float32, generator=torch.Generator().manual_seed(2))
    o = tk.opts_default(sketch=tk.TK_SKETCH_SPARSE, s=s, seed=4)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    assert np.array_equal(Y, oracle.sparse_over(A.double().numpy(), 4, s))


@pytest.mark.parametrize("m,n,s", [(20, 1000, 100), (3, 5000, 64)])
def test_sparse_under_is_bit_exact(tk, m, n, s):
    A = torch.randn(m, n, dtype=torch.float64, generator=torch.Generator().manual_seed(9))
    o = tk.opts_default(sketch=tk.TK_SKETCH_SPARSE, s=s, seed=4)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    assert np.array_equal(Y, oracle.sparse_under(A.numpy(), 4, s))


def problem(m, n, lo=1e-4, N=4, lam=(1e-6, 1.0), seed=3, dtype=torch.float64):
    sig = datagen.spectrum("log", min(m, n), hi=1.0, lo=lo)
    return datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(N, *lam), seed=seed, dtype=dtype)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_alg1_with_sparse_sketch_matches_oracle(tk, precision):
    p = problem(4000, 100, lo=1e-5, N=5, lam=(1e-8, 1.0))
    lams = p.lambdas.numpy()
    A, b = p.A.cuda(), p.b.cuda()
    prec = tk.TK_PREC_FP64 if precision == "fp64" else tk.TK_PREC_MIXED
    o = tk.opts_default(sketch=tk.TK_SKETCH_SPARSE, s=1600, seed=5, tol=1e-14, precision=prec)
    res = tk.tk_solve(A, b, lams, o)
    X = res.X.cpu().numpy()
    Ad, bd = p.A.numpy(), p.b.numpy()
    for i, lam in enumerate(lams):
        xr = oracle.ref_ridge_qr(Ad, bd, float(lam), refine=3)
        assert rel(X[i], xr) < TOL_X, (lam, rel(X[i], xr), res.info[i])
    if precision == "fp64":
        # the same sketch bit for bit: the iteration counts follow the oracle's Algorithm 1
        _, it_o, _, _ = oracle.alg1(Ad, bd, lams, oracle.SKETCH_SPARSE, 1600, 5, 1e-14, 500)
        its = np.array([q["iters"] for q in res.info])
        assert np.all(np.abs(its - it_o) <= 2), (its, it_o)


def test_alg2_with_sparse_sketch_matches_oracle(tk):
    m, n = 40, 3000
    sig = datagen.spectrum("exp", m, tau=10.0)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(4, 1e-6, 1e-1), seed=3)
    lams = p.lambdas.numpy()
    o = tk.opts_default(sketch=tk.TK_SKETCH_SPARSE, s=640, seed=3, tol=1e-14)
    X = tk.tk_solve(p.A.cuda(), p.b.cuda(), lams, o).X.cpu().numpy()
    for i, lam in enumerate(lams):
        xr = oracle.ref_ridge_under(p.A.numpy(), p.b.numpy(), lam, refine=3)
        assert rel(X[i], xr) < TOL_X, (lam, rel(X[i], xr))
