"""GPU parity of the SRDCT embedding (Section 2.1.1 with the discrete cosine
transform; the embedding of the paper's Fig. 1-2) through the C ABI.

The GPU forms the orthonormal DCT-II of each sign-flipped, zero-padded column
through one complex FFT of the same length (Makhoul's reordering, radix-2
passes in shared memory) and evaluates only the sampled rows; the oracle forms
each sampled row by its defining sum.  Both are float64: they agree to
rounding, 1e-12 of the largest |Y|.  The signs and rows are the SRHT's draws,
already compared bit for bit in test_gpu_parity.
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


@pytest.mark.parametrize("m,n,s", [(1000, 37, 300), (512, 16, 512), (3000, 130, 700), (700, 1, 50), (1, 1, 1),
                                   (2, 1, 2), (300, 7, 40)])
def test_srdct_over_matches_oracle(tk, m, n, s):
    A = torch.randn(m, n, dtype=torch.float64, generator=torch.Generator().manual_seed(m + 3 * n))
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRDCT, s=s, seed=6)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    Yo = oracle.srdct_over(A.numpy(), 6, s)
    np.testing.assert_allclose(Y, Yo, rtol=1e-12, atol=1e-12 * np.abs(Yo).max())


def test_srdct_over_three_passes(tk):
    # 2^17 padded rows: passes of 8 + 8 + 1 stages
    m, n, s = 70000, 3, 64
    A = torch.randn(m, n, dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRDCT, s=s, seed=2)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    Yo = oracle.srdct_over(A.numpy(), 2, s)
    np.testing.assert_allclose(Y, Yo, rtol=1e-11, atol=1e-11 * np.abs(Yo).max())


@pytest.mark.parametrize("m,n,s", [(20, 1000, 100), (3, 5000, 64)])
def test_srdct_under_matches_oracle(tk, m, n, s):
    A = torch.randn(m, n, dtype=torch.float64, generator=torch.Generator().manual_seed(9))
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRDCT, s=s, seed=4)
    Y = tk.tk_sketch_apply(A.cuda(), o).cpu().numpy()
    Yo = oracle.srdct_under(A.numpy(), 4, s)
    np.testing.assert_allclose(Y, Yo, rtol=1e-12, atol=1e-12 * np.abs(Yo).max())


@pytest.mark.parametrize("precision,precond", [("fp64", "chol"), ("mixed", "chol"), ("fp64", "qr")])
def test_alg1_with_srdct_matches_oracle(tk, precision, precond):
    # the paper's Fig. 2 pairing: an SRDCT sketch with the Cholesky (Algorithm 1) or BP2 preconditioner
    sig = datagen.spectrum("log", 100, hi=1.0, lo=1e-5)
    p = datagen.make_ridge_problem(3000, 100, sig, datagen.log_lambdas(4, 1e-8, 1.0), seed=5)
    lams = p.lambdas.numpy()
    o = tk.opts_default(sketch=tk.TK_SKETCH_SRDCT, s=500, seed=7,
                        precision=tk.TK_PREC_FP64 if precision == "fp64" else tk.TK_PREC_MIXED,
                        precond=tk.TK_PRECOND_CHOL if precond == "chol" else tk.TK_PRECOND_QR)
    res = tk.tk_solve(p.A.cuda(), p.b.cuda(), lams, o)
    X = res.X.cpu().numpy()
    Ad, bd = p.A.numpy(), p.b.numpy()
    for i, lam in enumerate(lams):
        xr = oracle.ref_ridge_qr(Ad, bd, float(lam), refine=3)
        assert rel(X[i], xr) < TOL_X, (lam, rel(X[i], xr), res.info[i])
    if precision == "fp64" and precond == "chol":
        _, it_o, _, _ = oracle.alg1(Ad, bd, lams, oracle.SKETCH_SRDCT, 500, 7, 1e-14, 500)
        its = np.array([q["iters"] for q in res.info])
        assert np.all(np.abs(its - it_o) <= 2), (its, it_o)
