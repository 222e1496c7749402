"""GPU parity of the float32 LSQR products for at most 16 lambda (the tail of the
mixed form's LSQR, Algorithm 1 step 5: u' = A R^-1 v - alpha u and A^T u'),
through the C ABI (tk_lsqr_step_products, mode 2).

Two kinds of checks:
  * integer-valued inputs small enough that every float32 partial sum is an
    integer below 2^24: the products are then exact in any order of addition,
    so they must equal the integer products bit for bit -- any wrong index, lost
    row, column or lambda, or wrong split shows;
  * Gaussian inputs against float64 products, within the float32 rounding of
    the sums (each lane or thread adds at most n/32 + 8, or m/splits + 8, terms
    in order; stated per test).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_07329_gb300 import build
    build.build()
    from paper_2203_07329_gb300 import tikhonov
    tikhonov.lib()
    return tikhonov


def int_inputs(m, n, count, seed, dtype):
    g = torch.Generator().manual_seed(seed)
    A = torch.randint(-1, 2, (m, n), generator=g).to(dtype)
    W = torch.randint(-4, 5, (count, n), generator=g).float()
    U = torch.randint(-4, 5, (count, m), generator=g).float()
    coef = torch.randint(-2, 3, (count,), generator=g).double()
    return A, W, U, coef


# counts 1..16 (4-, 8- and 16-lambda kernels), n a multiple of 128, ragged (not a multiple of 4:
# scalar loads), m ragged against the 4-row groups and the splits; n beyond one chunk of W in shared
# memory (3200 columns for 16 lambda: 5000 and 3300 take two chunks, 13000 with 8 lambda two)
@pytest.mark.parametrize("m,n,count", [(1000, 200, 1), (777, 129, 3), (4097, 2048, 16), (5003, 1000, 8),
                                       (64, 2048, 5), (3, 30, 9), (2500, 513, 12), (1000, 5000, 16),
                                       (300, 3301, 9), (500, 13000, 7)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_small_products_exact_on_integers(tk, m, n, count, dtype):
    A, W, U, coef = int_inputs(m, n, count, seed=m * 7 + n + count, dtype=dtype)
    Ai = A.to(torch.int64).numpy()
    Wi, Ui, ci = W.to(torch.int64).numpy(), U.to(torch.int64).numpy(), coef.to(torch.int64).numpy()
    Uc = U.cuda()
    G = tk.tk_lsqr_step_products(A.cuda(), W.cuda(), Uc, coef.cuda(), mode=2).cpu().numpy()
    U_ref = Wi @ Ai.T + ci[:, None] * Ui
    np.testing.assert_array_equal(Uc.cpu().numpy().astype(np.int64), U_ref)
    np.testing.assert_array_equal(G.astype(np.int64), U_ref @ Ai)
    assert np.all(G == np.round(G))


@pytest.mark.parametrize("m,n,count", [(3000, 2048, 16), (2001, 300, 7), (10000, 64, 2)])
def test_small_products_gaussian(tk, m, n, count):
    g = torch.Generator().manual_seed(m + count)
    A = torch.randn(m, n, dtype=torch.float32, generator=g)
    W = torch.randn(count, n, dtype=torch.float32, generator=g)
    U = torch.randn(count, m, dtype=torch.float32, generator=g)
    coef = torch.randn(count, dtype=torch.float64, generator=g)
    Uc = U.cuda()
    G = tk.tk_lsqr_step_products(A.cuda(), W.cuda(), Uc, coef.cuda(), mode=2).cpu().numpy()
    Ad, Wd, Ud, cd = A.double().numpy(), W.double().numpy(), U.double().numpy(), coef.numpy()
    Ug = Uc.cpu().double().numpy()
    U_ref = Wd @ Ad.T + cd[:, None] * Ud
    U_mag = np.abs(Wd) @ np.abs(Ad).T + np.abs(cd[:, None] * Ud)
    assert np.all(np.abs(Ug - U_ref) <= 2.0 ** -24 * (n / 32 + 8) * U_mag)
    G_ref = Ug @ Ad
    assert np.all(np.abs(G - G_ref) <= 2.0 ** -24 * (m + 8) * (np.abs(Ug) @ np.abs(Ad)))


def test_small_products_without_coef_and_limits(tk):
    A, W, U, _ = int_inputs(300, 256, 4, seed=1, dtype=torch.float32)
    Uc = U.cuda()
    G = tk.tk_lsqr_step_products(A.cuda(), W.cuda(), Uc, None, mode=2).cpu().numpy()
    Ai, Wi = A.to(torch.int64).numpy(), W.to(torch.int64).numpy()
    np.testing.assert_array_equal(Uc.cpu().numpy().astype(np.int64), Wi @ Ai.T)
    np.testing.assert_array_equal(G.astype(np.int64), (Wi @ Ai.T) @ Ai)
    # more than 16 lambda is not this form
    A2, W2, U2, c2 = int_inputs(100, 64, 17, seed=2, dtype=torch.float32)
    with pytest.raises(tk.TikhonovError):
        tk.tk_lsqr_step_products(A2.cuda(), W2.cuda(), U2.cuda(), c2.cuda(), mode=2)
