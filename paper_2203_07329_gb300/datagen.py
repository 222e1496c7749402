"""Seeded synthetic ridge problems shaped like the paper's workloads (Section 4).

The paper builds A as the product of two orthogonal factors of Gaussian
matrices and a diagonal of singular values, draws x with standard normal
entries, and sets b = A x + eta with small noise.  This module does exactly
that and nothing else: it holds none of the method's arithmetic (no sketch, no
factorization of a sketched matrix, no LSQR), so both the CUDA path and the
CPU oracle may take their inputs from it.

Orthogonal factors come from a Householder QR of a seeded N(0,1) matrix with
the signs fixed so that diag(R) > 0.  The stored (rounded) A is the problem;
U, sigma, V are kept only for closed-form checks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch


@dataclass
class RidgeProblem:
    A: torch.Tensor            # m x n, row-major, float64 or float32
    b: torch.Tensor            # m, float64
    lambdas: torch.Tensor      # N, float64 (host)
    x_true: torch.Tensor       # n, float64
    sigma: torch.Tensor        # min(m, n), float64, descending
    U: torch.Tensor | None = None  # m x k orthonormal (if kept)
    V: torch.Tensor | None = None  # n x k orthonormal (if kept)
    meta: dict = field(default_factory=dict)


def spectrum(kind: str, k: int, hi: float = 1.0, lo: float = 1e-6, tau: float = 200.0) -> torch.Tensor:
    """Singular values: 'log' = log-spaced from hi to lo (both ends included),
    'exp' = sigma_i = exp(-i / tau) for i = 0..k-1."""
    if kind == "log":
        if k == 1:
            return torch.tensor([hi], dtype=torch.float64)
        e = torch.linspace(math.log10(hi), math.log10(lo), k, dtype=torch.float64)
        return torch.pow(torch.tensor(10.0, dtype=torch.float64), e)
    if kind == "exp":
        return torch.exp(-torch.arange(k, dtype=torch.float64) / tau)
    raise ValueError(kind)


def log_lambdas(N: int, lo: float, hi: float) -> torch.Tensor:
    """N regularization parameters log-spaced from lo to hi (both included)."""
    if N == 1:
        return torch.tensor([hi], dtype=torch.float64)
    return torch.pow(torch.tensor(10.0, dtype=torch.float64),
                     torch.linspace(math.log10(lo), math.log10(hi), N, dtype=torch.float64))


def _orthonormal(rows: int, cols: int, gen: torch.Generator, device, dtype) -> torch.Tensor:
    G = torch.randn(rows, cols, generator=gen, device=device, dtype=dtype)
    Q, R = torch.linalg.qr(G, mode="reduced")
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1
    return Q * d.unsqueeze(0)


def make_ridge_problem(m: int, n: int, sigma: torch.Tensor, lambdas: torch.Tensor, *, seed: int,
                       noise: float = 1e-3, dtype=torch.float64, device="cpu", keep_factors: bool = False,
                       gen_dtype=None) -> RidgeProblem:
    """A = U diag(sigma) V^T (k = min(m, n)), x_true ~ N(0, 1), b = A x_true + noise * N(0, 1) per entry.

    ``gen_dtype`` is the precision of the QR/product that builds A (defaults to
    ``dtype``); b is formed in float64 from the stored A so that it is exactly
    the product of the stored data.
    """
    gen_dtype = gen_dtype or dtype
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    k = min(m, n)
    assert sigma.numel() == k
    U = _orthonormal(m, k, gen, dev, gen_dtype)
    V = _orthonormal(n, k, gen, dev, gen_dtype)
    sig = sigma.to(device=dev, dtype=gen_dtype)
    A = ((U * sig.unsqueeze(0)) @ V.T).to(dtype).contiguous()
    x_true = torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
    eta = torch.randn(m, generator=gen, device=dev, dtype=torch.float64) * noise
    b = torch.empty(m, device=dev, dtype=torch.float64)
    step = max(1, (1 << 26) // max(n, 1))
    for r0 in range(0, m, step):
        r1 = min(m, r0 + step)
        b[r0:r1] = A[r0:r1].to(torch.float64) @ x_true
    b += eta
    prob = RidgeProblem(A=A, b=b, lambdas=lambdas.to(torch.float64).cpu(), x_true=x_true,
                        sigma=sigma.to(torch.float64).cpu(),
                        meta=dict(m=m, n=n, seed=seed, noise=noise, dtype=str(dtype)))
    if keep_factors:
        prob.U, prob.V = U, V
    return prob


# Workloads, named by what they are (shapes and spectra of the paper's synthetic
# matrices; see Section 4).  `scale` shrinks the long dimension for test-sized
# variants with the same structure.
WORKLOADS = {
    "ridge_over_4096x256_f64": dict(m=4096, n=256, spec=("log", 1.0, 1e-6), lam=(8, 1e-6, 1.0),
                                    dtype="f64", sketch="gauss", s_factor=4, seed=20220316),
    "ridge_over_262144x2048_f64": dict(m=262144, n=2048, spec=("log", 1.0, 1e-8), lam=(32, 1e-8, 1.0),
                                       dtype="f64", sketch="srht", s_factor=4, seed=20220317),
    "ridge_under_2048x262144_f64": dict(m=2048, n=262144, spec=("exp", 200.0), lam=(32, 1e-6, 1e-1),
                                        dtype="f64", sketch="srht", s_factor=4, seed=20220318),
    "ridge_over_1048576x4096_f32": dict(m=1048576, n=4096, spec=("log", 1.0, 1e-5), lam=(64, 1e-5, 1.0),
                                        dtype="f32", sketch="gauss", s_factor=2, seed=20220319),
}


def workload_problem(name: str, *, device="cpu", m: int | None = None, n: int | None = None,
                     keep_factors: bool = False, N: int | None = None) -> tuple[RidgeProblem, dict]:
    """Build the named workload (optionally with overridden m/n for a smaller
    variant of the same structure)."""
    w = dict(WORKLOADS[name])
    m = m or w["m"]
    n = n or w["n"]
    k = min(m, n)
    spec = w["spec"]
    if spec[0] == "log":
        sig = spectrum("log", k, hi=spec[1], lo=spec[2])
    else:
        sig = spectrum("exp", k, tau=spec[1])
    Nl, lo, hi = w["lam"]
    lam = log_lambdas(N or Nl, lo, hi)
    dtype = torch.float64 if w["dtype"] == "f64" else torch.float32
    prob = make_ridge_problem(m, n, sig, lam, seed=w["seed"], dtype=dtype, device=device,
                              keep_factors=keep_factors)
    w.update(m=m, n=n, N=int(lam.numel()), s=w["s_factor"] * k)
    return prob, w


def uneven_batch(P: int = 256, *, seed: int = 20220320, m_range=(2000, 65536), n_range=(64, 1024), N: int = 16,
                 lam=(1e-6, 1.0), device="cpu", dtype=torch.float32, max_total_bytes: int | None = None,
                 keep_factors: bool = False):
    """Many independent problems of uneven size: m, n uniform in the given
    ranges (m >= n enforced), half with log-spaced spectra 1..1e-5, half with
    sigma_i = exp(-i/50) (small statistical dimension)."""
    g = torch.Generator()
    g.manual_seed(seed)
    probs = []
    total = 0
    for p in range(P):
        n = int(torch.randint(n_range[0], n_range[1] + 1, (1,), generator=g))
        m = int(torch.randint(max(m_range[0], n), m_range[1] + 1, (1,), generator=g))
        lowrank = (p % 2 == 1)
        sig = spectrum("exp", n, tau=50.0) if lowrank else spectrum("log", n, hi=1.0, lo=1e-5)
        pr = make_ridge_problem(m, n, sig, log_lambdas(N, lam[0], lam[1]), seed=seed * 1000 + p, dtype=dtype,
                                device=device, keep_factors=keep_factors)
        pr.meta["lowrank"] = lowrank
        probs.append(pr)
        total += m * n * pr.A.element_size()
        if max_total_bytes is not None and total >= max_total_bytes:
            break
    return probs
