// Batched preconditioned LSQR engine (internal).
#pragma once

#include <map>
#include <utility>
#include <vector>

#include "tk_internal.cuh"

namespace tk {

// Per-slot LSQR scalars (device resident).
struct Scal {
  double alpha, beta, rhobar, phibar, anorm2, bnorm, lam, sqrtl, coef, rnorm, arnorm, ynorm;
  int iters, istop, lam_idx, pad;
};

struct LsqrResult {
  int lam_idx, iters, istop;
  double rnorm, arnorm;
};

// Low-rank preconditioner apply (Section 3.1, eq. for R^-1):
// out_k = l^{-1/2} (in_k - V diag(S_l) V^T in_k) for each listed row k, with
// l = lam_idx[k]; V is n x s (row-major), S is N_lam x s (zero past s_l).
template <typename T>
tk_status lr_apply(int count, int64_t n, int64_t s, const T* V, const T* S, const int* lam_idx,
                   const double* lam_dev, const T* in, T* out, T* tmp, double* invs, cudaStream_t st);

// sd_i, s_i of Algorithm 3 step 5 (device in/out) and the S_i rows (step 7).
tk_status lowrank_ranks_dev(const double* sigma, int64_t s, const double* lam_dev, int N, double alpha,
                            double* sd_dev, int64_t* rank_dev, cudaStream_t st);
template <typename T>
tk_status lowrank_diag_dev(const double* sigma, int64_t s, const double* lam_dev, const int64_t* rank_dev, int N,
                           T* S, cudaStream_t st);

// One block's Golub-Kahan v-step for one slot (Paige & Saunders' LSQR):
// Vraw holds M^T u (length nv).  v' = Vraw - beta v, alpha = ||v'||, then the
// Givens rotation, the y and w updates and the stopping tests (istop 1: the
// residual test, 2: the normal-equation test, 5: non-finite, 7: iteration
// cap).  init: the first v (alpha_1 v_1 = M^T u_1), w = v, y = 0.  sh: 32
// doubles of shared memory.
template <typename T>
__device__ __forceinline__ void vstep_block(const T* __restrict__ Vraw, T* __restrict__ V, T* __restrict__ W,
                                            T* __restrict__ Y, int64_t nv, Scal* __restrict__ sq, double atol,
                                            double btol, int maxiter, int init, double* sh) {
  Scal q = *sq;
  if (!init && q.istop != 0) return;  // retired inside a chunk of steps: left as it is
  const int64_t off = 0;
  const double beta = q.beta;
  // v' = Vraw - beta v  (init: v' = Vraw)
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < nv; j += blockDim.x) {
    double v = (double)Vraw[off + j];
    if (!init) v = fma(-beta, (double)V[off + j], v);
    V[off + j] = (T)v;
    acc = fma(v, v, acc);
  }
  const double alpha = sqrt(block_sum(acc, sh));
  const double ainv = alpha > 0.0 ? 1.0 / alpha : 0.0;
  if (init) {
    double yn = 0.0;
    for (int64_t j = threadIdx.x; j < nv; j += blockDim.x) {
      T v = (T)((double)V[off + j] * ainv);
      V[off + j] = v;
      W[off + j] = v;
      Y[off + j] = T(0);
    }
    (void)yn;
    if (threadIdx.x == 0) {
      q.alpha = alpha;
      q.rhobar = alpha;
      q.coef = (q.beta > 0.0) ? -alpha / q.beta : 0.0;
      q.arnorm = alpha * q.beta;
      if (alpha == 0.0 && q.istop == 0) q.istop = 1;  // b orthogonal to range(M): y = 0 is exact
      if (!isfinite(alpha)) q.istop = 5;
      *sq = q;
    }
    return;
  }
  const double rho = sqrt(q.rhobar * q.rhobar + beta * beta);
  const double c = rho > 0.0 ? q.rhobar / rho : 1.0;
  const double sn = rho > 0.0 ? beta / rho : 0.0;
  const double theta = sn * alpha;
  const double rhobar = -c * alpha;
  const double phi = c * q.phibar;
  const double phibar = sn * q.phibar;
  const double t1 = rho > 0.0 ? phi / rho : 0.0;
  const double t2 = rho > 0.0 ? theta / rho : 0.0;
  double yy = 0.0;
  for (int64_t j = threadIdx.x; j < nv; j += blockDim.x) {
    double v = (double)V[off + j] * ainv;
    double w = (double)W[off + j];
    double y = fma(t1, w, (double)Y[off + j]);
    w = fma(-t2, w, v);
    V[off + j] = (T)v;
    W[off + j] = (T)w;
    Y[off + j] = (T)y;
    yy = fma(y, y, yy);
  }
  const double ynorm = sqrt(block_sum(yy, sh));
  if (threadIdx.x == 0) {
    q.alpha = alpha;
    q.rhobar = rhobar;
    q.phibar = phibar;
    q.iters += 1;
    q.coef = beta > 0.0 ? -alpha / beta : 0.0;
    const double rnorm = phibar;
    const double arnorm = phibar * alpha * fabs(c);
    const double anorm = sqrt(q.anorm2);
    q.rnorm = rnorm;
    q.arnorm = arnorm;
    q.ynorm = ynorm;
    int istop = 0;
    if (!isfinite(alpha) || !isfinite(beta) || !isfinite(ynorm)) istop = 5;
    else if (rnorm == 0.0) istop = 1;
    else if (arnorm / (anorm * rnorm) <= atol) istop = 2;
    else if (rnorm <= btol * q.bnorm + atol * anorm * ynorm) istop = 1;
    else if (q.iters >= maxiter) istop = 7;
    q.istop = istop;
    *sq = q;
  }
}

template <typename T>
struct Lsqr {
  // problem: A (m x n, row stride lda) in the compute type
  const T* A = nullptr;
  int64_t m = 0, n = 0, lda = 0;
  // bytes per element of A in the caller's dtype (the profiler's algorithmic bytes of one A pass)
  double a_es = sizeof(T);
  bool under = false;
  // preconditioner: per-lambda Cholesky factors R + l*rstride, or low rank
  tk_precond prec_kind = TK_PRECOND_CHOL;
  const T* R = nullptr;
  int64_t ldr = 0, rstride = 0;
  // explicit inverse: Mi = R^-1, Mti = R^-T (row stride ldm, matrix stride
  // mstride); when set it replaces the substitutions with R (overdetermined)
  const T* Mi = nullptr;
  const T* Mti = nullptr;
  int64_t ldm = 0, mstride = 0;
  int64_t lr_s = 0;
  const T* lrV = nullptr;
  const T* lrS = nullptr;
  // parameters
  int N_cap = 0;
  double atol = 1e-14, btol = 1e-14;
  int maxiter = 500;
  cudaStream_t st = nullptr;
  // workspace
  int64_t nv = 0;
  int splits = 1;      // split-K capacity of part_g
  int cur_splits = 1;  // splits of the last A^T U product (the tuned count, <= splits)
  T *V = nullptr, *W = nullptr, *Y = nullptr, *Vraw = nullptr, *Ut = nullptr, *Tt = nullptr, *Ub = nullptr,
    *xtmp = nullptr, *lr_tmp = nullptr;
  double *part_u = nullptr, *part_g = nullptr, *coef_buf = nullptr, *lr_inv = nullptr, *trsv_p = nullptr;
  Scal* sc = nullptr;
  int* slot_lam = nullptr;
  int* idx_buf = nullptr;
  const double* lam_all = nullptr;
  // tensor-core products (float32 engine only): AT = float32 A^T (n x m)
  bool tc = false;
  const T* AT = nullptr;
  void* tc_scratch = nullptr;
  // products from the 4-digit slices of A on the tensor cores (float32
  // engine, large problems): row-exponent slices of A (m x n) and
  // column-exponent slices of A^T (n x m) as made for the float64 passes
  bool oz = false;
  const void* oz_A = nullptr;
  const int* oz_EA = nullptr;
  const void* oz_AT = nullptr;
  const int* oz_EAT = nullptr;
  int* oz_err = nullptr;
  void* oz_q = nullptr;  // slices of the lambda-major vector of a product
  int* oz_e = nullptr;
  // the digit products read 8 bytes per element of A whatever the number of
  // lambdas, the float32 SIMT products 4 bytes but with work proportional to
  // it: the digits pay off for large A and more than 16 active lambdas
  bool use_oz(int count) const { return oz && oz_A && oz_AT && (int64_t)m * n > (int64_t(1) << 24) && count > 16; }
  // both products of an overdetermined step in one kernel over one read of
  // the digits (n <= 2048, at most 32 lambda per launch)
  bool oz_fused = false;
  bool use_fused(int count) const { return oz_fused && !under && use_oz(count) && oz_fused_supported(m, n, count); }

  static size_t workspace(int64_t m, int64_t n, int N_cap, bool under, int64_t lr_s);
  void carve(Arena& a);
  // Solve for `count` lambdas (indices lam_ids_dev[k] into lam_dev).  The
  // right-hand side of the k-th listed lambda is [b + k*ldbt; (bbot + k*ldbb) / sqrt(l)]
  // (overdetermined; ldbt = 0 shares b; b or bbot null = zero block) or b
  // (underdetermined).  Writes (or adds) x_l into Xout + l*ldo.
  tk_status run(const double* b, int64_t ldbt, const double* bbot, int64_t ldbb, const int* lam_ids_dev,
                const double* lam_dev, int count, double* Xout, int64_t ldo, bool accumulate,
                std::vector<LsqrResult>& results);
  tk_status apply_prec(bool transposed, const T* in, T* out, int count, int64_t len);
  tk_status prod_aw(const T* Win, int64_t ldw, T* C, const double* beta, int count);
  tk_status prod_atu(const T* Uin, int count);
  tk_status prod_fused(const T* Win, T* C, const double* beta, int count);
  tk_status gather_coef(int count);
  // one LSQR step for slots 0..nact-1; `count` of them (see steps())
  tk_status step(int nact);
  tk_status steps(int nact, int count);
  void release_graphs();
  int chunk = 1;
  std::map<int, std::pair<cudaGraphExec_t, size_t>> graphs;  // active count -> (replay, kernel nodes)
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
};

}  // namespace tk
