// Preconditioned LSQR for many lambda at once (Algorithm 1 step 5,
// Algorithm 2 step 5, Algorithm 3 step 8; LSQR of Paige & Saunders 1982).
//
// Every active lambda owns a "slot".  Per-slot vectors are stored
// lambda-major (slot s is row s of an N_cap x len matrix), so one GEMM with A
// advances all active lambda together and a converged lambda is retired by
// moving the last active slot into its place.
//
// Overdetermined (B R^-1, B = [A; sqrt(l) I]), one step for all slots:
//   T  = R^-1 V                                   (preconditioner apply)
//   Ut = T A^T - (alpha/beta) Ut                  (GEMM, u kept unnormalized)
//   Ub = sqrt(l) T - (alpha/beta) Ub,  beta = ||[Ut; Ub]||
//   G  = (Ut A + sqrt(l) Ub) / beta               (split-K GEMM)
//   H  = R^-T G;  alpha v = H - beta v;  Givens;  y += (phi/rho) w;  w = v - (theta/rho) w
// Underdetermined (R^-T D, D = [A sqrt(l) I], min-norm):
//   P  = V1 A^T + sqrt(l) V2;  u = R^-T P - alpha u;  beta = ||u||
//   T  = R^-1 u;  v = [T A; sqrt(l) T] - beta v;  alpha = ||v||;  Givens on z = [x; y]
#include <type_traits>
#include <vector>

#include "tk_lsqr.cuh"

namespace tk {
namespace {

constexpr int kVecThreads = 256;
constexpr int kSumChunks = 64;

// partial[s * chunks + c] = sum of squares of row s over chunk c
template <typename T>
__global__ void k_sumsq_rows(const T* __restrict__ X, int64_t ld, int64_t len, int chunks,
                             double* __restrict__ partial) {
  __shared__ double sh[32];
  const int s = blockIdx.y, c = blockIdx.x;
  const int64_t per = cdiv(len, chunks);
  const int64_t b = (int64_t)c * per, e = std::min(len, b + per);
  const T* x = X + (int64_t)s * ld;
  double acc = 0.0;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
    double v = (double)x[i];
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[s * chunks + c] = acc;
}

// ---- overdetermined ---------------------------------------------------
// Init of the right-hand side [bt; bb / sqrt(l)]: bt = b + s*ldbt (null = 0),
// bb = bbot + s*ldbb (null = 0).  At init, slot s holds the s-th listed lambda.
template <typename T>
__global__ void k_over_init_u(const double* __restrict__ b, int64_t ldbt, int64_t m, const double* __restrict__ bbot,
                              int64_t ldbb, int64_t n, const Scal* __restrict__ sc, T* __restrict__ Ut,
                              T* __restrict__ Ub) {
  const int s = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const double* bt = b ? b + (int64_t)s * ldbt : nullptr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride)
    Ut[(int64_t)s * m + i] = bt ? (T)bt[i] : T(0);
  const double* bb = bbot ? bbot + (int64_t)s * ldbb : nullptr;
  const double inv = 1.0 / sc[s].sqrtl;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += stride)
    Ub[(int64_t)s * n + j] = bb ? (T)(bb[j] * inv) : T(0);
}

// beta_1 = ||[Ut; Ub]||; scalars reset.
template <typename T>
__global__ void k_over_init_beta(const double* __restrict__ part, int chunks, const T* __restrict__ Ub, int64_t n,
                                 Scal* __restrict__ sc) {
  __shared__ double sh[32];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    double v = (double)Ub[(int64_t)s * n + j];
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    double t = acc;
    for (int c = 0; c < chunks; ++c) t += part[s * chunks + c];
    double beta = sqrt(t);
    Scal q = sc[s];
    q.beta = beta;
    q.bnorm = beta;
    q.phibar = beta;
    q.anorm2 = 0.0;
    q.iters = 0;
    q.istop = (beta == 0.0) ? 1 : 0;
    q.rnorm = beta;
    q.arnorm = 0.0;
    q.ynorm = 0.0;
    sc[s] = q;
  }
}

// Ub = sqrt(l) T + coef Ub;  beta = sqrt(sum partial + ||Ub||^2);  anorm2 += alpha^2 + beta^2
template <typename T>
__global__ void k_over_beta(const double* __restrict__ part, int chunks, const T* __restrict__ Tt,
                            T* __restrict__ Ub, int64_t n, Scal* __restrict__ sc) {
  __shared__ double sh[32];
  const int s = blockIdx.x;
  if (sc[s].istop != 0) return;  // retired inside a chunk of steps
  const double sl = sc[s].sqrtl, coef = sc[s].coef;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    int64_t k = (int64_t)s * n + j;
    double v = fma(sl, (double)Tt[k], coef * (double)Ub[k]);
    T vt = (T)v;
    Ub[k] = vt;
    acc = fma((double)vt, (double)vt, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    double t = acc;
    for (int c = 0; c < chunks; ++c) t += part[s * chunks + c];
    double beta = sqrt(t);
    Scal q = sc[s];
    q.anorm2 += q.alpha * q.alpha + beta * beta;
    q.beta = beta;
    sc[s] = q;
  }
}

// C[k] = sum_z partial[z][k] (the split-K planes of a product, in order)
template <typename T>
__global__ void k_sum_planes_to(const double* __restrict__ part, int splits, int64_t total, T* __restrict__ C) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < splits; ++z) acc += part[(int64_t)z * total + k];
    C[k] = (T)acc;
  }
}

// G = (sum_z partial_z + sqrt(l) Ub) / beta
template <typename T>
__global__ void k_over_g(const double* __restrict__ part, int splits, int count, const T* __restrict__ Ub, int64_t n,
                         const Scal* __restrict__ sc, T* __restrict__ G) {
  const int s = blockIdx.y;
  const double sl = sc[s].sqrtl, beta = sc[s].beta;
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  const int64_t plane = (int64_t)count * n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < splits; ++z) acc += part[z * plane + (int64_t)s * n + j];
    acc = fma(sl, (double)Ub[(int64_t)s * n + j], acc);
    G[(int64_t)s * n + j] = (T)(acc * inv);
  }
}

// ---- shared Golub-Kahan v-step + Givens + tests (body: vstep_block) ---
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
    k_vstep(const T* __restrict__ Vraw, T* __restrict__ V, T* __restrict__ W, T* __restrict__ Y, int64_t nv,
            Scal* __restrict__ sc, double atol, double btol, int maxiter, int init) {
  __shared__ double sh[32];
  const int s = blockIdx.x;
  const int64_t off = (int64_t)s * nv;
  vstep_block<T>(Vraw + off, V + off, W + off, Y + off, nv, sc + s, atol, btol, maxiter, init, sh);
}

// ---- underdetermined ----------------------------------------------------
// P = V1 A^T (from the GEMM) + sqrt(l) V2 ;  in place on P.
template <typename T>
__global__ void k_under_addv2(T* __restrict__ P, int64_t m, const T* __restrict__ V, int64_t nv, int64_t n,
                              const Scal* __restrict__ sc) {
  const int s = blockIdx.y;
  const double sl = sc[s].sqrtl;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    P[(int64_t)s * m + i] = (T)((double)P[(int64_t)s * m + i] + sl * (double)V[(int64_t)s * nv + n + i]);
}

// u = Q - alpha u (init: u = Q), beta = ||u||, u /= beta, anorm2 += alpha^2 + beta^2
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
    k_under_ustep(const T* __restrict__ Q, T* __restrict__ U, int64_t m, Scal* __restrict__ sc, int init) {
  __shared__ double sh[32];
  const int s = blockIdx.x;
  Scal q = sc[s];
  if (!init && q.istop != 0) return;  // retired inside a chunk of steps
  const int64_t off = (int64_t)s * m;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    double u = (double)Q[off + i];
    if (!init) u = fma(-q.alpha, (double)U[off + i], u);
    U[off + i] = (T)u;
    acc = fma(u, u, acc);
  }
  const double beta = sqrt(block_sum(acc, sh));
  const double binv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) U[off + i] = (T)((double)U[off + i] * binv);
  if (threadIdx.x == 0) {
    if (init) {
      q.beta = beta;
      q.bnorm = beta;
      q.phibar = beta;
      q.anorm2 = 0.0;
      q.iters = 0;
      q.istop = (beta == 0.0) ? 1 : 0;
      q.rnorm = beta;
      q.arnorm = 0.0;
      q.ynorm = 0.0;
    } else {
      q.anorm2 += q.alpha * q.alpha + beta * beta;
      q.beta = beta;
    }
    sc[s] = q;
  }
}

// Vraw = [sum_z partial_z ; sqrt(l) T]   (length n + m)
template <typename T>
__global__ void k_under_vraw(const double* __restrict__ part, int splits, int count, const T* __restrict__ Tm,
                             int64_t m, int64_t n, const Scal* __restrict__ sc, T* __restrict__ Vraw) {
  const int s = blockIdx.y;
  const double sl = sc[s].sqrtl;
  const int64_t nv = n + m, plane = (int64_t)count * n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nv; j += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (j < n) {
      v = 0.0;
      for (int z = 0; z < splits; ++z) v += part[z * plane + (int64_t)s * n + j];
    } else {
      v = sl * (double)Tm[(int64_t)s * m + (j - n)];
    }
    Vraw[(int64_t)s * nv + j] = (T)v;
  }
}

// Init of the underdetermined rhs: P = b for every slot (then R^-T applied).
template <typename T>
__global__ void k_bcast_rows(const double* __restrict__ b, int64_t m, T* __restrict__ P) {
  const int s = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    P[(int64_t)s * m + i] = (T)b[i];
}

// ---- slot bookkeeping -----------------------------------------------------
template <typename T>
__global__ void k_move_rows(T* __restrict__ X, int64_t len, const int* __restrict__ src, const int* __restrict__ dst,
                            int moves) {
  const int k = blockIdx.y;
  if (k >= moves) return;
  const int64_t a = src[k], b = dst[k];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    X[b * len + i] = X[a * len + i];
}

__global__ void k_move_scal(Scal* __restrict__ sc, int* __restrict__ slot_lam, const int* __restrict__ src,
                            const int* __restrict__ dst, int moves) {
  for (int k = threadIdx.x; k < moves; k += blockDim.x) {
    sc[dst[k]] = sc[src[k]];
    slot_lam[dst[k]] = slot_lam[src[k]];
  }
}

// X_out[lam] (+)= Xs[slot] for the listed slots (first n entries of rows of length ld)
template <typename T>
__global__ void k_scatter_out(const T* __restrict__ Xs, int64_t ld, int64_t n, const int* __restrict__ slots,
                              const int* __restrict__ slot_lam, double* __restrict__ Xout, int64_t ldo, int accumulate) {
  const int k = blockIdx.y;
  const int s = slots[k];
  const int l = slot_lam[s];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)Xs[(int64_t)k * ld + j];
    if (accumulate) Xout[(int64_t)l * ldo + j] += v;
    else Xout[(int64_t)l * ldo + j] = v;
  }
}

template <typename T>
__global__ void k_gather_rows(const T* __restrict__ X, int64_t ld, int64_t len, const int* __restrict__ slots,
                              T* __restrict__ out) {
  const int k = blockIdx.y;
  const int s = slots[k];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x)
    out[(int64_t)k * ld + j] = X[(int64_t)s * ld + j];
}

__global__ void k_init_scal(Scal* __restrict__ sc, int* __restrict__ slot_lam, const int* __restrict__ lam_ids,
                            const double* __restrict__ lam, int count) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  Scal q;
  memset(&q, 0, sizeof(q));
  int l = lam_ids[s];
  q.lam_idx = l;
  q.lam = lam[l];
  q.sqrtl = sqrt(lam[l]);
  sc[s] = q;
  slot_lam[s] = l;
}

inline dim3 rows_grid(int64_t len, int count) {
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(len, 256), 64)), (unsigned)count);
}

}  // namespace

// ------------------------------------------------------------------------
template <typename T>
size_t Lsqr<T>::workspace(int64_t m, int64_t n, int N_cap, bool under, int64_t lr_s) {
  Lsqr<T> e;
  e.m = m;
  e.n = n;
  e.N_cap = N_cap;
  e.under = under;
  e.lr_s = lr_s;
  e.tc = false;
  Arena a;
  e.carve(a);
  return a.used + 4096;
}

template <typename T>
void Lsqr<T>::carve(Arena& a) {
  nv = under ? n + m : n;
  const int64_t nu = m;  // length of the GEMM-facing u rows
  const int64_t gcols = n;
  splits = splitk_count(N_cap, gcols, m);
  if (std::is_same<T, float>::value) splits = std::max(splits, lm_small_atu_splits(m, n));  // <= 16 lambda
  if (oz && oz_fused) splits = std::max(splits, 152);  // one partial plane per cluster of the fused step
  V = a.take<T>((size_t)N_cap * nv);
  W = a.take<T>((size_t)N_cap * nv);
  Y = a.take<T>((size_t)N_cap * nv);
  Vraw = a.take<T>((size_t)N_cap * nv);
  Ut = a.take<T>((size_t)N_cap * nu);
  Tt = a.take<T>((size_t)N_cap * std::max(n, m));
  Ub = under ? nullptr : a.take<T>((size_t)N_cap * n);
  part_u = a.take<double>((size_t)N_cap * kSumChunks);
  part_g = a.take<double>((size_t)splits * N_cap * gcols);
  coef_buf = a.take<double>((size_t)N_cap);
  sc = a.take<Scal>((size_t)N_cap);
  slot_lam = a.take<int>((size_t)N_cap);
  idx_buf = a.take<int>((size_t)N_cap * 3);
  xtmp = a.take<T>((size_t)N_cap * std::max(n, m));
  trsv_p = a.take<double>((size_t)N_cap * std::max(n, m));
  if (lr_s > 0) {
    lr_tmp = a.take<T>((size_t)N_cap * lr_s);
    lr_inv = a.take<double>((size_t)N_cap);
  }
  if (tc) tc_scratch = a.take<char>(tc_lmaj_workspace(N_cap, std::max(n, m)));
  if (oz) {
    oz_q = a.take<char>(oz_slices_bytes(N_cap, std::max(n, m), OZ_LSQR_DIGITS));
    oz_e = a.take<int>((size_t)N_cap);
  }
}

template <typename T>
tk_status Lsqr<T>::apply_prec(bool transposed, const T* in, T* out, int count, int64_t len) {
  const double es = (double)sizeof(T);
  if (prec_kind == TK_PRECOND_CHOL) {
    int tok = prof_begin(TK_PHASE_PRECOND, st);
    tk_status r;
    if (Mi) {
      r = trmv_batched<T>(transposed, len, Mi, Mti, ldm, mstride, slot_lam, in, out, len, count, st);
      prof_end(tok, st, (double)count * len * len, es * count * (len * (len + 1) / 2 + 2 * len));
      return r;
    }
    r = trsv_batched<T, T>(transposed, len, R, ldr, rstride, slot_lam, in, out, len, count, trsv_p, st);
    prof_end(tok, st, (double)count * len * len, es * count * (len * (len + 1) / 2 + 2 * len));
    return r;
  }
  // Low rank: out = l^{-1/2}(in - V S V^T in); symmetric, so transposed is the same.
  int tok = prof_begin(TK_PHASE_PRECOND, st);
  tk_status r = lr_apply<T>(count, len, lr_s, lrV, lrS, slot_lam, lam_all, in, out, lr_tmp, lr_inv, st);
  prof_end(tok, st, 4.0 * count * len * lr_s, es * (len * lr_s + 2.0 * count * len));
  return r;
}

inline double total_count(int count, int64_t m) { return (double)count * (double)m; }

template <typename T>
tk_status Lsqr<T>::prod_aw(const T* Win, int64_t ldw, T* C, const double* beta, int count) {
  // C (count x m) = Win (count x n) A^T  [+ beta_row * C]
  const bool digits = use_oz(count);
  const double es = (double)sizeof(T);
  const double vec = es * (count * (double)n + 2.0 * count * m);
  int tok = prof_begin(digits ? TK_PHASE_AW_DIGITS : TK_PHASE_AW, st);
  tk_status r;
  if constexpr (std::is_same<T, float>::value) {
    if (digits) {
      r = oz_lsqr_aw(oz_A, oz_EA, m, n, Win, ldw, count, oz_q, oz_e, C, m, beta, oz_err, st);
      prof_end(tok, st, 2.0 * count * m * n, a_es * m * n + vec, 8.0 * m * n + vec);
      return r;
    }
    if (tc && beta) {
      r = tc_lmaj_product(true, A, m, n, lda, Win, ldw, count, C, m, beta, nullptr, 1, tc_scratch, st);
      prof_end(tok, st, 2.0 * count * m * n, a_es * m * n + vec, es * m * n + vec);
      return r;
    }
    if (!under && lm_small_aw_supported(n, count)) {  // <= 16 lambda: W on chip, one pass over A's rows
      r = lm_small_aw(A, lda, m, n, Win, ldw, count, C, m, beta, st);
      prof_end(tok, st, 2.0 * count * m * n, a_es * m * n + vec, es * m * n + vec);
      return r;
    }
  }
  if (under && !beta) {
    // the underdetermined product: a short output (count x m, m < n) against a long K = n; split K
    // over the GPU and add the planes (part_g holds splits x N_cap x n >= sp x count x m values)
    const int64_t cap = ((int64_t)splits * N_cap * n) / std::max<int64_t>((int64_t)count * m, 1);
    const int sp = (int)std::min<int64_t>(splitk_count(count, m, n), cap);
    if (sp > 1) {
      r = gemm_splitk<T, T>(false, true, count, m, n, Win, ldw, A, lda, part_g, sp, st);
      if (r == TK_OK) {
        const int64_t total = (int64_t)count * m;
        k_sum_planes_to<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), 152 * 8)), 256, 0,
                             st>>>(part_g, sp, total, C);
        TK_LAUNCH_CHECK();
      }
      prof_end(tok, st, 2.0 * count * m * n, a_es * m * n + vec + 16.0 * sp * total_count(count, m),
               es * m * n + vec + 16.0 * sp * total_count(count, m));
      return r;
    }
  }
  r = gemm<T, T, T>(false, true, count, m, n, Win, ldw, A, lda, C, m, 1.0, beta, beta ? C : nullptr, m, st);
  prof_end(tok, st, 2.0 * count * m * n, a_es * m * n + vec, es * m * n + vec);
  return r;
}

template <typename T>
tk_status Lsqr<T>::prod_atu(const T* Uin, int count) {
  // part_g (splits x count x n) = Uin (count x m) A
  const bool digits = use_oz(count);
  const double es = (double)sizeof(T);
  int tok = prof_begin(digits ? TK_PHASE_ATU_DIGITS : TK_PHASE_ATU, st);
  tk_status r;
  if constexpr (std::is_same<T, float>::value) {
    if (digits) {
      cur_splits = std::min(splits, oz_normal_splits(m, n, count, OZ_LSQR_DIGITS));
      const double vec = es * count * (double)m + 8.0 * cur_splits * count * n;
      r = oz_lsqr_atu(oz_AT, oz_EAT, m, n, Uin, m, count, oz_q, oz_e, part_g, cur_splits, oz_err, st);
      prof_end(tok, st, 2.0 * count * m * n, a_es * m * n + vec, 8.0 * m * n + vec);
      return r;
    }
    if (tc && AT) {
      cur_splits = splits;
      const double vec = es * count * (double)m + 8.0 * splits * count * n;
      r = tc_lmaj_product(false, AT, n, m, m, Uin, m, count, nullptr, 0, nullptr, part_g, splits, tc_scratch, st);
      prof_end(tok, st, 2.0 * count * m * n, a_es * m * n + vec, es * m * n + vec);
      return r;
    }
    if (count <= 16) {  // <= 16 lambda: NL x 4 accumulators per thread, U staged on chip
      cur_splits = std::min(splits, lm_small_atu_splits(m, n));
      const double vec = es * count * (double)m + 8.0 * cur_splits * count * n;
      r = lm_small_atu(A, lda, m, n, Uin, m, count, part_g, cur_splits, st);
      prof_end(tok, st, 2.0 * count * m * n, a_es * m * n + vec, es * m * n + vec);
      return r;
    }
  }
  cur_splits = splitk_tuned<T, T>(count, n, m, splits);
  const double vec = es * count * (double)m + 8.0 * cur_splits * count * n;
  r = gemm_splitk<T, T>(false, false, count, n, m, Uin, m, A, lda, part_g, cur_splits, st);
  prof_end(tok, st, 2.0 * count * m * n, a_es * m * n + vec, es * m * n + vec);
  return r;
}

template <typename T>
tk_status Lsqr<T>::prod_fused(const T* Win, T* C, const double* beta, int count) {
  // C (count x m) = Win A^T + beta .* C, then part_g (cur_splits x count x n) = C A
  const double es = (double)sizeof(T);
  int tok = prof_begin(TK_PHASE_LSQR_FUSED, st);
  tk_status r = TK_EINVAL;
  if constexpr (std::is_same<T, float>::value)
    r = oz_lsqr_fused(oz_A, oz_EA, m, n, Win, n, count, oz_q, oz_e, C, m, beta, part_g, splits, &cur_splits, oz_err,
                      st);
  // A once from memory (its second read, a few microseconds later, comes from L2)
  const double vec = es * (count * (double)n + 2.0 * count * m) + 8.0 * cur_splits * count * n;
  prof_end(tok, st, 4.0 * count * m * n, a_es * m * n + vec, 8.0 * m * n + vec);
  return r;
}

template <typename T>
tk_status Lsqr<T>::run(const double* b, int64_t ldbt, const double* bbot, int64_t ldbb, const int* lam_ids_dev,
                       const double* lam_dev, int count, double* Xout, int64_t ldo, bool accumulate,
                       std::vector<LsqrResult>& results) {
  if (count <= 0) return TK_OK;
  if (count > N_cap) {
    set_error_msg("lsqr: more lambdas than slots");
    return TK_EINVAL;
  }
  int nact = count;
  lam_all = lam_dev;
  k_init_scal<<<cdiv(count, 128), 128, 0, st>>>(sc, slot_lam, lam_ids_dev, lam_dev, count);
  TK_LAUNCH_CHECK();
  // ---------------------------------------------------------------- init
  if (!under) {
    k_over_init_u<T><<<rows_grid(std::max(m, n), nact), 256, 0, st>>>(b, ldbt, m, bbot, ldbb, n, sc, Ut, Ub);
    TK_LAUNCH_CHECK();
    k_sumsq_rows<T><<<dim3(kSumChunks, nact), 256, 0, st>>>(Ut, m, m, kSumChunks, part_u);
    TK_LAUNCH_CHECK();
    k_over_init_beta<T><<<nact, kVecThreads, 0, st>>>(part_u, kSumChunks, Ub, n, sc);
    TK_LAUNCH_CHECK();
    TK_TRY(prod_atu(Ut, nact));
    k_over_g<T><<<rows_grid(n, nact), 256, 0, st>>>(part_g, cur_splits, nact, Ub, n, sc, Tt);
    TK_LAUNCH_CHECK();
    TK_TRY(apply_prec(true, Tt, Vraw, nact, n));
  } else {
    k_bcast_rows<T><<<rows_grid(m, nact), 256, 0, st>>>(b, m, Tt);
    TK_LAUNCH_CHECK();
    TK_TRY(apply_prec(true, Tt, Tt, nact, m));
    k_under_ustep<T><<<nact, kVecThreads, 0, st>>>(Tt, Ut, m, sc, 1);
    TK_LAUNCH_CHECK();
    TK_TRY(apply_prec(false, Ut, Tt, nact, m));
    TK_TRY(prod_atu(Tt, nact));
    k_under_vraw<T><<<rows_grid(nv, nact), 256, 0, st>>>(part_g, cur_splits, nact, Tt, m, n, sc, Vraw);
    TK_LAUNCH_CHECK();
  }
  k_vstep<T><<<nact, kVecThreads, 0, st>>>(Vraw, V, W, Y, nv, sc, atol, btol, maxiter, 1);
  TK_LAUNCH_CHECK();

  // steps per read of the scalars: several for problems whose steps are
  // launch-bound (A of at most 2^24 elements), one otherwise
  chunk = ((int64_t)m * n <= (int64_t(1) << 24)) ? 4 : 1;
  std::vector<Scal> hsc(N_cap);
  std::vector<int> hlam(N_cap);
  int* d_src = idx_buf;
  int* d_dst = idx_buf + N_cap;
  int* d_ret = idx_buf + 2 * N_cap;
  for (;;) {
    // ------------------------------------------------ retire finished slots
    TK_CUDA(cudaMemcpyAsync(hsc.data(), sc, sizeof(Scal) * nact, cudaMemcpyDeviceToHost, st));
    TK_CUDA(cudaStreamSynchronize(st));
    std::vector<int> ret, keep;
    for (int s = 0; s < nact; ++s) (hsc[s].istop != 0 ? ret : keep).push_back(s);
    if (!ret.empty()) {
      const int nr = (int)ret.size();
      TK_CUDA(cudaMemcpyAsync(d_ret, ret.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, st));
      // x = R^-1 y (over) or x = z[0:n] (under)
      k_gather_rows<T><<<rows_grid(nv, nr), 256, 0, st>>>(Y, nv, nv, d_ret, Vraw);
      TK_LAUNCH_CHECK();
      const T* xs = Vraw;
      if (!under) {
        // slot_lam of the gathered rows: reuse d_src as the lambda index list
        for (int k = 0; k < nr; ++k) hlam[k] = hsc[ret[k]].lam_idx;
        TK_CUDA(cudaMemcpyAsync(d_src, hlam.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, st));
        if (prec_kind == TK_PRECOND_CHOL) {
          if (Mi) TK_TRY(trmv_batched<T>(false, n, Mi, Mti, ldm, mstride, d_src, Vraw, xtmp, n, nr, st));
          else TK_TRY((trsv_batched<T, T>(false, n, R, ldr, rstride, d_src, Vraw, xtmp, n, nr, trsv_p, st)));
        } else {
          TK_TRY(lr_apply<T>(nr, n, lr_s, lrV, lrS, d_src, lam_all, Vraw, xtmp, lr_tmp, lr_inv, st));
        }
        xs = xtmp;
      }
      k_scatter_out<T><<<rows_grid(n, nr), 256, 0, st>>>(xs, under ? nv : n, n, d_ret, slot_lam, Xout, ldo,
                                                         accumulate ? 1 : 0);
      TK_LAUNCH_CHECK();
      for (int k = 0; k < nr; ++k) {
        const Scal& q = hsc[ret[k]];
        LsqrResult r;
        r.lam_idx = q.lam_idx;
        r.iters = q.iters;
        r.istop = q.istop;
        r.rnorm = q.rnorm;
        r.arnorm = q.arnorm;
        results.push_back(r);
      }
      // compaction: survivors beyond the new end move into holes below it
      const int nnew = nact - nr;
      std::vector<int> holes, srcs;
      for (int s : ret)
        if (s < nnew) holes.push_back(s);
      for (int s : keep)
        if (s >= nnew) srcs.push_back(s);
      const int moves = (int)holes.size();
      if (moves > 0) {
        TK_CUDA(cudaMemcpyAsync(d_src, srcs.data(), sizeof(int) * moves, cudaMemcpyHostToDevice, st));
        TK_CUDA(cudaMemcpyAsync(d_dst, holes.data(), sizeof(int) * moves, cudaMemcpyHostToDevice, st));
        k_move_rows<T><<<rows_grid(nv, moves), 256, 0, st>>>(V, nv, d_src, d_dst, moves);
        k_move_rows<T><<<rows_grid(nv, moves), 256, 0, st>>>(W, nv, d_src, d_dst, moves);
        k_move_rows<T><<<rows_grid(nv, moves), 256, 0, st>>>(Y, nv, d_src, d_dst, moves);
        k_move_rows<T><<<rows_grid(m, moves), 256, 0, st>>>(Ut, m, d_src, d_dst, moves);
        if (!under) k_move_rows<T><<<rows_grid(n, moves), 256, 0, st>>>(Ub, n, d_src, d_dst, moves);
        k_move_scal<<<1, 128, 0, st>>>(sc, slot_lam, d_src, d_dst, moves);
        TK_LAUNCH_CHECK();
      }
      nact = nnew;
      // the host copies of d_src/d_dst/d_ret must stay valid until the copies ran
      TK_CUDA(cudaStreamSynchronize(st));
    }
    if (nact == 0) break;
    // ------------------------------------------- `chunk` steps, one replay
    // Small problems run several steps between two reads of the scalars (a
    // slot that converges inside the chunk stays as it is: its kernels skip
    // it), replayed from a CUDA graph captured once per active count.
    const tk_status sr = steps(nact, chunk);
    if (sr != TK_OK) {
      release_graphs();
      return sr;
    }
  }
  release_graphs();
  if (tc) TK_TRY(tc_lmaj_check(tc_scratch, N_cap, std::max(n, m), st));
  return TK_OK;
}

template <typename T>
tk_status Lsqr<T>::step(int nact) {
  if (!under) {
    TK_TRY(apply_prec(false, V, Tt, nact, n));  // T = R^-1 v
    TK_TRY(gather_coef(nact));
    if (use_fused(nact)) {  // u' = A R^-1 v - alpha u and A^T u' over one read of A's digits
      TK_TRY(prod_fused(Tt, Ut, coef_buf, nact));
      k_sumsq_rows<T><<<dim3(kSumChunks, nact), 256, 0, st>>>(Ut, m, m, kSumChunks, part_u);
      TK_LAUNCH_CHECK();
      k_over_beta<T><<<nact, kVecThreads, 0, st>>>(part_u, kSumChunks, Tt, Ub, n, sc);
      TK_LAUNCH_CHECK();
    } else {
      TK_TRY(prod_aw(Tt, n, Ut, coef_buf, nact));
      k_sumsq_rows<T><<<dim3(kSumChunks, nact), 256, 0, st>>>(Ut, m, m, kSumChunks, part_u);
      TK_LAUNCH_CHECK();
      k_over_beta<T><<<nact, kVecThreads, 0, st>>>(part_u, kSumChunks, Tt, Ub, n, sc);
      TK_LAUNCH_CHECK();
      TK_TRY(prod_atu(Ut, nact));
    }
    k_over_g<T><<<rows_grid(n, nact), 256, 0, st>>>(part_g, cur_splits, nact, Ub, n, sc, Tt);
    TK_LAUNCH_CHECK();
    TK_TRY(apply_prec(true, Tt, Vraw, nact, n));  // R^-T g
  } else {
    TK_TRY(prod_aw(V, nv, Tt, nullptr, nact));
    k_under_addv2<T><<<rows_grid(m, nact), 256, 0, st>>>(Tt, m, V, nv, n, sc);
    TK_LAUNCH_CHECK();
    TK_TRY(apply_prec(true, Tt, Tt, nact, m));
    k_under_ustep<T><<<nact, kVecThreads, 0, st>>>(Tt, Ut, m, sc, 0);
    TK_LAUNCH_CHECK();
    TK_TRY(apply_prec(false, Ut, Tt, nact, m));
    TK_TRY(prod_atu(Tt, nact));
    k_under_vraw<T><<<rows_grid(nv, nact), 256, 0, st>>>(part_g, cur_splits, nact, Tt, m, n, sc, Vraw);
    TK_LAUNCH_CHECK();
  }
  k_vstep<T><<<nact, kVecThreads, 0, st>>>(Vraw, V, W, Y, nv, sc, atol, btol, maxiter, 0);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

// `count` steps for `nact` active slots: launched directly (count 1, a
// profiling run, or the tensor-core products), else replayed from a graph
// captured the first time this active count is met.
template <typename T>
tk_status Lsqr<T>::steps(int nact, int count) {
  if (count <= 1 || prof_enabled() || tc) {
    for (int c = 0; c < count; ++c) TK_TRY(step(nact));
    return TK_OK;
  }
  // graphs are captured and replayed on a stream of the engine's own (the
  // caller's may be the legacy default stream, which cannot be captured),
  // ordered after the caller's stream and before its next work by events
  if (!gstream) {
    TK_CUDA(cudaStreamCreateWithFlags(&gstream, cudaStreamNonBlocking));
    TK_CUDA(cudaEventCreateWithFlags(&gev[0], cudaEventDisableTiming));
    TK_CUDA(cudaEventCreateWithFlags(&gev[1], cudaEventDisableTiming));
  }
  auto it = graphs.find(nact);
  if (it == graphs.end()) {
    cudaStream_t caller = st;
    st = gstream;
    TK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    tk_status r = TK_OK;
    for (int c = 0; c < count && r == TK_OK; ++c) r = step(nact);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    st = caller;
    if (r != TK_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (ce != cudaSuccess) {
      set_error(ce, __FILE__, __LINE__);
      return TK_ECUDA;
    }
    size_t nodes = 0;
    cudaGraphGetNodes(g, nullptr, &nodes);
    cudaGraphExec_t ge = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      set_error(ie, __FILE__, __LINE__);
      return TK_ECUDA;
    }
    it = graphs.emplace(nact, std::make_pair(ge, nodes)).first;
  }
  TK_CUDA(cudaEventRecord(gev[0], st));
  TK_CUDA(cudaStreamWaitEvent(gstream, gev[0], 0));
  TK_CUDA(cudaGraphLaunch(it->second.first, gstream));
  TK_CUDA(cudaEventRecord(gev[1], gstream));
  TK_CUDA(cudaStreamWaitEvent(st, gev[1], 0));
  count_launches(it->second.second);
  return TK_OK;
}

template <typename T>
void Lsqr<T>::release_graphs() {
  for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.first);
  graphs.clear();
  if (gstream) {
    cudaStreamSynchronize(gstream);
    cudaStreamDestroy(gstream);
    cudaEventDestroy(gev[0]);
    cudaEventDestroy(gev[1]);
    gstream = nullptr;
  }
}

// The GEMM epilogue takes a dense per-row coefficient array; Scal.coef is
// strided, so it is gathered each step.
namespace {
__global__ void k_coef(const Scal* __restrict__ sc, double* __restrict__ coef, int count) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < count) coef[s] = sc[s].coef;
}
}  // namespace

template <typename T>
tk_status Lsqr<T>::gather_coef(int count) {
  k_coef<<<cdiv(count, 128), 128, 0, st>>>(sc, coef_buf, count);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

template struct Lsqr<double>;
template struct Lsqr<float>;

}  // namespace tk
