// Dense building blocks of the path, all hand-written SIMT CUDA:
//   * GEMM / split-K GEMM   -- sketch products, Gram matrix (Algorithm 1 step 3)
//                              and the two products with A in every LSQR step
//   * batched Cholesky      -- R_i = chol(C + lambda_i I) for all lambda at once
//                              (Algorithm 1 step 4), blocked right-looking
//   * batched TRSV          -- R^-1 v and R^-T g (the preconditioner apply)
//
// FP64 on this part issues about two DFMA per clock per SM (58x below FP32),
// so every FP64 kernel here is DFMA-bound: the design goal is to keep the FP64
// pipe busy with enough resident warps, not to save bytes.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "tk_gemm_tiles.cuh"
#include "tk_internal.cuh"

namespace tk {
namespace {

using tiles::AccOf;

// C = alpha op(A) op(B) [+ beta_row[i] * Cin]     or, with `partial`, the raw
// split-K partial sum of K-range blockIdx.z into partial + z * M * N
// (tile body: tiles::gemm_tile).
template <typename TA, typename TB, typename TC, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_gemm(bool transA, bool transB, int64_t M, int64_t N, int64_t K, const TA* __restrict__ A, int64_t lda,
           const TB* __restrict__ B, int64_t ldb, TC* C, int64_t ldc, double alpha,
           const double* __restrict__ beta_row, const TC* Cin, int64_t ldcin, int64_t k_per_split,
           double* __restrict__ partial, bool upper_only) {
  __shared__ tiles::GemmSmem<TA, TB, BM, BN, BK> sm;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  // symmetric results (the Gram matrix): tiles strictly below the diagonal are skipped
  if (upper_only && m0 > n0 + BN - 1) return;
  const int64_t kbeg = (int64_t)blockIdx.z * k_per_split;
  const int64_t kend = std::min(K, kbeg + k_per_split);
  tiles::gemm_tile<TA, TB, TC, BM, BN, BK, TM, TN>(sm, transA, transB, M, N, A, lda, B, ldb, C, ldc, alpha, beta_row,
                                                   Cin, ldcin, m0, n0, kbeg, kend,
                                                   partial ? partial + (int64_t)blockIdx.z * M * N : nullptr);
}

// Lambda-major float32 products of LSQR (tile body: tiles::gemm_lm_tile): one
// column tile of 256 per blockIdx.x, K split blockIdx.y.
template <bool TRANSB, int BM, int TM>
__global__ void __launch_bounds__(256)
    k_gemm_lm(bool vec, int64_t M, int64_t N, int64_t K, const float* __restrict__ L, int64_t ldl,
              const float* __restrict__ A, int64_t lda, float* C, int64_t ldc, const double* __restrict__ beta_row,
              const float* Cin, int64_t ldcin, int64_t k_per_split, double* __restrict__ partial) {
  __shared__ __align__(16) tiles::LmSmem<BM> sm;
  const int64_t n0 = (int64_t)blockIdx.x * tiles::LM_BN;
  const int64_t kbeg = (int64_t)blockIdx.y * k_per_split;
  const int64_t kend = std::min(K, kbeg + k_per_split);
  tiles::gemm_lm_tile<TRANSB, BM, TM>(sm, vec, M, N, L, ldl, A, lda, C, ldc, beta_row, Cin, ldcin, n0, kbeg, kend,
                                      partial ? partial + (int64_t)blockIdx.y * M * N : nullptr);
}

template <typename T>
tk_status launch_gemm_lm(bool transB, int64_t M, int64_t N, int64_t K, const T* L, int64_t ldl, const T* A,
                         int64_t lda, T* C, int64_t ldc, double alpha, const double* beta_row, const T* Cin,
                         int64_t ldcin, int splits, double* partial, cudaStream_t st) {
  (void)alpha;  // callers of this path use alpha = 1
  constexpr int BN = 256;
  int64_t kps = cdiv(cdiv(K, splits), 16) * 16;
  if (kps <= 0) kps = 16;
  dim3 grid((unsigned)cdiv(N, BN), (unsigned)splits);
  if (grid.y > 65535u) {
    set_error_msg("gemm: too many K splits");
    return TK_EINVAL;
  }
  // 16-byte loads need 16-byte aligned rows
  const bool vec = ((uintptr_t)L % 16 == 0) && ((uintptr_t)A % 16 == 0) && (ldl % 4 == 0) && (lda % 4 == 0);
#define TK_LM(TRB, BM_, TM_)                                                                                  \
  k_gemm_lm<TRB, BM_, TM_><<<grid, 256, 0, st>>>(vec, M, N, K, L, ldl, A, lda, C, ldc, beta_row, Cin, ldcin, kps, \
                                                 partial)
  if (M <= 16) {
    if (transB) TK_LM(true, 16, 2); else TK_LM(false, 16, 2);
  } else if (M <= 32) {
    if (transB) TK_LM(true, 32, 4); else TK_LM(false, 32, 4);
  } else {
    if (transB) TK_LM(true, 64, 8); else TK_LM(false, 64, 8);
  }
#undef TK_LM
  TK_LAUNCH_CHECK();
  return TK_OK;
}

template <typename TA, typename TB, typename TC, int BM, int BN, int BK, int TM, int TN>
tk_status launch_gemm(bool transA, bool transB, int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda,
                      const TB* B, int64_t ldb, TC* C, int64_t ldc, double alpha, const double* beta_col,
                      const TC* Cin, int64_t ldcin, int splits, double* partial, cudaStream_t st,
                      bool upper_only = false) {
  int64_t kps = cdiv(cdiv(K, splits), BK) * BK;
  if (kps <= 0) kps = BK;
  dim3 grid((unsigned)cdiv(M, BM), (unsigned)cdiv(N, BN), (unsigned)splits);
  if (grid.y > 65535u || grid.z > 65535u) {
    set_error_msg("gemm: grid too large");
    return TK_EINVAL;
  }
  k_gemm<TA, TB, TC, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(
      transA, transB, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta_col, Cin, ldcin, kps, partial, upper_only);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

// Candidate tile shapes of the generic kernel for the lambda-row products
// (M <= 32 rows, double accumulation): the index the tuner records.
constexpr int kTuneCfgs = 5;
template <typename TA, typename TB, typename TC>
tk_status launch_cfg(int cfg, bool transA, bool transB, int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda,
                     const TB* B, int64_t ldb, TC* C, int64_t ldc, double alpha, const double* beta_row,
                     const TC* Cin, int64_t ldcin, int splits, double* partial, cudaStream_t st) {
#define TK_C(BM, BN, TM, TN)                                                                                    \
  return launch_gemm<TA, TB, TC, BM, BN, 16, TM, TN>(transA, transB, M, N, K, A, lda, B, ldb, C, ldc, alpha, \
                                                      beta_row, Cin, ldcin, splits, partial, st)
  switch (cfg) {
    case 0: TK_C(32, 128, 4, 4);
    case 1: TK_C(32, 64, 4, 2);
    case 2: TK_C(32, 32, 4, 1);
    case 3: TK_C(8, 256, 1, 8);
    default: TK_C(8, 64, 1, 2);
  }
#undef TK_C
}

template <typename TA, typename TB, typename TC>
tk_status gemm_dispatch(bool transA, bool transB, int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda,
                        const TB* B, int64_t ldb, TC* C, int64_t ldc, double alpha, const double* beta_row,
                        const TC* Cin, int64_t ldcin, int splits, double* partial, cudaStream_t st,
                        bool use_table = true) {
  if (M == 0 || N == 0) return TK_OK;
  constexpr bool f32 = std::is_same<TA, float>::value && std::is_same<TB, float>::value;
  if constexpr (!f32) {
    // a measured choice (tk_autotune) for this lambda-row shape
    if (use_table && !transA && M <= 32) {
      GemmKey key;
      key.ta = dtype_code<TA>(); key.tb = dtype_code<TB>(); key.tc = dtype_code<TC>();
      key.transA = 0; key.transB = transB ? 1 : 0; key.split = partial ? 1 : 0;
      key.M = M; key.N = N; key.K = K;
      TuneChoice ch;
      if (tune_lookup(key, &ch) && ch.cfg >= 0)
        return launch_cfg<TA, TB, TC>(ch.cfg, transA, transB, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta_row, Cin,
                                      ldcin, splits, partial, st);
    }
  }
  if constexpr (f32) {
    // the lambda-major products of LSQR (all active lambda in one tile)
    if (!transA && M <= 64 && N >= 256 && alpha == 1.0) {
      if (partial)
        return launch_gemm_lm<float>(transB, M, N, K, A, lda, B, ldb, nullptr, 0, alpha, nullptr, nullptr, 0, splits,
                                     partial, st);
      if constexpr (std::is_same<TC, float>::value)
        return launch_gemm_lm<float>(transB, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta_row, Cin, ldcin, splits,
                                     nullptr, st);
    }
  }
#define TK_G(BM, BN, TM, TN)                                                                                    \
  return launch_gemm<TA, TB, TC, BM, BN, 16, TM, TN>(transA, transB, M, N, K, A, lda, B, ldb, C, ldc, alpha, \
                                                      beta_row, Cin, ldcin, splits, partial, st)
  // Shapes: a few lambda rows against a long axis (M small), a long axis
  // against a few lambda columns (N small), or square-ish.  Few CTAs (a
  // small problem: fewer than one per SM) take the narrower column tile.
  const bool few = cdiv(N, 128) * (int64_t)splits < 152;
  if (!f32 && few) {
    if (M <= 8) TK_G(8, 64, 1, 2);
    if (M <= 32) TK_G(32, 32, 4, 1);
  }
  if (f32) {
    if (M <= 32) TK_G(32, 128, 4, 4);
    if (M <= 64) TK_G(64, 128, 8, 4);
    if (N <= 32) TK_G(128, 32, 8, 2);
    TK_G(128, 64, 8, 4);
  }
  if (M <= 8) TK_G(8, 256, 1, 8);
  if (M <= 32) TK_G(32, 128, 4, 4);
  if (N <= 8) TK_G(256, 8, 8, 1);
  if (N <= 32) TK_G(128, 32, 4, 4);
  TK_G(64, 64, 4, 4);
#undef TK_G
}

// ------------------------------------------------------------- Cholesky ---
constexpr int CB = 64;  // Cholesky tile

// R_l[i, j] = C[i, j] + lambda_l delta_ij on the n x n block (upper triangle),
// identity on the padding, zero below the diagonal.
__global__ void k_chol_init(const double* __restrict__ Cm, int64_t n, int64_t np, const double* __restrict__ lam,
                            double* __restrict__ R, int64_t ldr, int64_t rstride, int* __restrict__ info) {
  const int l = blockIdx.y;
  double* Rl = R + (int64_t)l * rstride;
  const double lv = lam[l];
  if (blockIdx.x == 0 && threadIdx.x == 0) info[l] = 0;
  int64_t total = np * np;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = k / np, j = k - i * np;
    double v = 0.0;
    if (j >= i) {
      if (i < n && j < n) v = Cm[i * n + j] + (i == j ? lv : 0.0);
      else v = (i == j) ? 1.0 : 0.0;
    }
    Rl[i * ldr + j] = v;
  }
}

// Factor the diagonal tile (kb, kb) of every lambda in shared memory
// (right-looking within the tile).  A non-positive pivot records the global
// row + 1 in info[l] (first one only; its negative when the pivot is NaN, i.e.
// non-finite input rather than a matrix that is not positive definite) and
// continues with pivot 1.
__global__ void __launch_bounds__(256) k_chol_diag(double* __restrict__ R, int64_t ldr, int64_t rstride, int kb,
                                                   int* __restrict__ info) {
  __shared__ double T[CB][CB + 1];
  const int l = blockIdx.x;
  double* Rl = R + (int64_t)l * rstride + (int64_t)kb * CB * ldr + (int64_t)kb * CB;
  for (int idx = threadIdx.x; idx < CB * CB; idx += blockDim.x) {
    int i = idx / CB, j = idx % CB;
    T[i][j] = Rl[(int64_t)i * ldr + j];
  }
  __syncthreads();
  for (int j = 0; j < CB; ++j) {
    if (threadIdx.x == 0) {
      double d = T[j][j];
      if (!(d > 0.0)) {
        if (info[l] == 0) info[l] = (d != d) ? -(kb * CB + j + 1) : kb * CB + j + 1;
        d = 1.0;
      }
      T[j][j] = sqrt(d);
    }
    __syncthreads();
    const double rjj = T[j][j];
    for (int k = j + 1 + threadIdx.x; k < CB; k += blockDim.x) T[j][k] /= rjj;
    __syncthreads();
    // trailing update of the upper triangle: T[i][k] -= T[j][i] T[j][k], j < i <= k
    const int rem = CB - j - 1;
    for (int p = threadIdx.x; p < rem * rem; p += blockDim.x) {
      int i = j + 1 + p / rem, k = j + 1 + p % rem;
      if (k >= i) T[i][k] -= T[j][i] * T[j][k];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < CB * CB; idx += blockDim.x) {
    int i = idx / CB, j = idx % CB;
    if (j >= i) Rl[(int64_t)i * ldr + j] = T[i][j];
  }
}

// Row panel: tile (kb, jb), jb > kb, becomes R_kk^-T tile (forward
// substitution; one column of the tile per thread, held in registers).  The
// 64 reciprocals of the diagonal are formed once per tile (thread r forms
// 1/D[r][r]): GB300's float64 division is slow, and every column would
// otherwise divide by each of them.
__global__ void __launch_bounds__(CB) k_chol_trsm(double* __restrict__ R, int64_t ldr, int64_t rstride, int kb) {
  __shared__ double D[CB][CB + 1];
  __shared__ double Dinv[CB];
  const int l = blockIdx.y;
  const int jb = kb + 1 + blockIdx.x;
  double* Rl = R + (int64_t)l * rstride;
  const double* Dg = Rl + (int64_t)kb * CB * ldr + (int64_t)kb * CB;
  double* Xg = Rl + (int64_t)kb * CB * ldr + (int64_t)jb * CB;
  const int c = threadIdx.x;
  double xr[CB];
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    D[i][c] = Dg[(int64_t)i * ldr + c];
    xr[i] = Xg[(int64_t)i * ldr + c];
  }
  Dinv[c] = 1.0 / Dg[(int64_t)c * ldr + c];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < CB; ++r) {
    xr[r] = xr[r] * Dinv[r];
#pragma unroll
    for (int q = r + 1; q < CB; ++q) xr[q] = fma(-D[r][q], xr[r], xr[q]);
  }
#pragma unroll
  for (int i = 0; i < CB; ++i) Xg[(int64_t)i * ldr + c] = xr[i];
}

// Trailing update of tiles (ib, jb), kb < ib <= jb:
// T[ib, jb] -= R[kb, ib]^T R[kb, jb].  One CTA per (tile pair, lambda).
__global__ void __launch_bounds__(256) k_chol_update(double* __restrict__ R, int64_t ldr, int64_t rstride, int kb,
                                                     int nt) {
  constexpr int KC = 16;
  __shared__ double P[KC][CB + 1];  // rows of R[kb, ib]
  __shared__ double Q[KC][CB + 1];  // rows of R[kb, jb]
  const int l = blockIdx.y;
  // decode the linear tile-pair index into (ib, jb) with ib <= jb
  const int r = nt - kb - 1;
  int t = blockIdx.x, ib = 0;
  {
    int row_len = r;
    while (t >= row_len) {
      t -= row_len;
      --row_len;
      ++ib;
    }
  }
  int jb = ib + t;
  ib += kb + 1;
  jb += kb + 1;
  double* Rl = R + (int64_t)l * rstride;
  const double* Pg = Rl + (int64_t)kb * CB * ldr + (int64_t)ib * CB;
  const double* Qg = Rl + (int64_t)kb * CB * ldr + (int64_t)jb * CB;
  double* Tg = Rl + (int64_t)ib * CB * ldr + (int64_t)jb * CB;
  // thread owns a 4 x 4 block of the 64 x 64 output
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int kc = 0; kc < CB; kc += KC) {
    for (int idx = threadIdx.x; idx < KC * CB; idx += blockDim.x) {
      int k = idx / CB, j = idx % CB;
      P[k][j] = Pg[(int64_t)(kc + k) * ldr + j];
      Q[k][j] = Qg[(int64_t)(kc + k) * ldr + j];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      double pa[4], qb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) pa[a] = P[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) qb[b] = Q[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(pa[a], qb[b], acc[a][b]);
    }
    __syncthreads();
  }
  const bool diag = (ib == jb);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = ty + 16 * a, j = tx + 16 * b;
      if (diag && j < i) continue;
      Tg[(int64_t)i * ldr + j] -= acc[a][b];
    }
}

// --------------------------------------------------- triangular inverse ---
// M = R^-1 of the upper triangular factors as an explicit preconditioner (in
// float32 for the float32 LSQR of the mixed form, in float64 for small
// factors of the float64 form): every application of R^-1 or R^-T is then
// one batched triangular matrix-vector product (HBM-bound, one launch)
// instead of a substitution (a chain of dependent launches).  Blocks of 64 rows are finished from the bottom: R M = I gives
// M_ii = R_ii^-1 (float64, in shared memory) and, for c > i,
// M_ic = M_ii S_ic with S_ic = -sum_{i<k<=c} R_ik M_kc, accumulated
// right-looking in the not yet finished blocks of M (zero on entry).  Mt
// receives M^T (its blocks above the diagonal are left unwritten).

// M_kk = R_kk^-1: thread c back-substitutes column c of the identity.
template <typename T>
__global__ void __launch_bounds__(CB) k_tinv_diag(const double* __restrict__ R, int64_t ldr, int64_t rstride,
                                                  T* __restrict__ M, T* __restrict__ Mt, int64_t ldm,
                                                  int64_t mstride) {
  __shared__ double D[CB][CB + 1];
  const int kb = blockIdx.x, l = blockIdx.y, c = threadIdx.x;
  const double* Rg = R + (int64_t)l * rstride + (int64_t)kb * CB * ldr + (int64_t)kb * CB;
  for (int i = 0; i < CB; ++i) D[i][c] = Rg[(int64_t)i * ldr + c];
  __syncthreads();
  double x[CB];
#pragma unroll
  for (int r = 0; r < CB; ++r) x[r] = (r == c) ? 1.0 : 0.0;
#pragma unroll
  for (int r = CB - 1; r >= 0; --r) {
    x[r] = x[r] / D[r][r];
#pragma unroll
    for (int q = 0; q < r; ++q) x[q] = fma(-D[q][r], x[r], x[q]);
  }
  __syncthreads();
  T* Mg = M + (int64_t)l * mstride + (int64_t)kb * CB * ldm + (int64_t)kb * CB;
#pragma unroll
  for (int r = 0; r < CB; ++r) {
    Mg[(int64_t)r * ldm + c] = (T)x[r];
    D[r][c] = x[r];
  }
  __syncthreads();
  T* Mtg = Mt + (int64_t)l * mstride + (int64_t)kb * CB * ldm + (int64_t)kb * CB;
  for (int i = 0; i < CB; ++i) Mtg[(int64_t)i * ldm + c] = (T)D[c][i];
}

// S_{rb,cb} -= R_{rb,k} M_{k,cb} for rb < k <= cb (arithmetic in T; R read as float64).
template <typename T>
__global__ void __launch_bounds__(256) k_tinv_update(const double* __restrict__ R, int64_t ldr, int64_t rstride,
                                                     T* __restrict__ M, int64_t ldm, int64_t mstride, int k,
                                                     int nt) {
  constexpr int KC = 32;
  __shared__ T P[KC][CB + 4];  // P[kk][i] = R[rb*64 + i, k*64 + kc + kk]
  __shared__ T Q[KC][CB];      // Q[kk][j] = M[k*64 + kc + kk, cb*64 + j]
  const int l = blockIdx.y;
  const int rb = blockIdx.x / (nt - k), cb = k + blockIdx.x % (nt - k);
  const double* Pg = R + (int64_t)l * rstride + (int64_t)rb * CB * ldr + (int64_t)k * CB;
  T* Ml = M + (int64_t)l * mstride;
  const T* Qg = Ml + (int64_t)k * CB * ldm + (int64_t)cb * CB;
  T* Sg = Ml + (int64_t)rb * CB * ldm + (int64_t)cb * CB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4] = {};
  for (int kc = 0; kc < CB; kc += KC) {
    for (int idx = threadIdx.x; idx < KC * CB; idx += blockDim.x) {
      const int i = idx / KC, kk = idx % KC;
      P[kk][i] = (T)Pg[(int64_t)i * ldr + kc + kk];
      const int q = idx / CB, j = idx % CB;
      Q[q][j] = Qg[(int64_t)(kc + q) * ldm + j];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T pa[4], qb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) pa[a] = P[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) qb[b] = Q[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(pa[a], qb[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) Sg[(int64_t)(ty + 16 * a) * ldm + tx + 16 * b] -= acc[a][b];
}

// M_{i,cb} = M_{i,i} S_{i,cb} for cb > i (in place: every read of the tile
// precedes the barrier, every write follows it), and Mt_{cb,i} = M_{i,cb}^T.
template <typename T>
__global__ void __launch_bounds__(256) k_tinv_final(T* __restrict__ M, T* __restrict__ Mt, int64_t ldm,
                                                    int64_t mstride, int i) {
  __shared__ T D[CB][CB + 1];
  const int l = blockIdx.y, cb = i + 1 + blockIdx.x;
  T* Ml = M + (int64_t)l * mstride;
  const T* Dg = Ml + (int64_t)i * CB * ldm + (int64_t)i * CB;
  T* Sg = Ml + (int64_t)i * CB * ldm + (int64_t)cb * CB;
  for (int idx = threadIdx.x; idx < CB * CB; idx += blockDim.x) {
    const int r = idx / CB, c = idx % CB;
    D[r][c] = Dg[(int64_t)r * ldm + c];
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4] = {};
#pragma unroll 8
  for (int kk = 0; kk < CB; ++kk) {
    T da[4], sb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) da[a] = D[ty + 16 * a][kk];
#pragma unroll
    for (int b = 0; b < 4; ++b) sb[b] = Sg[(int64_t)kk * ldm + tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(da[a], sb[b], acc[a][b]);
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      Sg[(int64_t)(ty + 16 * a) * ldm + tx + 16 * b] = acc[a][b];
      D[ty + 16 * a][tx + 16 * b] = acc[a][b];
    }
  __syncthreads();
  T* Mtg = Mt + (int64_t)l * mstride + (int64_t)cb * CB * ldm + (int64_t)i * CB;
  for (int idx = threadIdx.x; idx < CB * CB; idx += blockDim.x) {
    const int r = idx / CB, c = idx % CB;
    Mtg[(int64_t)r * ldm + c] = D[c][r];
  }
}

// ------------------------------------------------------------------ TRMV --
template <typename T, bool UPPER>
__global__ void __launch_bounds__(256) k_trmv(int64_t n, const T* __restrict__ M, int64_t ldm, int64_t mstride,
                                              const int* __restrict__ idx, const T* in, T* out, int64_t ldx) {
  extern __shared__ float4 trmv_v4[];
  const int slot = blockIdx.y;
  tiles::trmv_rows<T, UPPER>(n, M + (int64_t)(idx ? idx[slot] : slot) * mstride, ldm, in + (int64_t)slot * ldx,
                             out + (int64_t)slot * ldx, (int64_t)blockIdx.x * tiles::kTrmvRows, trmv_v4);
}

// ------------------------------------------------------------------ TRSV --
constexpr int kTrsvThreads = 256;

// x <- R^-1 x (back substitution) for each slot, R upper triangular.
// Blocks of 32 rows from the bottom: the 8 warps first subtract the solved
// part (row i of R against the solved tail, one warp per row), then warp 0
// solves the 32 x 32 diagonal block with shuffles.
template <typename TR, typename TX>
__global__ void __launch_bounds__(kTrsvThreads)
    k_trsv_upper(int64_t n, const TR* __restrict__ R, int64_t ldr, int64_t rstride, const int* __restrict__ idx,
                 const TX* Xin, TX* X, int64_t ldx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* x = reinterpret_cast<double*>(smem_raw);
  const int slot = blockIdx.x;
  const TR* Rs = R + (int64_t)(idx ? idx[slot] : slot) * rstride;
  TX* xg = X + (int64_t)slot * ldx;
  const TX* xin = Xin + (int64_t)slot * ldx;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = (double)xin[i];
  __syncthreads();
  const int64_t nb = cdiv(n, 32);
  for (int64_t b = nb - 1; b >= 0; --b) {
    const int64_t r0 = b * 32, r1 = std::min<int64_t>(n, r0 + 32);
    for (int64_t i = r0 + wid; i < r1; i += nw) {
      double acc = 0.0;
      for (int64_t k = r1 + lane; k < n; k += 32) acc = fma((double)Rs[i * ldr + k], x[k], acc);
      acc = warp_sum(acc);
      if (lane == 0) x[i] -= acc;
    }
    __syncthreads();
    if (wid == 0) {
      int64_t i = r0 + lane;
      bool live = i < r1;
      double xi = live ? x[i] : 0.0;
      for (int q = (int)(r1 - r0) - 1; q >= 0; --q) {
        double rq = live ? (double)Rs[i * ldr + r0 + q] : 0.0;  // R[i, r0+q]
        double xq = __shfl_sync(0xffffffffu, xi, q);
        if (lane == q) {
          xq = xq / rq;
          xi = xq;
        }
        xq = __shfl_sync(0xffffffffu, xi, q);
        if (lane < q) xi = fma(-rq, xq, xi);
      }
      if (live) x[i] = xi;
    }
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xg[i] = (TX)x[i];
}

// x <- R^-T x (forward substitution with the lower triangular R^T).
// Block b of 32 unknowns first receives -sum_{k < r0} R[k, i] x_k: warps take
// rows k, lanes take the 32 columns i (coalesced), partials meet in shared
// memory; then warp 0 solves the diagonal block.
template <typename TR, typename TX>
__global__ void __launch_bounds__(kTrsvThreads)
    k_trsv_upper_t(int64_t n, const TR* __restrict__ R, int64_t ldr, int64_t rstride, const int* __restrict__ idx,
                   const TX* Xin, TX* X, int64_t ldx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* x = reinterpret_cast<double*>(smem_raw);
  __shared__ double part[kTrsvThreads / 32][32];
  const int slot = blockIdx.x;
  const TR* Rs = R + (int64_t)(idx ? idx[slot] : slot) * rstride;
  TX* xg = X + (int64_t)slot * ldx;
  const TX* xin = Xin + (int64_t)slot * ldx;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = (double)xin[i];
  __syncthreads();
  const int64_t nb = cdiv(n, 32);
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t r0 = b * 32, r1 = std::min<int64_t>(n, r0 + 32);
    const int64_t i = r0 + lane;
    const bool live = i < r1;
    double acc = 0.0;
    for (int64_t k = wid; k < r0; k += nw)
      if (live) acc = fma((double)Rs[k * ldr + i], x[k], acc);
    part[wid][lane] = acc;
    __syncthreads();
    if (wid == 0) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += part[w][lane];
      double xi = live ? x[i] - s : 0.0;
      for (int q = 0; q < (int)(r1 - r0); ++q) {
        double rq = live ? (double)Rs[(r0 + q) * ldr + i] : 0.0;  // R[r0+q, i]
        double xq = __shfl_sync(0xffffffffu, xi, q);
        if (lane == q) {
          xq = xq / rq;
          xi = xq;
        }
        xq = __shfl_sync(0xffffffffu, xi, q);
        if (lane > q) xi = fma(-rq, xq, xi);
      }
      if (live) x[i] = xi;
    }
    __syncthreads();
  }
  for (int64_t i2 = threadIdx.x; i2 < n; i2 += blockDim.x) xg[i2] = (TX)x[i2];
}

// ---- column-sweep solves across the grid ---------------------------------
// The remaining right-hand side P (float64, one row of n per slot) starts as
// the input vector.  Launch b solves the 32 x 32 diagonal block b from P (every
// CTA of the slot does it redundantly; CTA 0 stores x_b), then each CTA folds
// x_b into P for its share of the unsolved rows.  No CTA waits on another; the
// launches of one solve are ordered by the stream.
constexpr int kSweepRows = 256;  // unsolved rows per CTA

template <typename TX>
__global__ void k_sweep_init(const TX* __restrict__ Xin, int64_t ldx, int64_t n, TX* __restrict__ P) {
  const int s = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    P[(int64_t)s * n + i] = Xin[(int64_t)s * ldx + i];
}

// Arithmetic runs in the vector's type TX (float64 is ~58x slower than float32
// on this part, so the float32 path must not widen).  The dependent chain of
// the 32 x 32 diagonal solve multiplies by reciprocals computed up front.

// upper: x = R^-1 v, step for diagonal block b (rows r0..r1); updates rows < r0
template <typename TR, typename TX>
__global__ void __launch_bounds__(kTrsvThreads)
    k_sweep_upper(int64_t n, const TR* __restrict__ R, int64_t ldr, int64_t rstride, const int* __restrict__ idx,
                  TX* __restrict__ X, int64_t ldx, TX* __restrict__ P, int64_t b, int rows_per_cta) {
  __shared__ TX xs[32];
  const int slot = blockIdx.y;
  const TR* Rs = R + (int64_t)(idx ? idx[slot] : slot) * rstride;
  TX* p = P + (int64_t)slot * n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t r0 = b * 32, r1 = std::min<int64_t>(n, r0 + 32);
  const int cols = (int)(r1 - r0);
  if (wid == 0) {
    const int64_t i = r0 + lane;
    const bool live = lane < cols;
    TX rr[32];  // row i of the diagonal block, loaded up front
#pragma unroll
    for (int q = 0; q < 32; ++q) rr[q] = (live && q < cols) ? (TX)Rs[i * ldr + r0 + q] : TX(0);
    const TX rinv = live ? TX(1) / (TX)Rs[i * ldr + i] : TX(0);
    TX xi = live ? p[i] : TX(0);
#pragma unroll
    for (int q = 31; q >= 0; --q) {
      if (q < cols) {
        TX xq = __shfl_sync(0xffffffffu, xi, q);
        if (lane == q) xi = xq * rinv;
        xq = __shfl_sync(0xffffffffu, xi, q);
        if (lane < q) xi = fma(-rr[q], xq, xi);
      }
    }
    xs[lane] = live ? xi : TX(0);
    if (blockIdx.x == 0 && live) X[(int64_t)slot * ldx + i] = xi;
  }
  __syncthreads();
  const int64_t beg = (int64_t)blockIdx.x * rows_per_cta, end = std::min<int64_t>(r0, beg + rows_per_cta);
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const TR* row = Rs + i * ldr + r0;
    TX acc = TX(0);
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if (k < cols) acc = fma((TX)row[k], xs[k], acc);
    p[i] -= acc;
  }
}

// transposed: x = R^-T v, step for diagonal block b; updates rows >= r1
template <typename TR, typename TX>
__global__ void __launch_bounds__(kTrsvThreads)
    k_sweep_lower(int64_t n, const TR* __restrict__ R, int64_t ldr, int64_t rstride, const int* __restrict__ idx,
                  TX* __restrict__ X, int64_t ldx, TX* __restrict__ P, int64_t b, int rows_per_cta) {
  __shared__ TX xs[32];
  const int slot = blockIdx.y;
  const TR* Rs = R + (int64_t)(idx ? idx[slot] : slot) * rstride;
  TX* p = P + (int64_t)slot * n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t r0 = b * 32, r1 = std::min<int64_t>(n, r0 + 32);
  const int cols = (int)(r1 - r0);
  if (wid == 0) {
    const int64_t i = r0 + lane;
    const bool live = lane < cols;
    TX rr[32];  // column i of the diagonal block (row i of R^T), loaded up front
#pragma unroll
    for (int q = 0; q < 32; ++q) rr[q] = (live && q < cols) ? (TX)Rs[(r0 + q) * ldr + i] : TX(0);
    const TX rinv = live ? TX(1) / (TX)Rs[i * ldr + i] : TX(0);
    TX xi = live ? p[i] : TX(0);
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      if (q < cols) {
        TX xq = __shfl_sync(0xffffffffu, xi, q);
        if (lane == q) xi = xq * rinv;
        xq = __shfl_sync(0xffffffffu, xi, q);
        if (lane > q) xi = fma(-rr[q], xq, xi);
      }
    }
    xs[lane] = live ? xi : TX(0);
    if (blockIdx.x == 0 && live) X[(int64_t)slot * ldx + i] = xi;
  }
  __syncthreads();
  const int64_t beg = r1 + (int64_t)blockIdx.x * rows_per_cta, end = std::min<int64_t>(n, beg + rows_per_cta);
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    TX acc = TX(0);
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if (k < cols) acc = fma((TX)Rs[(r0 + k) * ldr + i], xs[k], acc);
    p[i] -= acc;
  }
}

}  // namespace

// ----------------------------------------------------------- host side ----
// C (c x c) = Y^T Y (Y r x c), upper triangle (and the diagonal tiles) only.
// C[i][j] = sum_z partial[z][i][j] on the upper triangle (j >= i)
__global__ void k_gram_reduce(const double* __restrict__ part, int splits, int64_t c, double* __restrict__ C) {
  const int64_t total = c * c;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / c, j = k - i * c;
    if (j < i) continue;
    double acc = 0.0;
    for (int z = 0; z < splits; ++z) acc += part[(int64_t)z * total + k];
    C[k] = acc;
  }
}

size_t gram_scratch_bytes(int64_t r, int64_t c) {
  const int64_t nt = cdiv(c, 64), upper = nt * (nt + 1) / 2;
  if (upper >= 152) return 0;
  const int64_t splits = std::max<int64_t>(1, std::min<int64_t>(cdiv(2 * 152, upper), r / 64));
  return splits > 1 ? sizeof(double) * (size_t)splits * c * c : 0;
}

tk_status gram_upper(const double* Y, int64_t r, int64_t c, double* C, void* scratch, size_t scratch_bytes,
                     cudaStream_t st) {
  if (c <= 0) return TK_OK;
  // few output tiles (a small n): split the sum over the r rows of Y
  const int64_t total = c * c;
  const size_t want = gram_scratch_bytes(r, c);
  const int splits = (scratch && want > 0 && scratch_bytes >= want) ? (int)(want / (sizeof(double) * total)) : 1;
  if (splits < 2) {
    return launch_gemm<double, double, double, 64, 64, 16, 4, 4>(true, false, c, c, r, Y, c, Y, c, C, c, 1.0,
                                                                  nullptr, nullptr, 0, 1, nullptr, st, true);
  }
  double* part = static_cast<double*>(scratch);
  TK_TRY((launch_gemm<double, double, double, 64, 64, 16, 4, 4>(true, false, c, c, r, Y, c, Y, c, nullptr, 0, 1.0,
                                                                 nullptr, nullptr, 0, splits, part, st, true)));
  k_gram_reduce<<<(unsigned)std::min<int64_t>(cdiv(total, 256), 152 * 8), 256, 0, st>>>(part, splits, c, C);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

template <typename TA, typename TB, typename TC>
tk_status gemm(bool transA, bool transB, int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda, const TB* B,
               int64_t ldb, TC* C, int64_t ldc, double alpha, const double* beta_col, const TC* Cin, int64_t ldcin,
               cudaStream_t st) {
  return gemm_dispatch<TA, TB, TC>(transA, transB, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta_col, Cin, ldcin, 1,
                                   nullptr, st);
}

int splitk_count(int64_t M, int64_t N, int64_t K) {
  int64_t tiles = cdiv(M, 32) * cdiv(N, 256);
  int64_t want = cdiv(152 * 4, std::max<int64_t>(tiles, 1));
  int64_t maxs = std::max<int64_t>(1, K / 64);  // at least 64 rows of K per split
  return (int)std::max<int64_t>(1, std::min<int64_t>({want, maxs, 4096}));
}

template <typename TA, typename TB>
int splitk_tuned(int64_t M, int64_t N, int64_t K, int cap) {
  GemmKey key;
  key.ta = dtype_code<TA>(); key.tb = dtype_code<TB>(); key.tc = 1;
  key.split = 1;
  key.M = M; key.N = N; key.K = K;
  TuneChoice ch;
  if (tune_lookup(key, &ch) && ch.splits > 0) return std::min(ch.splits, cap);
  return cap;
}
template int splitk_tuned<double, double>(int64_t, int64_t, int64_t, int);
template int splitk_tuned<double, float>(int64_t, int64_t, int64_t, int);
template int splitk_tuned<float, float>(int64_t, int64_t, int64_t, int);

template <typename TA, typename TB, typename TC>
tk_status tune_gemm(bool transA, bool transB, int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda, const TB* B,
                    int64_t ldb, TC* C, int64_t ldc, double alpha, const double* beta_row, const TC* Cin,
                    int64_t ldcin, int split_cap, double* partial, cudaStream_t st) {
  if (M == 0 || N == 0 || K == 0) return TK_OK;
  constexpr bool f32 = std::is_same<TA, float>::value && std::is_same<TB, float>::value;
  std::vector<int> cfgs;
  if (!f32 && !transA && M <= 32) {
    for (int c = 0; c < kTuneCfgs; ++c)
      if (c < 3 || M <= 8) cfgs.push_back(c);
  } else {
    cfgs.push_back(-1);  // the fixed rule's tile (the lambda-major float32 kernel sizes its tile by M)
  }
  std::vector<int> sps{1};
  if (partial) {
    sps.assign(1, std::max(split_cap, 1));
    for (int q = split_cap / 2; q >= 1 && sps.size() < 3; q /= 2) sps.push_back(q);
  }
  // candidates: (tile configuration, split count); index 0 is the fixed rule
  std::vector<std::pair<int, int>> cand;
  cand.push_back({-1, sps[0]});
  for (int cfg : cfgs)
    for (int sp : sps)
      if (!(cfg == -1 && sp == sps[0])) cand.push_back({cfg, sp});
  cudaEvent_t e0, e1;
  TK_CUDA(cudaEventCreate(&e0));
  TK_CUDA(cudaEventCreate(&e1));
  std::vector<float> best(cand.size(), 1e30f);
  tk_status err = TK_OK;
  auto run = [&](int cfg, int sp) -> tk_status {
    if (cfg >= 0) {
      if constexpr (!f32)
        return launch_cfg<TA, TB, TC>(cfg, transA, transB, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta_row, Cin,
                                      ldcin, sp, partial, st);
    }
    return gemm_dispatch<TA, TB, TC>(transA, transB, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta_row, Cin, ldcin,
                                     sp, partial, st, false);
  };
  // three interleaved rounds over all candidates (clock drift hits every
  // candidate alike); each candidate keeps its fastest of two launches
  for (int round = 0; round < 3 && err == TK_OK; ++round) {
    for (size_t c = 0; c < cand.size() && err == TK_OK; ++c) {
      if (round == 0) err = run(cand[c].first, cand[c].second);  // warm-up
      for (int r = 0; r < 2 && err == TK_OK; ++r) {
        cudaEventRecord(e0, st);
        err = run(cand[c].first, cand[c].second);
        cudaEventRecord(e1, st);
        if (err == TK_OK && cudaEventSynchronize(e1) == cudaSuccess) {
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          best[c] = std::min(best[c], ms);
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != TK_OK) return err;
  // keep the fixed rule unless a candidate is at least 3 % faster
  size_t win = 0;
  for (size_t c = 1; c < cand.size(); ++c)
    if (best[c] < best[win]) win = c;
  if (best[win] > 0.97f * best[0]) win = 0;
  TuneChoice bc;
  bc.cfg = win == 0 ? -1 : cand[win].first;
  bc.splits = partial ? cand[win].second : 0;
  GemmKey key;
  key.ta = dtype_code<TA>(); key.tb = dtype_code<TB>(); key.tc = dtype_code<TC>();
  key.transA = transA ? 1 : 0; key.transB = transB ? 1 : 0; key.split = partial ? 1 : 0;
  key.M = M; key.N = N; key.K = K;
  tune_store(key, bc);
  return TK_OK;
}
template tk_status tune_gemm<double, double, double>(bool, bool, int64_t, int64_t, int64_t, const double*, int64_t,
                                                     const double*, int64_t, double*, int64_t, double, const double*,
                                                     const double*, int64_t, int, double*, cudaStream_t);
template tk_status tune_gemm<double, float, double>(bool, bool, int64_t, int64_t, int64_t, const double*, int64_t,
                                                    const float*, int64_t, double*, int64_t, double, const double*,
                                                    const double*, int64_t, int, double*, cudaStream_t);
template tk_status tune_gemm<float, float, double>(bool, bool, int64_t, int64_t, int64_t, const float*, int64_t,
                                                   const float*, int64_t, double*, int64_t, double, const double*,
                                                   const double*, int64_t, int, double*, cudaStream_t);

template <typename TA, typename TB>
tk_status gemm_splitk(bool transA, bool transB, int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda,
                      const TB* B, int64_t ldb, double* partial, int splits, cudaStream_t st) {
  return gemm_dispatch<TA, TB, double>(transA, transB, M, N, K, A, lda, B, ldb, nullptr, 0, 1.0, nullptr, nullptr,
                                       0, splits, partial, st);
}

#define TK_INST_GEMM(TA, TB, TC)                                                                            \
  template tk_status gemm<TA, TB, TC>(bool, bool, int64_t, int64_t, int64_t, const TA*, int64_t, const TB*, \
                                      int64_t, TC*, int64_t, double, const double*, const TC*, int64_t,      \
                                      cudaStream_t);
TK_INST_GEMM(double, double, double)
TK_INST_GEMM(float, float, float)
TK_INST_GEMM(float, float, double)
TK_INST_GEMM(float, double, double)
TK_INST_GEMM(double, float, float)
TK_INST_GEMM(double, float, double)
#undef TK_INST_GEMM
template tk_status gemm_splitk<double, double>(bool, bool, int64_t, int64_t, int64_t, const double*, int64_t,
                                               const double*, int64_t, double*, int, cudaStream_t);
template tk_status gemm_splitk<float, float>(bool, bool, int64_t, int64_t, int64_t, const float*, int64_t,
                                             const float*, int64_t, double*, int, cudaStream_t);
template tk_status gemm_splitk<float, double>(bool, bool, int64_t, int64_t, int64_t, const float*, int64_t,
                                              const double*, int64_t, double*, int, cudaStream_t);
template tk_status gemm_splitk<double, float>(bool, bool, int64_t, int64_t, int64_t, const double*, int64_t,
                                              const float*, int64_t, double*, int, cudaStream_t);

template <typename T>
tk_status tri_inverse(const double* R, int64_t n, int64_t ldr, int64_t rstride, int N, T* M, T* Mt, cudaStream_t st) {
  if (N == 0 || n == 0) return TK_OK;
  const int64_t np = cdiv(n, CB) * CB;
  const int nt = (int)(np / CB);
  TK_CUDA(cudaMemsetAsync(M, 0, sizeof(T) * (size_t)N * np * np, st));
  k_tinv_diag<T><<<dim3((unsigned)nt, (unsigned)N), CB, 0, st>>>(R, ldr, rstride, M, Mt, np, np * np);
  TK_LAUNCH_CHECK();
  for (int k = nt - 1; k >= 1; --k) {
    k_tinv_update<T><<<dim3((unsigned)(k * (nt - k)), (unsigned)N), 256, 0, st>>>(R, ldr, rstride, M, np, np * np,
                                                                                 k, nt);
    TK_LAUNCH_CHECK();
    k_tinv_final<T><<<dim3((unsigned)(nt - k), (unsigned)N), 256, 0, st>>>(M, Mt, np, np * np, k - 1);
    TK_LAUNCH_CHECK();
  }
  return TK_OK;
}
template tk_status tri_inverse<float>(const double*, int64_t, int64_t, int64_t, int, float*, float*, cudaStream_t);
template tk_status tri_inverse<double>(const double*, int64_t, int64_t, int64_t, int, double*, double*, cudaStream_t);

template <typename T>
tk_status trmv_batched(bool transposed, int64_t n, const T* M, const T* Mt, int64_t ldm, int64_t mstride,
                       const int* idx, const T* in, T* out, int64_t ldx, int count, cudaStream_t st) {
  if (count == 0 || n == 0) return TK_OK;
  const dim3 grid((unsigned)cdiv(n, tiles::kTrmvRows), (unsigned)count);
  const size_t smem = tiles::trmv_smem_bytes<T>(n);
  if (!transposed) k_trmv<T, true><<<grid, 256, smem, st>>>(n, M, ldm, mstride, idx, in, out, ldx);
  else k_trmv<T, false><<<grid, 256, smem, st>>>(n, Mt, ldm, mstride, idx, in, out, ldx);
  TK_LAUNCH_CHECK();
  return TK_OK;
}
template tk_status trmv_batched<float>(bool, int64_t, const float*, const float*, int64_t, int64_t, const int*,
                                       const float*, float*, int64_t, int, cudaStream_t);
template tk_status trmv_batched<double>(bool, int64_t, const double*, const double*, int64_t, int64_t, const int*,
                                        const double*, double*, int64_t, int, cudaStream_t);

size_t chol_workspace(int64_t n, int N) {
  Arena a;
  a.take<double>((size_t)N);
  a.take<int>((size_t)N);
  return a.used + 512;
}

// R: N matrices of padded order np = ceil(n/64)*64, row stride ldr >= np,
// matrix stride rstride.  lambdas_dev: device N.  info_dev: device N.
tk_status chol_shifted(const double* Cm, int64_t n, const double* lambdas_dev, int N, double* R, int64_t ldr,
                       int64_t rstride, int* info_dev, Arena& ar, cudaStream_t st, const OzCholPlan* oz) {
  (void)ar;
  if (N == 0 || n == 0) return TK_OK;
  const int64_t np = cdiv(n, CB) * CB;
  const int nt = (int)(np / CB);
  dim3 gi((unsigned)std::min<int64_t>(cdiv(np * np, 256), 4096), (unsigned)N);
  k_chol_init<<<gi, 256, 0, st>>>(Cm, n, np, lambdas_dev, R, ldr, rstride, info_dev);
  TK_LAUNCH_CHECK();
  for (int kb = 0; kb < nt; ++kb) {
    const int r = nt - kb - 1;
    // with the update on the tensor cores the caller leaves the timing to this loop: the diagonal
    // block and the panel solve are CHOLESKY, the update CHOL_UPDATE
    const int tok = oz ? prof_begin(TK_PHASE_CHOLESKY, st) : -1;
    k_chol_diag<<<N, 256, 0, st>>>(R, ldr, rstride, kb, info_dev);
    TK_LAUNCH_CHECK();
    if (r > 0) {
      k_chol_trsm<<<dim3((unsigned)r, (unsigned)N), CB, 0, st>>>(R, ldr, rstride, kb);
      TK_LAUNCH_CHECK();
    }
    prof_end(tok, st, (double)N * ((double)CB * CB * CB / 3.0 + (double)r * CB * CB * CB),
             8.0 * N * ((double)CB * CB + 2.0 * r * CB * CB));
    if (r == 0) break;
    if (oz) {
      const int64_t w = np - (int64_t)(kb + 1) * CB;
      const int tok = prof_begin(TK_PHASE_CHOL_UPDATE, st);
      TK_TRY(oz_chol_step(*oz, kb, st));
      // algorithmic: the float64 update of the w x w trailing triangle (K = 64) read and written
      prof_end(tok, st, (double)N * w * (w + 1) * CB, 16.0 * N * w * (w + 1) / 2);
    } else {
      k_chol_update<<<dim3((unsigned)(r * (r + 1) / 2), (unsigned)N), 256, 0, st>>>(R, ldr, rstride, kb, nt);
      TK_LAUNCH_CHECK();
    }
  }
  return TK_OK;
}

template <typename TR, typename TX>
tk_status trsv_batched(bool transposed, int64_t n, const TR* R, int64_t ldr, int64_t rstride, const int* idx,
                       const TX* Xin, TX* X, int64_t ldx, int count, double* pbuf, cudaStream_t st) {
  if (count <= 0 || n <= 0) return TK_OK;
  if (pbuf && n > 512) {
    // column sweep across the grid: nb + 1 launches, R read once
    TX* pb = reinterpret_cast<TX*>(pbuf);  // count x n of TX (the buffer holds count x n doubles)
    dim3 gi((unsigned)std::min<int64_t>(cdiv(n, 256), 64), (unsigned)count);
    k_sweep_init<TX><<<gi, 256, 0, st>>>(Xin, ldx, n, pb);
    TK_LAUNCH_CHECK();
    const int64_t nb = cdiv(n, 32);
    const int rpc = count >= 16 ? kSweepRows : 64;  // more CTAs per slot when few slots
    for (int64_t k = 0; k < nb; ++k) {
      if (!transposed) {
        const int64_t b = nb - 1 - k;
        dim3 g((unsigned)std::max<int64_t>(1, cdiv(b * 32, rpc)), (unsigned)count);
        k_sweep_upper<TR, TX><<<g, kTrsvThreads, 0, st>>>(n, R, ldr, rstride, idx, X, ldx, pb, b, rpc);
      } else {
        const int64_t b = k;
        const int64_t rest = n - std::min<int64_t>(n, b * 32 + 32);
        dim3 g((unsigned)std::max<int64_t>(1, cdiv(rest, rpc)), (unsigned)count);
        k_sweep_lower<TR, TX><<<g, kTrsvThreads, 0, st>>>(n, R, ldr, rstride, idx, X, ldx, pb, b, rpc);
      }
      TK_LAUNCH_CHECK();
    }
    return TK_OK;
  }
  const size_t smem = sizeof(double) * (size_t)n;
  if (smem > 200 * 1024) {
    set_error_msg("trsv: order too large for the shared-memory solve");
    return TK_EINVAL;
  }
  // The cap is set to the same constant by every caller: host threads of the
  // batched solver launch concurrently, and a per-call value would race.
  constexpr int kCap = 200 * 1024;
  if (transposed) {
    auto kern = k_trsv_upper_t<TR, TX>;
    TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kCap));
    kern<<<count, kTrsvThreads, smem, st>>>(n, R, ldr, rstride, idx, Xin, X, ldx);
  } else {
    auto kern = k_trsv_upper<TR, TX>;
    TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kCap));
    kern<<<count, kTrsvThreads, smem, st>>>(n, R, ldr, rstride, idx, Xin, X, ldx);
  }
  TK_LAUNCH_CHECK();
  return TK_OK;
}

template tk_status trsv_batched<double, double>(bool, int64_t, const double*, int64_t, int64_t, const int*,
                                                const double*, double*, int64_t, int, double*, cudaStream_t);
template tk_status trsv_batched<float, float>(bool, int64_t, const float*, int64_t, int64_t, const int*, const float*,
                                              float*, int64_t, int, double*, cudaStream_t);
template tk_status trsv_batched<double, float>(bool, int64_t, const double*, int64_t, int64_t, const int*,
                                               const float*, float*, int64_t, int, double*, cudaStream_t);

}  // namespace tk
