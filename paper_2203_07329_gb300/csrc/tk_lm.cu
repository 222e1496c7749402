// The float32 products of LSQR (Algorithm 1 step 5: A R^-1 v and A^T u, for
// every active lambda at once) when at most 16 lambda are active -- the tail of
// the mixed form's LSQR, where the digit products of A would read 8 bytes per
// element of A for few lambda.  Both read the float32 copy of A once, in
// 16-byte vectors along its rows, and keep the lambda-side operand on chip:
//
//  * aw:  C[l][i] = sum_k W[l][k] A[i][k] (+ beta_l C[l][i]).  W (count x n,
//    zero-padded to NL x n_pad) sits in shared memory; a warp takes 4 rows of
//    A at a time, each lane 4 consecutive k of every 128, the next 128 loaded
//    while the current ones are used; the 4 NL dot products per lane are added
//    across the warp by halving exchanges (each step keeps half of the values
//    and adds the partner's other half), then written.
//  * atu: partial[z][l][j] = sum over the rows i of split z of U[l][i] A[i][j].
//    A thread owns CW consecutive columns (4, or 2 for 16 lambda) and NL x CW
//    accumulators, with 8 rows' loads in flight; the rows' U values are staged
//    in shared memory ([row][lambda], read as broadcasts).
#include "tk_lm_body.cuh"

namespace tk {
namespace {

constexpr int LM_AW_THREADS = 512;

// W in column chunks of kc (a multiple of 128) when NL x n floats exceed shared memory: the warps keep
// the same rows in every chunk and add each chunk's sums to C
template <int NL>
__global__ void __launch_bounds__(LM_AW_THREADS)
    k_lm_aw(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n, int64_t kc,
            const float* __restrict__ W, int64_t ldw, int count, float* C, int64_t ldc,
            const double* __restrict__ beta, bool vec) {
  extern __shared__ __align__(16) float lm_ws[];  // [NL][kc]
  constexpr int nwarps = LM_AW_THREADS / 32;
  const int64_t groups = (m + lmb::kRows - 1) / lmb::kRows;
  for (int64_t k0 = 0; k0 < n; k0 += kc) {
    const int64_t len = n - k0 < kc ? n - k0 : kc;
    const int64_t n_pad = (len + 127) / 128 * 128;
    __syncthreads();  // the previous chunk of W is no longer read
    lmb::load_w<NL>(lm_ws, W + k0, ldw, count, len, n_pad);
    __syncthreads();
    lmb::aw_rows<NL>(lm_ws, n_pad, A + k0, lda, m, len, count, C, ldc, beta, vec,
                     (int64_t)blockIdx.x * nwarps + (threadIdx.x >> 5), (int64_t)gridDim.x * nwarps, groups, k0 == 0);
  }
}

// CW columns per thread (4 for <= 8 lambda, 2 for 16: NL x CW accumulators); three CTAs per SM
template <int NL, int CW>
__global__ void __launch_bounds__(lmb::kAtuThreads, 3)
    k_lm_atu(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n, const float* __restrict__ U, int64_t ldu,
             int count, int64_t rows_per, double* __restrict__ partial, bool vec) {
  __shared__ __align__(16) float us[lmb::kAtuRB][NL];
  const int64_t z = blockIdx.x;
  const int64_t rb = z * rows_per, re = rb + rows_per < m ? rb + rows_per : m;
  const int64_t c = (int64_t)blockIdx.y * (CW * lmb::kAtuThreads) + CW * threadIdx.x;
  lmb::atu_cols<NL, CW>(us, A, lda, m, n, U, ldu, count, rb, re, c, partial + z * (int64_t)count * n, vec);
}

int lm_nl(int count) { return count <= 4 ? 4 : (count <= 8 ? 8 : 16); }

}  // namespace

bool lm_small_aw_supported(int64_t n, int count) { return count >= 1 && count <= 16 && n >= 1; }

tk_status lm_small_aw(const float* A, int64_t lda, int64_t m, int64_t n, const float* W, int64_t ldw, int count,
                      float* C, int64_t ldc, const double* beta, cudaStream_t st) {
  if (m == 0 || count == 0) return TK_OK;
  if (!lm_small_aw_supported(n, count)) {
    set_error_msg("float32 product: at most 16 lambda");
    return TK_EINVAL;
  }
  const int nl = lm_nl(count);
  const int64_t kc = lmb::aw_chunk(nl, n);
  const size_t smem = (size_t)nl * (size_t)kc * sizeof(float);
  const bool vec = ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
  const int64_t groups = cdiv(m, lmb::kRows);
#define TK_AW(NL_)                                                                                          \
  {                                                                                                         \
    /* one fixed cap for every call: host lanes launch concurrently with different sizes */             \
    TK_CUDA(cudaFuncSetAttribute(k_lm_aw<NL_>, cudaFuncAttributeMaxDynamicSharedMemorySize, lmb::kAwSmemCap)); \
    int per_sm = 0;                                                                                         \
    TK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lm_aw<NL_>, LM_AW_THREADS, smem));     \
    const int64_t grid = std::max<int64_t>(                                                                 \
        1, std::min<int64_t>(cdiv(groups, LM_AW_THREADS / 32), 152 * (int64_t)std::max(per_sm, 1)));        \
    k_lm_aw<NL_><<<(unsigned)grid, LM_AW_THREADS, smem, st>>>(A, lda, m, n, kc, W, ldw, count, C, ldc, beta, \
                                                              vec);                                         \
  }
  if (nl == 4) TK_AW(4) else if (nl == 8) TK_AW(8) else TK_AW(16)
#undef TK_AW
  TK_LAUNCH_CHECK();
  return TK_OK;
}

int lm_small_atu_splits(int64_t m, int64_t n) {
  const int64_t tiles = cdiv(n, 2 * lmb::kAtuThreads);
  const int64_t want = cdiv(3 * 152, tiles);                 // three CTAs per SM
  const int64_t maxs = std::max<int64_t>(1, cdiv(m, 64));    // at least 64 rows per split
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, maxs));
}

tk_status lm_small_atu(const float* A, int64_t lda, int64_t m, int64_t n, const float* U, int64_t ldu, int count,
                       double* partial, int splits, cudaStream_t st) {
  if (n == 0 || count == 0) return TK_OK;
  if (count > 16 || splits < 1) {
    set_error_msg("float32 product: at most 16 lambda");
    return TK_EINVAL;
  }
  const int64_t rows_per = std::max<int64_t>(1, cdiv(m, splits));
  const int nl = lm_nl(count);
  const int cw = nl == 16 ? 2 : 4;
  const dim3 grid((unsigned)splits, (unsigned)cdiv(n, (int64_t)cw * lmb::kAtuThreads));
  if (grid.y > 65535u) {
    set_error_msg("float32 product: too many columns");
    return TK_EINVAL;
  }
  if (m == 0) {
    TK_CUDA(cudaMemsetAsync(partial, 0, sizeof(double) * (size_t)splits * count * n, st));
    return TK_OK;
  }
  const bool vec = ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
  if (nl == 4) k_lm_atu<4, 4><<<grid, lmb::kAtuThreads, 0, st>>>(A, lda, m, n, U, ldu, count, rows_per, partial, vec);
  else if (nl == 8) k_lm_atu<8, 4><<<grid, lmb::kAtuThreads, 0, st>>>(A, lda, m, n, U, ldu, count, rows_per, partial, vec);
  else k_lm_atu<16, 2><<<grid, lmb::kAtuThreads, 0, st>>>(A, lda, m, n, U, ldu, count, rows_per, partial, vec);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

}  // namespace tk
