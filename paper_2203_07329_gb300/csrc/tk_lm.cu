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
#include "tk_internal.cuh"

namespace tk {
namespace {

constexpr int LM_ROWS = 4;        // rows of A per warp (aw)
constexpr int LM_AW_THREADS = 512;
constexpr int LM_ATU_THREADS = 256;
constexpr int LM_ATU_RB = 128;                   // rows of U staged at a time (atu)

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}

// 4 consecutive floats of a row from column k (zero past `len`); vector load when allowed
__device__ __forceinline__ float4 load4(const float* __restrict__ row, int64_t k, int64_t len, bool vec) {
  if (vec && k + 3 < len) return __ldg(reinterpret_cast<const float4*>(row + k));
  float e[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) e[t] = k + t < len ? __ldg(row + k + t) : 0.f;
  return make_float4(e[0], e[1], e[2], e[3]);
}

template <int NL>
__global__ void __launch_bounds__(LM_AW_THREADS)
    k_lm_aw(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n, int64_t n_pad,
            const float* __restrict__ W, int64_t ldw, int count, float* C, int64_t ldc,
            const double* __restrict__ beta, bool vec) {
  extern __shared__ __align__(16) float lm_ws[];  // [NL][n_pad]
  for (int64_t idx = threadIdx.x; idx < (int64_t)NL * n_pad; idx += blockDim.x) {
    const int l = (int)(idx / n_pad);
    const int64_t k = idx % n_pad;
    lm_ws[idx] = (l < count && k < n) ? W[(int64_t)l * ldw + k] : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = LM_AW_THREADS / 32;
  const int64_t groups = (m + LM_ROWS - 1) / LM_ROWS;
  const int nj = (int)(n_pad / 128);
  for (int64_t g = (int64_t)blockIdx.x * nwarps + warp; g < groups; g += (int64_t)gridDim.x * nwarps) {
    const int64_t i0 = g * LM_ROWS;
    const float* rows[LM_ROWS];
#pragma unroll
    for (int r = 0; r < LM_ROWS; ++r) rows[r] = A + (i0 + r < m ? i0 + r : i0) * lda;
    const int rmax = (int)(m - i0 < LM_ROWS ? m - i0 : LM_ROWS);
    float acc[LM_ROWS][NL];
#pragma unroll
    for (int r = 0; r < LM_ROWS; ++r)
#pragma unroll
      for (int l = 0; l < NL; ++l) acc[r][l] = 0.f;
    float4 cur[LM_ROWS], nxt[LM_ROWS];
#pragma unroll
    for (int r = 0; r < LM_ROWS; ++r)
      cur[r] = r < rmax ? load4(rows[r], 4 * lane, n, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = 0; j < nj; ++j) {
      const int64_t k = (int64_t)128 * j + 4 * lane;
      if (j + 1 < nj) {
#pragma unroll
        for (int r = 0; r < LM_ROWS; ++r)
          nxt[r] = r < rmax ? load4(rows[r], k + 128, n, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        const float4 w4 = *reinterpret_cast<const float4*>(lm_ws + (int64_t)l * n_pad + k);
#pragma unroll
        for (int r = 0; r < LM_ROWS; ++r) acc[r][l] = dot4(cur[r], w4, acc[r][l]);
      }
#pragma unroll
      for (int r = 0; r < LM_ROWS; ++r) cur[r] = nxt[r];
    }
    // add the V = 4 NL values across the warp: each halving step keeps half (the lanes with bit s
    // set keep the upper half) and adds the partner's copy of it; once one value is left, plain steps
    constexpr int V = LM_ROWS * NL;
    float v[V];
#pragma unroll
    for (int r = 0; r < LM_ROWS; ++r)
#pragma unroll
      for (int l = 0; l < NL; ++l) v[r * NL + l] = acc[r][l];
    int nv = V, qbase = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      if (nv > 1) {
        const int half = nv / 2;
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int q = 0; q < V / 2; ++q) {
          if (q < half) {
            const float send = up ? v[q] : v[q + half];
            const float keep = up ? v[q + half] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, s);
          }
        }
        if (up) qbase += half;
        nv = half;
      } else {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], s);
      }
    }
    // lane holds values qbase .. qbase + nv - 1 (V >= 32: 2 or 1 per lane; V = 16: the same value on
    // two lanes, written by the one with bit 0 clear)
    const bool writer = V >= 32 || (lane & 1) == 0;
    if (writer) {
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (t < nv) {
          const int q = qbase + t, r = q / NL, l = q % NL;
          const int64_t i = i0 + r;
          if (i < m && l < count) {
            double val = (double)v[t];
            if (beta) val += beta[l] * (double)C[(int64_t)l * ldc + i];
            C[(int64_t)l * ldc + i] = (float)val;
          }
        }
      }
    }
  }
}

// CW consecutive floats of a row from column k (zero past `len`); vector load when allowed
template <int CW>
__device__ __forceinline__ void loadv(const float* __restrict__ row, int64_t k, int64_t len, bool vec, float (&o)[CW]) {
  if (vec && k + CW - 1 < len) {
    if constexpr (CW == 4) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(row + k));
      o[0] = f.x; o[1] = f.y; o[2] = f.z; o[3] = f.w;
    } else {
      const float2 f = __ldg(reinterpret_cast<const float2*>(row + k));
      o[0] = f.x; o[1] = f.y;
    }
    return;
  }
#pragma unroll
  for (int t = 0; t < CW; ++t) o[t] = k + t < len ? __ldg(row + k + t) : 0.f;
}

// CW columns per thread (4 for <= 8 lambda, 2 for 16: NL x CW accumulators), 8 rows' loads in flight
template <int NL, int CW>
__global__ void __launch_bounds__(LM_ATU_THREADS, 2)
    k_lm_atu(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n, const float* __restrict__ U, int64_t ldu,
             int count, int64_t rows_per, double* __restrict__ partial, bool vec) {
  constexpr int RU = 8;
  __shared__ __align__(16) float us[LM_ATU_RB][NL];
  const int64_t z = blockIdx.x;
  const int64_t rb = z * rows_per, re = rb + rows_per < m ? rb + rows_per : m;
  const int64_t c = (int64_t)blockIdx.y * (CW * LM_ATU_THREADS) + CW * threadIdx.x;
  float acc[NL][CW];
#pragma unroll
  for (int l = 0; l < NL; ++l)
#pragma unroll
    for (int t = 0; t < CW; ++t) acc[l][t] = 0.f;
  for (int64_t i0 = rb; i0 < re; i0 += LM_ATU_RB) {
    const int nr = (int)(re - i0 < LM_ATU_RB ? re - i0 : LM_ATU_RB);
    __syncthreads();  // the previous rows' U values are no longer read
    for (int idx = threadIdx.x; idx < LM_ATU_RB * NL; idx += LM_ATU_THREADS) {
      const int l = idx / LM_ATU_RB, r = idx % LM_ATU_RB;
      us[r][l] = (l < count && r < nr) ? U[(int64_t)l * ldu + i0 + r] : 0.f;
    }
    __syncthreads();
    if (c < n) {
      for (int r = 0; r < nr; r += RU) {
        float a[RU][CW];
#pragma unroll
        for (int q = 0; q < RU; ++q) {
          if (r + q < nr) loadv<CW>(A + (i0 + r + q) * lda, c, n, vec, a[q]);
          else {
#pragma unroll
            for (int t = 0; t < CW; ++t) a[q][t] = 0.f;  // us is zero there too
          }
        }
#pragma unroll
        for (int q = 0; q < RU; ++q) {
#pragma unroll
          for (int l4 = 0; l4 < NL / 4; ++l4) {
            const float4 u4 = *reinterpret_cast<const float4*>(&us[r + q][4 * l4]);
            const float uu[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
            for (int t4 = 0; t4 < 4; ++t4)
#pragma unroll
              for (int t = 0; t < CW; ++t) acc[4 * l4 + t4][t] = fmaf(uu[t4], a[q][t], acc[4 * l4 + t4][t]);
          }
        }
      }
    }
  }
  if (c < n) {
    double* out = partial + z * (int64_t)count * n;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      if (l < count) {
#pragma unroll
        for (int t = 0; t < CW; ++t)
          if (c + t < n) out[(int64_t)l * n + c + t] = (double)acc[l][t];
      }
    }
  }
}

int lm_nl(int count) { return count <= 4 ? 4 : (count <= 8 ? 8 : 16); }

}  // namespace

constexpr int kLmAwSmemCap = 200 * 1024;  // W in shared memory (aw)

bool lm_small_aw_supported(int64_t n, int count) {
  if (count < 1 || count > 16) return false;
  const int64_t n_pad = cdiv(n, 128) * 128;
  return (size_t)lm_nl(count) * (size_t)n_pad * sizeof(float) <= (size_t)kLmAwSmemCap;
}

tk_status lm_small_aw(const float* A, int64_t lda, int64_t m, int64_t n, const float* W, int64_t ldw, int count,
                      float* C, int64_t ldc, const double* beta, cudaStream_t st) {
  if (m == 0 || count == 0) return TK_OK;
  if (!lm_small_aw_supported(n, count)) {
    set_error_msg("float32 product: lambda-side operand too large for shared memory");
    return TK_EINVAL;
  }
  const int64_t n_pad = cdiv(n, 128) * 128;
  const int nl = lm_nl(count);
  const size_t smem = (size_t)nl * (size_t)n_pad * sizeof(float);
  const bool vec = ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
  const int64_t groups = cdiv(m, LM_ROWS);
#define TK_AW(NL_)                                                                                          \
  {                                                                                                         \
    /* one fixed cap for every call: host lanes launch concurrently with different sizes */             \
    TK_CUDA(cudaFuncSetAttribute(k_lm_aw<NL_>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLmAwSmemCap)); \
    int per_sm = 0;                                                                                         \
    TK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lm_aw<NL_>, LM_AW_THREADS, smem));     \
    const int64_t grid = std::max<int64_t>(                                                                 \
        1, std::min<int64_t>(cdiv(groups, LM_AW_THREADS / 32), 152 * (int64_t)std::max(per_sm, 1)));        \
    k_lm_aw<NL_><<<(unsigned)grid, LM_AW_THREADS, smem, st>>>(A, lda, m, n, n_pad, W, ldw, count, C, ldc, beta, \
                                                              vec);                                         \
  }
  if (nl == 4) TK_AW(4) else if (nl == 8) TK_AW(8) else TK_AW(16)
#undef TK_AW
  TK_LAUNCH_CHECK();
  return TK_OK;
}

int lm_small_atu_splits(int64_t m, int64_t n) {
  const int64_t tiles = cdiv(n, 2 * LM_ATU_THREADS);
  const int64_t want = cdiv(2 * 152, tiles);                 // two CTAs per SM
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
  const dim3 grid((unsigned)splits, (unsigned)cdiv(n, (int64_t)cw * LM_ATU_THREADS));
  if (grid.y > 65535u) {
    set_error_msg("float32 product: too many columns");
    return TK_EINVAL;
  }
  if (m == 0) {
    TK_CUDA(cudaMemsetAsync(partial, 0, sizeof(double) * (size_t)splits * count * n, st));
    return TK_OK;
  }
  const bool vec = ((uintptr_t)A % 16 == 0) && (lda % 4 == 0);
  if (nl == 4) k_lm_atu<4, 4><<<grid, LM_ATU_THREADS, 0, st>>>(A, lda, m, n, U, ldu, count, rows_per, partial, vec);
  else if (nl == 8) k_lm_atu<8, 4><<<grid, LM_ATU_THREADS, 0, st>>>(A, lda, m, n, U, ldu, count, rows_per, partial, vec);
  else k_lm_atu<16, 2><<<grid, LM_ATU_THREADS, 0, st>>>(A, lda, m, n, U, ldu, count, rows_per, partial, vec);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

}  // namespace tk
