// Device bodies of the float32 LSQR products for at most 16 lambda, shared by
// the single-problem kernels (tk_lm.cu) and the grouped engine (tk_group.cu).
// Both read the float32 A once in 16-byte vectors along its rows and keep the
// lambda-side operand on chip:
//  * aw_rows: C[l][i] = sum_k W[l][k] A[i][k] (+ beta_l C[l][i]; first = false:
//    C[l][i] += the sum, for a later chunk of columns) for the 4-row
//    groups g_first, g_first + g_stride, ... < g_end, one warp per group at a
//    time; W (zero-padded to NL x n_pad) is in shared memory (load_w); each lane
//    takes 4 consecutive k of every 128, the next 128 loaded while the current
//    ones are used; the 4 NL dot products per lane are added across the warp by
//    halving exchanges (each step keeps half of the values and adds the
//    partner's other half), then written.
//  * atu_cols: out[l][c + t] = sum over rows rb <= i < re of U[l][i] A[i][c + t]
//    for the thread's CW columns (NL x CW accumulators, 8 rows' loads in flight);
//    the rows' U values are staged in shared memory ([row][lambda], read as
//    broadcasts).  Every thread of the block must call it (it synchronizes).
#pragma once
#include "tk_internal.cuh"

namespace tk {
namespace lmb {

constexpr int kRows = 4;          // rows of A per warp (aw)
constexpr int kAtuThreads = 256;  // threads of an atu block
constexpr int kAtuRB = 128;       // rows of U staged at a time (atu)
constexpr int kAwSmemCap = 200 * 1024;  // W's column chunk in shared memory (aw)

// Columns of W (and A) per chunk of the aw product: the most, in 128s, whose NL x chunk floats fit
__host__ __device__ inline int64_t aw_chunk(int nl, int64_t n) {
  const int64_t fit = (int64_t)kAwSmemCap / (4 * nl) / 128 * 128;
  const int64_t n_pad = (n + 127) / 128 * 128;
  return n_pad < fit ? n_pad : fit;
}

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

// ws[l][k] = W[l][k] for l < count, k < n, zero elsewhere (NL x n_pad); the caller synchronizes
template <int NL>
__device__ __forceinline__ void load_w(float* ws, const float* __restrict__ W, int64_t ldw, int count, int64_t n,
                                       int64_t n_pad) {
  for (int64_t idx = threadIdx.x; idx < (int64_t)NL * n_pad; idx += blockDim.x) {
    const int l = (int)(idx / n_pad);
    const int64_t k = idx % n_pad;
    ws[idx] = (l < count && k < n) ? W[(int64_t)l * ldw + k] : 0.f;
  }
}

template <int NL>
__device__ __forceinline__ void aw_rows(const float* ws, int64_t n_pad, const float* __restrict__ A, int64_t lda,
                                        int64_t m, int64_t n, int count, float* C, int64_t ldc,
                                        const double* __restrict__ beta, bool vec, int64_t g_first,
                                        int64_t g_stride, int64_t g_end, bool first = true) {
  constexpr int LM_ROWS = kRows;
  const int lane = threadIdx.x & 31;
  const int nj = (int)(n_pad / 128);
  for (int64_t g = g_first; g < g_end; g += g_stride) {
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
        const float4 w4 = *reinterpret_cast<const float4*>(ws + (int64_t)l * n_pad + k);
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
            if (!first) val += (double)C[(int64_t)l * ldc + i];  // a later column chunk: add to the sum
            else if (beta) val += beta[l] * (double)C[(int64_t)l * ldc + i];
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
__device__ __forceinline__ void atu_cols(float (*us)[NL], const float* __restrict__ A, int64_t lda, int64_t m,
                                         int64_t n, const float* __restrict__ U, int64_t ldu, int count, int64_t rb,
                                         int64_t re, int64_t c, double* __restrict__ out, bool vec) {
  constexpr int RU = 8;
  constexpr int LM_ATU_RB = kAtuRB, LM_ATU_THREADS = kAtuThreads;
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

}  // namespace lmb
}  // namespace tk
