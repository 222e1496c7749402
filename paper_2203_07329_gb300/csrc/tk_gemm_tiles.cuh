// Tile bodies of the two SIMT GEMMs, as device functions, so that the plain
// kernels (one problem per launch, tk_dense.cu) and the grouped kernels (a
// tile list over many problems per launch, tk_group.cu) run the same code.
// A tile is told its coordinates and K range explicitly; the caller owns the
// shared memory.
#pragma once

#include <algorithm>
#include <type_traits>

#include "tk_internal.cuh"

namespace tk {
namespace tiles {

template <typename A, typename B>
struct AccOf { using type = double; };
template <>
struct AccOf<float, float> { using type = float; };

// ---------------------------------------------------------------------------
// Generic tile: C = alpha op(A) op(B) [+ beta_row[i] * Cin], or with `partial`
// the raw partial sum of the K range [kbeg, kend) into partial (M x N).
// op(A) is M x K: A[i*lda + k] (N) or A[k*lda + i] (T).  op(B) is K x N:
// B[k*ldb + j] (N) or B[j*ldb + k] (T).  ldcin = 0 broadcasts one Cin row.
template <typename TA, typename TB, int BM, int BN, int BK>
struct GemmSmem {
  using Acc = typename AccOf<TA, TB>::type;
  Acc As[BK][BM + 1];
  Acc Bs[BK][BN + 1];
};

template <typename TA, typename TB, typename TC, int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void gemm_tile(GemmSmem<TA, TB, BM, BN, BK>& sm, bool transA, bool transB, int64_t M,
                                          int64_t N, const TA* __restrict__ A, int64_t lda,
                                          const TB* __restrict__ B, int64_t ldb, TC* C, int64_t ldc, double alpha,
                                          const double* __restrict__ beta_row, const TC* Cin, int64_t ldcin,
                                          int64_t m0, int64_t n0, int64_t kbeg, int64_t kend,
                                          double* __restrict__ partial) {
  using Acc = typename AccOf<TA, TB>::type;
  constexpr int NT = (BM / TM) * (BN / TN);
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  Acc acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Acc(0);

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    // A tile: BM x BK; the fastest thread index walks the contiguous axis.
    for (int idx = tid; idx < BM * BK; idx += NT) {
      int i, k;
      if (!transA) { k = idx % BK; i = idx / BK; } else { i = idx % BM; k = idx / BM; }
      int64_t gi = m0 + i, gk = k0 + k;
      Acc v = Acc(0);
      if (gi < M && gk < kend) v = (Acc)(transA ? A[gk * lda + gi] : A[gi * lda + gk]);
      sm.As[k][i] = v;
    }
    for (int idx = tid; idx < BK * BN; idx += NT) {
      int j, k;
      if (!transB) { j = idx % BN; k = idx / BN; } else { k = idx % BK; j = idx / BK; }
      int64_t gj = n0 + j, gk = k0 + k;
      Acc v = Acc(0);
      if (gj < N && gk < kend) v = (Acc)(transB ? B[gj * ldb + gk] : B[gk * ldb + gj]);
      sm.Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Acc a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = sm.As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = sm.Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t r = m0 + ty * TM + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t c = n0 + tx * TN + j;
      if (c >= N) continue;
      if (partial) {
        partial[r * N + c] = (double)acc[i][j];
      } else {
        double v = alpha * (double)acc[i][j];
        if (beta_row) v += beta_row[r] * (double)Cin[r * ldcin + c];
        C[r * ldc + c] = (TC)v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Lambda-major float32 tile of LSQR: C (M x N) = L (M x K) op(A) with M <= BM
// (every active lambda in one tile) and a long N.  op(A)[k][j] is
// A[j*lda + k] (TRANSB: the product with A^T, N = rows of A) or A[k*lda + j].
// Warps are arranged 2 x 4 over the tile and lanes 4 x 8 inside a warp, so a
// warp's shared-memory reads of L touch 4 rows (broadcast) and of B 8 column
// groups; every thread keeps TM x TN accumulators.  The next K-slab is loaded
// into registers (16-byte loads when `vec`) while the current one is consumed
// from shared memory (two buffers, one barrier per slab).  Epilogue: C =
// D + beta_row .* Cin, or the raw partial sum into `partial` (M x N).
constexpr int LM_BK = 16;
constexpr int LM_BN = 256;

template <int BM>
struct LmSmem {
  float Ls[2][LM_BK][BM];
  float Bs[2][LM_BK][LM_BN + 4];
};

template <bool TRANSB, int BM, int TM>
__device__ __forceinline__ void gemm_lm_tile(LmSmem<BM>& sm, bool vec, int64_t M, int64_t N,
                                             const float* __restrict__ L, int64_t ldl, const float* __restrict__ A,
                                             int64_t lda, float* C, int64_t ldc, const double* __restrict__ beta_row,
                                             const float* Cin, int64_t ldcin, int64_t n0, int64_t kbeg, int64_t kend,
                                             double* __restrict__ partial) {
  constexpr int BK = LM_BK, BN = LM_BN, TN = 8;
  constexpr int LV = (BM * BK) / (4 * 256) > 0 ? (BM * BK) / (4 * 256) : 1;  // float4 per thread for L
  constexpr int BV = (BN * BK) / (4 * 256);                                 // float4 per thread for B
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  static_assert(BM / TM == 8 && BN / TN == 32, "2 x 4 warps of 4 x 8 lanes");
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ty = (w >> 2) * 4 + (lane >> 3);  // 0..7  row group
  const int tx = (w & 3) * 8 + (lane & 7);    // 0..31 column group
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  float4 rl[LV], rb[BV];
  // quad q of L: row i = q / (BK/4), k = 4 * (q % (BK/4)); of B (TRANSB): row j = q / 4, k = 4 * (q % 4);
  // of B (not TRANSB): k = q / (BN/4), j = 4 * (q % (BN/4))
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int v = 0; v < LV; ++v) {
      const int q = tid + v * 256;
      const int i = q / (BK / 4), k = 4 * (q % (BK / 4));
      float e[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) e[t] = 0.f;
      if (q < BM * BK / 4 && i < M) {
        const int64_t gk = k0 + k;
        if (vec && gk + 3 < kend) {
          const float4 f = *reinterpret_cast<const float4*>(L + (int64_t)i * ldl + gk);
          e[0] = f.x; e[1] = f.y; e[2] = f.z; e[3] = f.w;
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t) e[t] = (gk + t < kend) ? L[(int64_t)i * ldl + gk + t] : 0.f;
        }
      }
      rl[v] = make_float4(e[0], e[1], e[2], e[3]);
    }
#pragma unroll
    for (int v = 0; v < BV; ++v) {
      const int q = tid + v * 256;
      float e[4];
      if (TRANSB) {
        const int j = q / 4, k = 4 * (q % 4);
        const int64_t gj = n0 + j, gk = k0 + k;
        if (gj < N && vec && gk + 3 < kend) {
          const float4 f = *reinterpret_cast<const float4*>(A + gj * lda + gk);
          e[0] = f.x; e[1] = f.y; e[2] = f.z; e[3] = f.w;
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t) e[t] = (gj < N && gk + t < kend) ? A[gj * lda + gk + t] : 0.f;
        }
      } else {
        const int k = q / (BN / 4), j = 4 * (q % (BN / 4));
        const int64_t gj = n0 + j, gk = k0 + k;
        if (gk < kend && vec && gj + 3 < N) {
          const float4 f = *reinterpret_cast<const float4*>(A + gk * lda + gj);
          e[0] = f.x; e[1] = f.y; e[2] = f.z; e[3] = f.w;
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t) e[t] = (gk < kend && gj + t < N) ? A[gk * lda + gj + t] : 0.f;
        }
      }
      rb[v] = make_float4(e[0], e[1], e[2], e[3]);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int v = 0; v < LV; ++v) {
      const int q = tid + v * 256;
      if (q < BM * BK / 4) {
        const int i = q / (BK / 4), k = 4 * (q % (BK / 4));
        sm.Ls[buf][k + 0][i] = rl[v].x;
        sm.Ls[buf][k + 1][i] = rl[v].y;
        sm.Ls[buf][k + 2][i] = rl[v].z;
        sm.Ls[buf][k + 3][i] = rl[v].w;
      }
    }
#pragma unroll
    for (int v = 0; v < BV; ++v) {
      const int q = tid + v * 256;
      if (TRANSB) {
        const int j = q / 4, k = 4 * (q % 4);
        sm.Bs[buf][k + 0][j] = rb[v].x;
        sm.Bs[buf][k + 1][j] = rb[v].y;
        sm.Bs[buf][k + 2][j] = rb[v].z;
        sm.Bs[buf][k + 3][j] = rb[v].w;
      } else {
        const int k = q / (BN / 4), j = 4 * (q % (BN / 4));
        *reinterpret_cast<float4*>(&sm.Bs[buf][k][j]) = rb[v];
      }
    }
  };
  int cur = 0;
  if (kbeg < kend) {
    load(kbeg);
    store(0);
  }
  __syncthreads();
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = sm.Ls[cur][kk][ty * TM + i];
      // column pairs 64 j2 + 2 tx + {0, 1}: a warp's 8 column groups read one
      // contiguous 64-byte chunk per 8-byte load (no bank conflicts)
#pragma unroll
      for (int j2 = 0; j2 < TN / 2; ++j2) {
        const float2 f = *reinterpret_cast<const float2*>(&sm.Bs[cur][kk][64 * j2 + 2 * tx]);
        bv[2 * j2] = f.x;
        bv[2 * j2 + 1] = f.y;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], bv[j], acc[i][j]);
    }
    if (more) store(cur ^ 1);
    __syncthreads();
    cur ^= 1;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t r = ty * TM + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t c = n0 + 64 * (j >> 1) + 2 * tx + (j & 1);
      if (c >= N) continue;
      if (partial) {
        partial[r * N + c] = (double)acc[i][j];
      } else {
        double v = (double)acc[i][j];
        if (beta_row) v += beta_row[r] * (double)Cin[r * ldcin + c];
        C[r * ldc + c] = (float)v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Triangular matrix-vector rows: out[i] = M[i, :] x for rows
// i0 <= i < min(n, i0 + kTrmvRows), UPPER over columns i..n-1, else (the
// stored transpose, lower) over 0..i.  The vector is staged in shared memory
// (rounded up to 16 bytes, zero past n); rows are read in 16-byte vectors
// (row stride and base 16-byte aligned), starting at the vector that holds
// column i (upper) or ending at it (lower): the extra entries lie in the
// 64-aligned diagonal block, where that triangle is stored as zeros.  256 threads.
constexpr int kTrmvRows = 64;  // rows per CTA (8 warps x 8 rows)

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int W = 4;
  __device__ static float dot(const float4& a, const float4& b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
  }
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int W = 2;
  __device__ static double dot(const double2& a, const double2& b, double acc) {
    acc = fma(a.x, b.x, acc);
    return fma(a.y, b.y, acc);
  }
};

template <typename T>
inline size_t trmv_smem_bytes(int64_t n) {
  return sizeof(T) * (size_t)Vec16<T>::W * (size_t)cdiv(n, Vec16<T>::W);
}

template <typename T, bool UPPER>
__device__ __forceinline__ void trmv_rows(int64_t n, const T* __restrict__ Ml, int64_t ldm, const T* x, T* out,
                                          int64_t i0, void* smem) {
  using V = typename Vec16<T>::type;
  constexpr int W = Vec16<T>::W;
  T* v = reinterpret_cast<T*>(smem);
  const V* vv = reinterpret_cast<const V*>(smem);
  const int64_t nv = cdiv(n, W);
  for (int64_t j = threadIdx.x; j < W * nv; j += blockDim.x) v[j] = j < n ? x[j] : T(0);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = 0; q < kTrmvRows / 8; ++q) {
    const int64_t i = i0 + w + 8 * q;
    if (i >= n) break;
    const V* row = reinterpret_cast<const V*>(Ml + i * ldm);
    const int64_t j0 = UPPER ? (i / W) : 0, j1 = UPPER ? nv : (i / W) + 1;
    T acc = T(0);
#pragma unroll 4
    for (int64_t j = j0 + lane; j < j1; j += 32) acc = Vec16<T>::dot(__ldg(row + j), vv[j], acc);
    acc = warp_sum(acc);
    if (lane == 0) out[i] = acc;
  }
}

}  // namespace tiles
}  // namespace tk
