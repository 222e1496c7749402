// Float64-accurate products on the BF16 tensor cores (splitting into exact
// integer slices, in the manner of Ozaki's error-free matrix multiplication).
//
// GB300 issues about two float64 FMA per clock per SM, so the float64 passes
// of the mixed form's refinement (r = b - X A^T, a float64 GEMM with 32 lambda
// rows) are bound by that pipe.  Here every row of A is scaled by a power of
// two so that its entries lie in (-1, 1) and split into S = 8 signed 7-bit
// integer slices,  a = sum_p s_p 2^(-7(p+1)),  |s_p| <= 127,  exactly
// representable in BF16; the lambda rows of X are split the same way.  A
// product of two slices is an integer below 2^14; the pairs (p, q) with
// p + q = t share one FP32 accumulator ("level" t), and a level sum of at most
// 8 pairs over 128 values of K stays below 2^24, so the tensor core's FP32
// accumulation is exact.  Every 128 values of K the level sums are scaled by
// 2^(-7(t+2)) and added into float64 accumulators (smallest level first).
// Pairs with p + q > 7 are dropped: their contribution is below
// 9 * 2^-56 of max|a| max|x| per product, and the 56-bit slicing of a and x
// rounds at 2^-57 of their row maxima: the float64 accuracy of a float64
// GEMM.  The products are mma.sync m16n8k16 BF16 (FP32 accumulate).
#include <algorithm>
#include <cuda_bf16.h>

#include "tk_internal.cuh"

namespace tk {
namespace {

constexpr int OZ_S = 8;          // slices
constexpr int OZ_LV = OZ_S;      // levels t = p + q in 0..7 kept
constexpr int OZ_BM = 64;        // rows of A per CTA
constexpr int OZ_BN = 32;        // lambda rows per CTA
constexpr int OZ_BK = 32;        // K per pipeline stage
constexpr int OZ_STAGES = 3;
constexpr int OZ_LDS = OZ_BK + 8;  // padded smem row (bf16): 80 bytes
constexpr int OZ_CHUNK = 128;    // K per exact level accumulation

// Exponent E with max_j |row_j| < 2^E (0 for a zero row); one warp per row.
template <typename T>
__global__ void k_oz_rowexp(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld, int* __restrict__ E) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const int lane = threadIdx.x & 31;
  double mx = 0.0;
  for (int64_t j = lane; j < cols; j += 32) mx = fmax(mx, fabs((double)X[r * ld + j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, 0.5 <= f < 1, so mx < 2^e
    E[r] = e;
  }
}

// Exponent E with max_r |X[r][c]| < 2^E per column (0 for a zero column):
// the bit patterns of non-negative doubles order like the values, so the
// column maxima are combined with an integer atomicMax (mx zeroed first).
template <typename T>
__global__ void k_oz_colmax(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld, int64_t rows_per,
                            unsigned long long* __restrict__ mx) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per, r1 = r0 + rows_per < rows ? r0 + rows_per : rows;
  double v = 0.0;
#pragma unroll 8
  for (int64_t r = r0; r < r1; ++r) v = fmax(v, fabs((double)X[r * ld + c]));
  atomicMax(&mx[c], (unsigned long long)__double_as_longlong(v));
}
__global__ void k_oz_colexp(const unsigned long long* __restrict__ mx, int64_t cols, int* __restrict__ E) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const double v = __longlong_as_double((long long)mx[c]);
  int e = 0;
  if (v > 0.0) frexp(v, &e);
  E[c] = e;
}

// Slices of X: planes out[p][r][c] (bf16, row stride cols_pad, zero in the
// padding) with X[r][c] 2^-E = sum_p out[p][r][c] 2^(-7(p+1)) to within 2^-57
// (rounded to nearest, so the errors of a row do not share a sign), E = E[r]
// (row exponents) or E[c] (column exponents, COLS).  The fixed-point value is
// formed with one scaling by a power of two and one conversion to int64.
template <typename T, bool COLS>
__global__ void k_oz_slice(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld, const int* __restrict__ E,
                           int64_t cols_pad, __nv_bfloat16* __restrict__ out) {
  const int64_t total = rows * cols_pad;
  const int64_t plane = total;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = k / cols_pad, c = k - r * cols_pad;
    long long v = 0;
    if (c < cols) v = llrint(ldexp((double)X[r * ld + c], 7 * OZ_S - E[COLS ? c : r]));  // |v| <= 2^56
    const bool neg = v < 0;
    unsigned long long u = neg ? (unsigned long long)(-v) : (unsigned long long)v;
    u = u < (1ull << (7 * OZ_S)) ? u : (1ull << (7 * OZ_S)) - 1;  // 56 bits
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) {
      const int s = (int)((u >> (7 * (OZ_S - 1 - p))) & 127u);
      out[p * plane + k] = __int2bfloat16_rn(neg ? -s : s);
    }
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;  // zero-fill when out of range
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct OzSmem {
  __nv_bfloat16 a[OZ_STAGES][OZ_S][OZ_BM][OZ_LDS];  // A slices: rows x K
  __nv_bfloat16 x[OZ_STAGES][OZ_S][OZ_BN][OZ_LDS];  // X slices: lambda rows x K
};

// R[l][i] = b[i] - sum_k X[l][k] A[i][k] for i < m, l < M (float64 result).
// A slices: OZ_S planes of m x kp (kp = K rounded up to 8, zero padded), row
// exponents EA; X slices: OZ_S planes of M x kp, row exponents EX.  CTA: 64
// rows of A x 32 lambda rows; 8 warps = 4 (16 rows) x 2 (16 lambda).
__global__ void __launch_bounds__(256, 1)
    k_oz_residual(const __nv_bfloat16* __restrict__ As, const int* __restrict__ EA, int64_t m, int64_t kp,
                  const __nv_bfloat16* __restrict__ Xs, const int* __restrict__ EX, int64_t M,
                  const double* __restrict__ b, double* __restrict__ R, int64_t ldr) {
  extern __shared__ __align__(16) unsigned char oz_raw[];
  OzSmem& S = *reinterpret_cast<OzSmem*>(oz_raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int wr = w & 3, wc = w >> 2;
  const int64_t i0 = (int64_t)blockIdx.x * OZ_BM, l0 = (int64_t)blockIdx.y * OZ_BN;
  const int64_t planeA = m * kp, planeX = M * kp;
  const int nk = (int)(kp / OZ_BK) + (kp % OZ_BK ? 1 : 0);

  auto load = [&](int stage, int kt) {
    const int64_t k0 = (int64_t)kt * OZ_BK;
    // A: OZ_S x 64 rows x 4 chunks of 8 bf16; X: OZ_S x 32 rows x 4 chunks
    for (int q = tid; q < OZ_S * OZ_BM * 4; q += 256) {
      const int p = q / (OZ_BM * 4), rem = q % (OZ_BM * 4), r = rem >> 2, c = (rem & 3) * 8;
      const int64_t gi = i0 + r, gk = k0 + c;
      const bool ok = gi < m && gk < kp;
      cp_async16(&S.a[stage][p][r][c], ok ? (const void*)(As + p * planeA + gi * kp + gk) : (const void*)As, ok);
    }
    for (int q = tid; q < OZ_S * OZ_BN * 4; q += 256) {
      const int p = q / (OZ_BN * 4), rem = q % (OZ_BN * 4), r = rem >> 2, c = (rem & 3) * 8;
      const int64_t gl = l0 + r, gk = k0 + c;
      const bool ok = gl < M && gk < kp;
      cp_async16(&S.x[stage][p][r][c], ok ? (const void*)(Xs + p * planeX + gl * kp + gk) : (const void*)Xs, ok);
    }
  };

  float acc[OZ_LV][2][4];
  double acc64[2][4];
#pragma unroll
  for (int t = 0; t < OZ_LV; ++t)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[t][j][e] = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc64[j][e] = 0.0;

  auto flush = [&]() {
#pragma unroll
    for (int t = OZ_LV - 1; t >= 0; --t) {
      const double sc = ldexp(1.0, -7 * (t + 2));
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          acc64[j][e] = fma((double)acc[t][j][e], sc, acc64[j][e]);
          acc[t][j][e] = 0.f;
        }
    }
  };

  // prologue
#pragma unroll
  for (int s = 0; s < OZ_STAGES - 1; ++s) {
    if (s < nk) load(s, s);
    cp_commit();
  }
  const int steps_per_chunk = OZ_CHUNK / OZ_BK;
  for (int kt = 0; kt < nk; ++kt) {
    cp_wait<OZ_STAGES - 2>();
    __syncthreads();
    {
      const int nt = kt + OZ_STAGES - 1;
      if (nt < nk) load(nt % OZ_STAGES, nt);
      cp_commit();
    }
    const int st = kt % OZ_STAGES;
#pragma unroll
    for (int kk = 0; kk < OZ_BK; kk += 16) {
      uint32_t af[OZ_S][4], xf[OZ_S][4];
      // A: rows 16 wr + (lane & 15), k kk + 8 (lane >> 4); X: lambda rows 16 wc + ..., same k pattern
      const int ar = wr * 16 + (lane & 15), ac = kk + (lane >> 4) * 8;
      const int xr = wc * 16 + (lane & 7) + ((lane >> 4) << 3), xc = kk + ((lane >> 3) & 1) * 8;
#pragma unroll
      for (int p = 0; p < OZ_S; ++p) {
        ldsm_x4(af[p], &S.a[st][p][ar][ac]);
        ldsm_x4(xf[p], &S.x[st][p][xr][xc]);
      }
#pragma unroll
      for (int p = 0; p < OZ_S; ++p)
#pragma unroll
        for (int q = 0; q < OZ_S - p; ++q) {
          mma_bf16(acc[p + q][0], af[p], xf[q][0], xf[q][1]);
          mma_bf16(acc[p + q][1], af[p], xf[q][2], xf[q][3]);
        }
    }
    if ((kt + 1) % steps_per_chunk == 0 || kt + 1 == nk) flush();
  }
  cp_wait<0>();

  // epilogue: fragment (row g = lane / 4 (+8), col 2 (lane % 4) (+1)) of each n8 tile
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t i = i0 + wr * 16 + (lane >> 2) + ((e >> 1) << 3);
      const int64_t l = l0 + wc * 16 + j * 8 + (lane & 3) * 2 + (e & 1);
      if (i < m && l < M) R[l * ldr + i] = b[i] - ldexp(acc64[j][e], EA[i] + EX[l]);
    }
}

// ---- the normal-equation pass -----------------------------------------------
// G = R A (g_l = A^T r_l): the slices of A here are scaled per COLUMN (the
// output index), those of R per row, so every output carries the float64
// accuracy of its own column whatever the scales of A's columns.
__device__ __forceinline__ void ldsm_x4_trans(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

constexpr int OZ_NJ = 64;           // columns of A (outputs) per CTA
constexpr int OZ_LDT = OZ_NJ + 8;   // padded smem row (bf16): 144 bytes

struct OzSmemT {
  __nv_bfloat16 a[OZ_STAGES][OZ_S][OZ_BK][OZ_LDT];  // A slices: K (rows of A) x 64 columns
  __nv_bfloat16 x[OZ_STAGES][OZ_S][OZ_BN][OZ_LDS];  // R slices: lambda rows x K
};

// partial[z][l][j] = sum_{i in split z} A[i][j] R[l][i] for j < n, l < M, from
// the slices of A (OZ_S planes m x kpA, column exponents EC) and of R (OZ_S
// planes M x kpR, row exponents EX).  Split z covers rows [z kps, (z+1) kps)
// of A, kps a multiple of 128.  CTA: 64 columns x 32 lambda; warps 4 x 2.
__global__ void __launch_bounds__(256, 1)
    k_oz_normal(const __nv_bfloat16* __restrict__ As, const int* __restrict__ EC, int64_t m, int64_t n, int64_t kpA,
                const __nv_bfloat16* __restrict__ Rs, const int* __restrict__ EX, int64_t M, int64_t kpR,
                int64_t kps, double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char oz_raw_t[];
  OzSmemT& S = *reinterpret_cast<OzSmemT*>(oz_raw_t);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int wr = w & 3, wc = w >> 2;
  const int64_t j0 = (int64_t)blockIdx.x * OZ_NJ, l0 = (int64_t)blockIdx.y * OZ_BN;
  const int64_t kb = (int64_t)blockIdx.z * kps, ke = std::min<int64_t>(m, kb + kps);
  const int64_t planeA = m * kpA, planeR = M * kpR;
  const int nk = ke > kb ? (int)((ke - kb + OZ_BK - 1) / OZ_BK) : 0;

  auto load = [&](int stage, int kt) {
    const int64_t k0 = kb + (int64_t)kt * OZ_BK;
    // A: OZ_S x 32 rows (i) x 8 chunks of 8 columns
    for (int q = tid; q < OZ_S * OZ_BK * 8; q += 256) {
      const int p = q / (OZ_BK * 8), rem = q % (OZ_BK * 8), r = rem >> 3, c = (rem & 7) * 8;
      const int64_t gi = k0 + r, gj = j0 + c;
      const bool ok = gi < ke && gj < kpA;
      cp_async16(&S.a[stage][p][r][c], ok ? (const void*)(As + p * planeA + gi * kpA + gj) : (const void*)As, ok);
    }
    // R: OZ_S x 32 lambda rows x 4 chunks of 8 values of K
    for (int q = tid; q < OZ_S * OZ_BN * 4; q += 256) {
      const int p = q / (OZ_BN * 4), rem = q % (OZ_BN * 4), r = rem >> 2, c = (rem & 3) * 8;
      const int64_t gl = l0 + r, gk = k0 + c;
      const bool ok = gl < M && gk < ke;
      cp_async16(&S.x[stage][p][r][c], ok ? (const void*)(Rs + p * planeR + gl * kpR + gk) : (const void*)Rs, ok);
    }
  };

  float acc[OZ_LV][2][4];
  double acc64[2][4];
#pragma unroll
  for (int t = 0; t < OZ_LV; ++t)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[t][j][e] = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc64[j][e] = 0.0;
  auto flush = [&]() {
#pragma unroll
    for (int t = OZ_LV - 1; t >= 0; --t) {
      const double sc = ldexp(1.0, -7 * (t + 2));
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          acc64[j][e] = fma((double)acc[t][j][e], sc, acc64[j][e]);
          acc[t][j][e] = 0.f;
        }
    }
  };

#pragma unroll
  for (int s = 0; s < OZ_STAGES - 1; ++s) {
    if (s < nk) load(s, s);
    cp_commit();
  }
  const int steps_per_chunk = OZ_CHUNK / OZ_BK;
  for (int kt = 0; kt < nk; ++kt) {
    cp_wait<OZ_STAGES - 2>();
    __syncthreads();
    {
      const int nt = kt + OZ_STAGES - 1;
      if (nt < nk) load(nt % OZ_STAGES, nt);
      cp_commit();
    }
    const int st = kt % OZ_STAGES;
#pragma unroll
    for (int kk = 0; kk < OZ_BK; kk += 16) {
      uint32_t af[OZ_S][4], xf[OZ_S][4];
      // A^T fragment (rows j, K i): transposed 8x8 loads of rows i, 8 columns j each
      const int ai = kk + (lane & 7) + ((lane >> 4) << 3), aj = wr * 16 + ((lane >> 3) & 1) * 8;
      const int xr = wc * 16 + (lane & 7) + ((lane >> 4) << 3), xc = kk + ((lane >> 3) & 1) * 8;
#pragma unroll
      for (int p = 0; p < OZ_S; ++p) {
        ldsm_x4_trans(af[p], &S.a[st][p][ai][aj]);
        ldsm_x4(xf[p], &S.x[st][p][xr][xc]);
      }
#pragma unroll
      for (int p = 0; p < OZ_S; ++p)
#pragma unroll
        for (int q = 0; q < OZ_S - p; ++q) {
          mma_bf16(acc[p + q][0], af[p], xf[q][0], xf[q][1]);
          mma_bf16(acc[p + q][1], af[p], xf[q][2], xf[q][3]);
        }
    }
    if ((kt + 1) % steps_per_chunk == 0 || kt + 1 == nk) flush();
  }
  cp_wait<0>();
  double* P = partial + (int64_t)blockIdx.z * M * n;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t jj = j0 + wr * 16 + (lane >> 2) + ((e >> 1) << 3);
      const int64_t l = l0 + wc * 16 + j * 8 + (lane & 3) * 2 + (e & 1);
      if (jj < n && l < M) P[l * n + jj] = ldexp(acc64[j][e], EX[l] + EC[jj]);
    }
}

}  // namespace

size_t oz_slices_bytes(int64_t rows, int64_t cols) {
  return sizeof(__nv_bfloat16) * (size_t)OZ_S * (size_t)rows * (size_t)(cdiv(cols, 8) * 8);
}

tk_status oz_prepare(const void* X, tk_dtype dt, int64_t rows, int64_t cols, int64_t ld, void* slices, int* E,
                     cudaStream_t st) {
  if (rows == 0 || cols == 0) return TK_OK;
  const int64_t kp = cdiv(cols, 8) * 8;
  const unsigned gr = (unsigned)cdiv(rows, 8);
  const unsigned gs = (unsigned)std::min<int64_t>(cdiv(rows * kp, 256), 152 * 32);
  __nv_bfloat16* out = static_cast<__nv_bfloat16*>(slices);
  if (dt == TK_F64) {
    k_oz_rowexp<double><<<gr, 256, 0, st>>>((const double*)X, rows, cols, ld, E);
    TK_LAUNCH_CHECK();
    k_oz_slice<double, false><<<gs, 256, 0, st>>>((const double*)X, rows, cols, ld, E, kp, out);
  } else {
    k_oz_rowexp<float><<<gr, 256, 0, st>>>((const float*)X, rows, cols, ld, E);
    TK_LAUNCH_CHECK();
    k_oz_slice<float, false><<<gs, 256, 0, st>>>((const float*)X, rows, cols, ld, E, kp, out);
  }
  TK_LAUNCH_CHECK();
  return TK_OK;
}

size_t oz_colmax_bytes(int64_t cols) { return sizeof(unsigned long long) * (size_t)std::max<int64_t>(cols, 1); }

tk_status oz_prepare_cols(const void* X, tk_dtype dt, int64_t rows, int64_t cols, int64_t ld, void* slices, int* E,
                          void* colmax, cudaStream_t st) {
  if (rows == 0 || cols == 0) return TK_OK;
  const int64_t kp = cdiv(cols, 8) * 8;
  unsigned long long* mx = static_cast<unsigned long long*>(colmax);
  TK_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * (size_t)cols, st));
  // about 4 CTAs of 256 columns per SM, each over a band of rows
  const int64_t cb = cdiv(cols, 256);
  const int64_t bands = std::max<int64_t>(1, std::min<int64_t>(cdiv(4 * 152, cb), cdiv(rows, 64)));
  const int64_t rows_per = cdiv(rows, bands);
  const dim3 gm((unsigned)cb, (unsigned)cdiv(rows, rows_per));
  const unsigned gs = (unsigned)std::min<int64_t>(cdiv(rows * kp, 256), 152 * 32);
  __nv_bfloat16* out = static_cast<__nv_bfloat16*>(slices);
  if (dt == TK_F64) k_oz_colmax<double><<<gm, 256, 0, st>>>((const double*)X, rows, cols, ld, rows_per, mx);
  else k_oz_colmax<float><<<gm, 256, 0, st>>>((const float*)X, rows, cols, ld, rows_per, mx);
  TK_LAUNCH_CHECK();
  k_oz_colexp<<<(unsigned)cb, 256, 0, st>>>(mx, cols, E);
  TK_LAUNCH_CHECK();
  if (dt == TK_F64) k_oz_slice<double, true><<<gs, 256, 0, st>>>((const double*)X, rows, cols, ld, E, kp, out);
  else k_oz_slice<float, true><<<gs, 256, 0, st>>>((const float*)X, rows, cols, ld, E, kp, out);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

tk_status oz_residual(const void* Aslices, const int* EA, int64_t m, int64_t n, const void* Xslices, const int* EX,
                      int64_t M, const double* b, double* R, int64_t ldr, cudaStream_t st) {
  if (m == 0 || M == 0) return TK_OK;
  const int64_t kp = cdiv(n, 8) * 8;
  const size_t smem = sizeof(OzSmem);
  TK_CUDA(cudaFuncSetAttribute(k_oz_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(OzSmem)));
  const dim3 grid((unsigned)cdiv(m, OZ_BM), (unsigned)cdiv(M, OZ_BN));
  k_oz_residual<<<grid, 256, smem, st>>>(static_cast<const __nv_bfloat16*>(Aslices), EA, m, kp,
                                        static_cast<const __nv_bfloat16*>(Xslices), EX, M, b, R, ldr);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

int oz_normal_splits(int64_t m, int64_t n, int64_t M) {
  const int64_t tiles = cdiv(n, OZ_NJ) * cdiv(M, OZ_BN);
  const int64_t want = cdiv(4 * 152, std::max<int64_t>(tiles, 1));  // one CTA per SM: four full waves
  const int64_t maxs = std::max<int64_t>(1, cdiv(m, OZ_CHUNK));
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, maxs));
}

tk_status oz_normal(const void* AslicesC, const int* EC, int64_t m, int64_t n, const double* R, int64_t ldr,
                    int64_t M, void* Rslices, int* EX, double* partial, int splits, cudaStream_t st) {
  if (M == 0 || n == 0) return TK_OK;
  const int64_t kpA = cdiv(n, 8) * 8, kpR = cdiv(m, 8) * 8;
  TK_TRY(oz_prepare(R, TK_F64, M, m, ldr, Rslices, EX, st));
  const int64_t kps = cdiv(cdiv(m, splits), OZ_CHUNK) * OZ_CHUNK;
  const int sp = (int)cdiv(m, kps);
  TK_CUDA(cudaFuncSetAttribute(k_oz_normal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(OzSmemT)));
  const dim3 grid((unsigned)cdiv(n, OZ_NJ), (unsigned)cdiv(M, OZ_BN), (unsigned)sp);
  k_oz_normal<<<grid, 256, sizeof(OzSmemT), st>>>(static_cast<const __nv_bfloat16*>(AslicesC), EC, m, n, kpA,
                                                  static_cast<const __nv_bfloat16*>(Rslices), EX, M, kpR, kps,
                                                  partial);
  TK_LAUNCH_CHECK();
  if (sp < splits) {  // the caller sums `splits` planes: the unused ones are zero
    TK_CUDA(cudaMemsetAsync(partial + (int64_t)sp * M * n, 0, sizeof(double) * (size_t)(splits - sp) * M * n, st));
  }
  return TK_OK;
}

}  // namespace tk
