// Gaussian sketch on the 5th-generation tensor cores (the mixed form,
// Section 2.1.1's Gaussian embedding): Y = G A with G (s x m) of N(0, 1/s)
// entries and A (m x n), both rounded to BF16, FP32 accumulation.  A sketch
// only has to be an embedding, so BF16 inputs suffice; Y is then widened to
// float64 for the Gram matrix and the Cholesky factors.
//
// Structure (one 128 x 256 output tile per CTA, 128 threads):
//   * G (s x ldk) and A^T (n x ldk) are first written as K-major BF16 (ldk =
//     m rounded up to 8, zero padded) so both MMA operands are K-major.
//   * warp 0 / lane 0 streams 64-wide K slabs of both operands into a 4-stage
//     ring with TMA (cp.async.bulk.tensor, 128-byte swizzle), completion on
//     a per-stage "full" mbarrier;
//   * warp 1 / lane 0 issues tcgen05.mma (M = 128, N = 256, K = 16, kind::f16)
//     into a 128 x 256 FP32 accumulator in tensor memory and releases each
//     stage with tcgen05.commit on its "empty" mbarrier;
//   * all four warps read the accumulator back with tcgen05.ld (32 lanes x 32
//     columns per load) and store Y.
// Every mbarrier wait is bounded; a wait that gives up sets an error flag,
// the other roles see it and stop, the tensor memory is freed and the kernel
// returns (the host reports TK_ETIMEOUT).
#include <cuda.h>
#include <cuda_bf16.h>

#include "tk_internal.cuh"
#include "tk_tcgen05.cuh"

namespace tk {
namespace {

constexpr int TC_M = 128;       // tile rows (of G / Y)
constexpr int TC_N = 256;       // tile columns (of Y)
constexpr int TC_K = 64;        // K per stage: 64 BF16 = 128 bytes per row
constexpr int TC_STAGES = 4;
constexpr uint32_t TC_A_BYTES = TC_M * TC_K * 2;  // 16 KiB
constexpr uint32_t TC_B_BYTES = TC_N * TC_K * 2;  // 32 KiB
constexpr uint32_t TC_TMEM_COLS = 256;            // FP32 accumulator: 128 lanes x 256 columns

struct TcSmem {
  uint8_t a[TC_STAGES][TC_A_BYTES];
  uint8_t b[TC_STAGES][TC_B_BYTES];
  uint64_t full[TC_STAGES];
  uint64_t empty[TC_STAGES];
  uint64_t accum;
  uint32_t tmem_base;
};

__global__ void __launch_bounds__(128, 1)
    k_tc_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t M,
                   int64_t N, int64_t K, double* __restrict__ Y, int64_t ldy, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = (int)blockIdx.x * TC_M, n0 = (int)blockIdx.y * TC_N;
  const int nk = (int)((K + TC_K - 1) / TC_K);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0 && lane == 0) {
    // TMA producer
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % TC_STAGES;
      const uint32_t ph = (uint32_t)(kb / TC_STAGES) & 1u;
      if (!mbar_wait(&S.empty[s], ph ^ 1u, err)) break;
      mbar_expect_tx(&S.full[s], TC_A_BYTES + TC_B_BYTES);
      tma_load_2d(&tmA, &S.full[s], S.a[s], kb * TC_K, m0);
      tma_load_2d(&tmB, &S.full[s], S.b[s], kb * TC_K, n0);
      ++issued;
    }
    if (*(volatile int*)err) tma_drain_ring(S.full, TC_STAGES, issued);  // no copy lands after the exit
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(TC_M, TC_N);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % TC_STAGES;
      const uint32_t ph = (uint32_t)(kb / TC_STAGES) & 1u;
      if (!mbar_wait(&S.full[s], ph, err)) break;
      tc_fence_after();
      const uint64_t ad = sdesc_sw128(smem_u32(S.a[s]));
      const uint64_t bd = sdesc_sw128(smem_u32(S.b[s]));
#pragma unroll
      for (int k = 0; k < TC_K / 16; ++k) {
        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
        // K = 16 BF16 = 32 bytes further along the 128-byte row: +2 in the >>4 address field
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(ad + 2ull * k), "l"(bd + 2ull * k), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&S.empty[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&S.accum))
                 : "memory");
  }
  __syncwarp();

  // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w+31
  const bool ok = mbar_wait(&S.accum, 0u, err);
  if (!ok) mbar_drain(&S.accum, 0u);  // gave up: the issued MMAs finish before tensor memory is freed
  tc_fence_after();
  if (ok) {
    const int64_t row = (int64_t)m0 + warp * 32 + lane;
    for (int c = 0; c < TC_N; c += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int64_t col = (int64_t)n0 + c + j;
          if (col < N) Y[row * ldy + col] = (double)__uint_as_float(r[j]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// G (s x ldk) BF16, entry (i, k) = N(0, 1/s) draw number i*m + k of Philox
// stream 2 (the same counter convention as the float64 sketch, generated in
// float32), zero for k >= m.
__global__ void k_gauss_bf16(uint64_t seed, int64_t s, int64_t m, int64_t ldk, float inv_sqrt_s,
                             __nv_bfloat16* __restrict__ G) {
  const int64_t total = s * ldk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ldk, k = e - i * ldk;
    float v = 0.f;
    if (k < m) {
      const uint64_t idx = (uint64_t)(i * m + k);
      const uint4 w = philox(idx >> 2, STREAM_GAUSS, seed);
      const int lane = (int)(idx & 3u);
      const uint32_t a = (lane < 2) ? w.x : w.z, b = (lane < 2) ? w.y : w.w;
      const float u1 = ((float)a + 1.0f) * 2.3283064365386962890625e-10f;
      const float u2 = (float)b * 2.3283064365386962890625e-10f;
      const float r = sqrtf(-2.0f * logf(u1));
      float sn, cs;
      sincospif(2.0f * u2, &sn, &cs);
      v = ((lane & 1) ? r * sn : r * cs) * inv_sqrt_s;
    }
    G[e] = __float2bfloat16_rn(v);
  }
}

// AT (n x ldk) BF16 = A^T, zero for k >= m.  32 x 32 tiles through shared memory.
template <typename T>
__global__ void k_transpose_bf16(const T* __restrict__ A, int64_t m, int64_t n, int64_t lda, int64_t ldk,
                                 __nv_bfloat16* __restrict__ AT) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;  // rows of A = k, cols = j
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < m && c < n) ? (float)A[r * lda + c] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t j = c0 + y, k = r0 + threadIdx.x;
    if (j < n && k < ldk) AT[j * ldk + k] = __float2bfloat16_rn(t[threadIdx.x][y]);
  }
}

// 2D BF16 K-major map: rows x ldk elements, box = 64 (K) x box_rows, 128-byte swizzle.
tk_status make_map(CUtensorMap* map, void* base, int64_t rows, int64_t ldk, uint32_t box_rows) {
  EncodeTiledFn fn;
  TK_TRY(encode_fn(&fn));
  const cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TC_K, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error_msg("cuTensorMapEncodeTiled rejected the operand layout");
    return TK_ECUDA;
  }
  return TK_OK;
}

// ---------------------------------------------------------------------------
// LSQR products on the tensor cores with the 3-term TF32 split
//   D (rows x N) = X_tile (rows x K) L^T,   L = lambda-major (N_act x K)
// X is float32 K-major: A itself (product with A^T: rows of A) or a float32
// copy of A^T (product with A).  tf32 MMAs read the top 19 bits of each float,
// so with X = Xh + Xl (Xl = X - tf32(X)) and L = Lh + Ll,
//   D ~= Xh Lh + Xh Ll + Xl Lh      (error ~ 2^-22 |X||L|, float32 level).
// Xl is formed in shared memory by four converter warps from the TMA tile;
// Ll is formed once per call in global memory.  Epilogue: the lambda-major
// update U = D^T + coef .* U (A W product) or a split-K partial (A^T U).
constexpr int T3_M = 128;         // rows of X per tile
constexpr int T3_K = 32;          // K per stage: 32 floats = 128 bytes per row
constexpr int T3_STAGES = 4;
constexpr uint32_t T3_X_BYTES = T3_M * T3_K * 4;  // 16 KiB

template <int NP>  // lambda columns, padded to a multiple of 16 (<= 64)
struct T3Smem {
  uint8_t xh[T3_STAGES][T3_X_BYTES];
  uint8_t xl[T3_STAGES][T3_X_BYTES];
  uint8_t lh[T3_STAGES][NP * 128];
  uint8_t ll[T3_STAGES][NP * 128];
  uint64_t full[T3_STAGES];
  uint64_t lo_ready[T3_STAGES];
  uint64_t empty[T3_STAGES];
  uint64_t accum;
  uint32_t tmem_base;
};

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

template <int NP, bool UPDATE>
__global__ void __launch_bounds__(256, 1)
    k_tc_lmaj_tf32x3(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmLh,
                     const __grid_constant__ CUtensorMap tmLl, int64_t rows, int N, int64_t k_per_split,
                     int64_t K, float* __restrict__ U, int64_t ldu, const double* __restrict__ coef,
                     double* __restrict__ partial, int* __restrict__ err) {
  constexpr uint32_t TMEM_COLS = NP <= 32 ? 32 : 64;
  constexpr uint32_t L_BYTES = NP * 128;
  extern __shared__ __align__(1024) uint8_t t3_smem_raw[];
  T3Smem<NP>& S = *reinterpret_cast<T3Smem<NP>*>((reinterpret_cast<uintptr_t>(t3_smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * T3_M;
  const int64_t kbeg = (int64_t)blockIdx.y * k_per_split;
  const int64_t kend = std::min(K, kbeg + k_per_split);
  const int nk = kend > kbeg ? (int)((kend - kbeg + T3_K - 1) / T3_K) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < T3_STAGES; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.lo_ready[s], 128);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % T3_STAGES;
      const uint32_t ph = (uint32_t)(kb / T3_STAGES) & 1u;
      if (!mbar_wait(&S.empty[s], ph ^ 1u, err)) break;
      mbar_expect_tx(&S.full[s], T3_X_BYTES + 2 * L_BYTES);
      const int kc = (int)(kbeg + (int64_t)kb * T3_K);
      tma_load_2d(&tmX, &S.full[s], S.xh[s], kc, (int)r0);
      tma_load_2d(&tmLh, &S.full[s], S.lh[s], kc, 0);
      tma_load_2d(&tmLl, &S.full[s], S.ll[s], kc, 0);
      ++issued;
    }
    if (*(volatile int*)err) tma_drain_ring(S.full, T3_STAGES, issued);  // no copy lands after the exit
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_tf32(T3_M, NP);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % T3_STAGES;
      const uint32_t ph = (uint32_t)(kb / T3_STAGES) & 1u;
      if (!mbar_wait(&S.lo_ready[s], ph, err)) break;
      tc_fence_after();
      const uint64_t xh = sdesc_sw128(smem_u32(S.xh[s])), xl = sdesc_sw128(smem_u32(S.xl[s]));
      const uint64_t lh = sdesc_sw128(smem_u32(S.lh[s])), ll = sdesc_sw128(smem_u32(S.ll[s]));
#pragma unroll
      for (int k = 0; k < T3_K / 8; ++k) {  // K = 8 floats = 32 bytes per MMA
        const uint64_t o = 2ull * k;
        const uint32_t first = (kb == 0 && k == 0) ? 0u : 1u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(xh + o), "l"(lh + o), "r"(idesc), "r"(first)
            : "memory");
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(xh + o), "l"(ll + o), "r"(idesc), "r"(1u)
            : "memory");
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(xl + o), "l"(lh + o), "r"(idesc), "r"(1u)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&S.empty[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&S.accum))
                 : "memory");
  } else if (warp >= 4) {
    // converters: Xl = X - tf32(X), element by element at the same byte offset
    // (the swizzle permutes 16-byte chunks, so positions need no decoding)
    const int t = threadIdx.x - 128;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % T3_STAGES;
      const uint32_t ph = (uint32_t)(kb / T3_STAGES) & 1u;
      if (!mbar_wait(&S.full[s], ph, err)) break;
      const float4* src = reinterpret_cast<const float4*>(S.xh[s]);
      float4* dst = reinterpret_cast<float4*>(S.xl[s]);
#pragma unroll
      for (int q = t; q < (int)(T3_X_BYTES / 16); q += 128) {
        const float4 v = src[q];
        dst[q] = make_float4(v.x - tf32_trunc(v.x), v.y - tf32_trunc(v.y), v.z - tf32_trunc(v.z),
                             v.w - tf32_trunc(v.w));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core reads
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&S.lo_ready[s])) : "memory");
    }
  }
  __syncwarp();

  // epilogue (warps 0-3: accumulator lanes 32w .. 32w+31 = rows of this tile)
  const bool ok = (warp < 4) ? mbar_wait(&S.accum, 0u, err) : true;
  if (!ok) mbar_drain(&S.accum, 0u);  // gave up: the issued MMAs finish before tensor memory is freed
  tc_fence_after();
  if (warp < 4 && ok) {
    const int64_t row = r0 + warp * 32 + lane;
    for (int c = 0; c < NP; c += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
      if (row < rows) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int l = c + j;
          if (l < N) {
            const float d = nk > 0 ? __uint_as_float(r[j]) : 0.f;  // an empty K split contributes zero
            if (UPDATE) {
              float* u = U + (int64_t)l * ldu + row;
              *u = (float)((double)d + coef[l] * (double)(*u));
            } else {
              partial[((int64_t)blockIdx.y * N + l) * rows + row] = (double)d;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Ll = L - tf32(L)  (the low half of the lambda-major operand)
__global__ void k_tf32_lo(const float* __restrict__ L, int64_t total, float* __restrict__ Ll) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = L[i];
    Ll[i] = v - tf32_trunc(v);
  }
}

tk_status make_map_f32(CUtensorMap* map, const void* base, int64_t rows, int64_t ld, int64_t cols, uint32_t box_rows) {
  EncodeTiledFn fn;
  TK_TRY(encode_fn(&fn));
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)T3_K, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error_msg("cuTensorMapEncodeTiled rejected the float32 operand layout");
    return TK_ECUDA;
  }
  return TK_OK;
}

template <int NP, bool UPDATE>
tk_status launch_t3(const CUtensorMap& mX, const CUtensorMap& mLh, const CUtensorMap& mLl, int64_t rows, int N,
                    int64_t kps, int64_t K, int splits, float* U, int64_t ldu, const double* coef, double* partial,
                    int* err, cudaStream_t st) {
  const size_t smem = sizeof(T3Smem<NP>) + 1024;
  auto kern = k_tc_lmaj_tf32x3<NP, UPDATE>;
  TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)cdiv(rows, T3_M), (unsigned)splits);
  kern<<<grid, 256, smem, st>>>(mX, mLh, mLl, rows, N, kps, K, U, ldu, coef, partial, err);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

}  // namespace

size_t tc_sketch_workspace(int64_t m, int64_t n, int64_t s) {
  const int64_t ldk = cdiv(m, 8) * 8;
  Arena a;
  a.take<__nv_bfloat16>((size_t)s * ldk);
  a.take<__nv_bfloat16>((size_t)n * ldk);
  a.take<int>(4);
  return a.used + 2048;
}

// Y (s x n, float64) = G A with G, A rounded to BF16 (Gaussian embedding of the mixed form).
tk_status tc_gauss_sketch(const void* A, tk_dtype dt, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                          double* Y, Arena& ar, cudaStream_t st) {
  const int64_t ldk = cdiv(m, 8) * 8;  // 16-byte aligned BF16 rows for TMA
  __nv_bfloat16* G = ar.take<__nv_bfloat16>((size_t)s * ldk);
  __nv_bfloat16* AT = ar.take<__nv_bfloat16>((size_t)n * ldk);
  int* err = ar.take<int>(4);
  if (!ar.ok()) return TK_ENOMEM;
  if (s <= 0 || n <= 0) return TK_OK;
  if (s > (int64_t)INT32_MAX - TC_M || n > (int64_t)INT32_MAX - TC_N || ldk > (int64_t)INT32_MAX) {
    set_error_msg("tensor-core sketch: dimensions exceed the 32-bit TMA coordinates");
    return TK_EINVAL;
  }
  const int64_t total = s * ldk;
  k_gauss_bf16<<<(unsigned)std::min<int64_t>(cdiv(total, 256), 152 * 64), 256, 0, st>>>(
      seed, s, m, ldk, (float)(1.0 / sqrt((double)s)), G);
  TK_LAUNCH_CHECK();
  dim3 tg((unsigned)cdiv(n, 32), (unsigned)cdiv(ldk, 32));
  if (tg.y > 65535u) {
    set_error_msg("tensor-core sketch: m too large for the transpose grid");
    return TK_EINVAL;
  }
  if (dt == TK_F64) k_transpose_bf16<double><<<tg, dim3(32, 8), 0, st>>>((const double*)A, m, n, lda, ldk, AT);
  else k_transpose_bf16<float><<<tg, dim3(32, 8), 0, st>>>((const float*)A, m, n, lda, ldk, AT);
  TK_LAUNCH_CHECK();
  CUtensorMap mA, mB;
  TK_TRY(make_map(&mA, G, s, ldk, TC_M));
  TK_TRY(make_map(&mB, AT, n, ldk, TC_N));
  TK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  const size_t smem = sizeof(TcSmem) + 1024;
  TK_CUDA(cudaFuncSetAttribute(k_tc_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)cdiv(s, TC_M), (unsigned)cdiv(n, TC_N));
  k_tc_gemm_bf16<<<grid, 128, smem, st>>>(mA, mB, s, n, ldk, Y, n, err);
  TK_LAUNCH_CHECK();
  int herr = 0;
  TK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    set_error_msg("tensor-core sketch: a pipeline wait timed out");
    return TK_ETIMEOUT;
  }
  return TK_OK;
}

}  // namespace tk

namespace tk {

size_t tc_lmaj_workspace(int N_cap, int64_t K) {
  Arena a;
  a.take<float>((size_t)N_cap * K);  // low half of the lambda-major operand
  a.take<int>(4);
  return a.used + 1024;
}

// D = X L^T on the tensor cores (3-term TF32).  X: rows x K float32 (row stride
// ldx, 16-byte multiple), L: N x K float32 lambda-major (row stride ldl).
// UPDATE: U[l][r] = D[r][l] + coef[l] U[l][r]; else partial[z][l][r] = D[r][l]
// for the K split z.  scratch: tc_lmaj_workspace(N, K) bytes.
tk_status tc_lmaj_product(bool update, const float* X, int64_t rows, int64_t K, int64_t ldx, const float* L,
                          int64_t ldl, int N, float* U, int64_t ldu, const double* coef, double* partial, int splits,
                          void* scratch, cudaStream_t st) {
  if (N < 1 || N > 64) {
    set_error_msg("tensor-core LSQR product: 1..64 lambda per pass");
    return TK_EINVAL;
  }
  if ((ldx % 4) || (ldl % 4) || ((uintptr_t)X % 16) || ((uintptr_t)L % 16) || rows > INT32_MAX || K > INT32_MAX) {
    set_error_msg("tensor-core LSQR product: operands must have 16-byte aligned rows");
    return TK_EINVAL;
  }
  Arena a;
  a.base = (char*)scratch;
  a.cap = tc_lmaj_workspace(N, K);
  float* Ll = a.take<float>((size_t)N * K);
  int* err = a.take<int>(4);
  // the low half is packed with row stride K
  {
    // copy-with-stride into Ll: Ll[l][k] = L[l][k] - tf32(L[l][k])
    const int64_t total = (int64_t)N * K;
    if (ldl == K) {
      k_tf32_lo<<<(unsigned)std::min<int64_t>(cdiv(total, 256), 152 * 8), 256, 0, st>>>(L, total, Ll);
      TK_LAUNCH_CHECK();
    } else {
      for (int l = 0; l < N; ++l) {
        k_tf32_lo<<<(unsigned)std::min<int64_t>(cdiv(K, 256), 152), 256, 0, st>>>(L + (int64_t)l * ldl, K, Ll + (int64_t)l * K);
        TK_LAUNCH_CHECK();
      }
    }
  }
  const int NP = N <= 32 ? (N <= 16 ? 16 : 32) : (N <= 48 ? 48 : 64);
  CUtensorMap mX, mLh, mLl;
  TK_TRY(make_map_f32(&mX, X, rows, ldx, K, T3_M));
  TK_TRY(make_map_f32(&mLh, L, N, ldl, K, (uint32_t)NP));
  TK_TRY(make_map_f32(&mLl, Ll, N, K, K, (uint32_t)NP));
  TK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  const int sp = update ? 1 : std::max(1, splits);
  int64_t kps = cdiv(cdiv(K, sp), T3_K) * T3_K;
#define TK_T3(NPV)                                                                                                 \
  do {                                                                                                             \
    if (update) TK_TRY((launch_t3<NPV, true>(mX, mLh, mLl, rows, N, kps, K, sp, U, ldu, coef, nullptr, err, st))); \
    else TK_TRY((launch_t3<NPV, false>(mX, mLh, mLl, rows, N, kps, K, sp, nullptr, 0, nullptr, partial, err, st))); \
  } while (0)
  switch (NP) {
    case 16: TK_T3(16); break;
    case 32: TK_T3(32); break;
    case 48: TK_T3(48); break;
    default: TK_T3(64); break;
  }
#undef TK_T3
  return TK_OK;
}

// Error flag of the last tensor-core LSQR product (1 = a pipeline wait timed out).
tk_status tc_lmaj_check(void* scratch, int N, int64_t K, cudaStream_t st) {
  Arena a;
  a.base = (char*)scratch;
  a.cap = tc_lmaj_workspace(N, K);
  a.take<float>((size_t)N * K);
  int* err = a.take<int>(4);
  int h = 0;
  TK_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  if (h) {
    set_error_msg("tensor-core LSQR product: a pipeline wait timed out");
    return TK_ETIMEOUT;
  }
  return TK_OK;
}

}  // namespace tk

// ---- the bounded wait on its own ------------------------------------------------
// One thread waits on a freshly initialized mbarrier that nothing arrives at:
// its first phase never completes, so the wait must give up after budget_ns
// and set the error word, exactly as a stuck pipeline stage of the kernels
// above would.  Nothing is in flight (no copy, no MMA, no tensor memory).
namespace tk {
namespace {
__global__ void k_wait_selftest(uint64_t budget_ns, int* __restrict__ err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) (void)mbar_wait_for(&bar, 0u, err, budget_ns);
}
}  // namespace
}  // namespace tk

extern "C" TK_API tk_status tk_wait_selftest(int64_t budget_us, void* work, size_t work_bytes, void* stream) {
  using namespace tk;
  if (budget_us < 1 || budget_us > 2000000) {
    set_error_msg("tk_wait_selftest: budget_us must be in [1, 2000000]");
    return TK_EINVAL;
  }
  if (!work || work_bytes < 16) {
    set_error_msg("tk_wait_selftest: work must hold at least 16 bytes");
    return TK_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* err = static_cast<int*>(work);
  TK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  k_wait_selftest<<<1, 32, 0, st>>>((uint64_t)budget_us * 1000ull, err);
  TK_LAUNCH_CHECK();
  int h = 0;
  TK_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  if (h) {
    set_error_msg("tk_wait_selftest: the bounded wait gave up as it should");
    return TK_ETIMEOUT;
  }
  return TK_OK;
}
