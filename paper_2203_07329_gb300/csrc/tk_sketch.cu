// Sketch of A (Section 2.1.1; Algorithm 1 step 2 / Algorithm 2 step 2).
//
// Every sketch here acts along the long axis of an L x cols row-major matrix
// (the overdetermined A directly; the underdetermined A after a transpose, so
// that Y = A X becomes Y^T = X^T A^T with the same kernels).
//
// SRHT: Y = sqrt(Lp/s) S (H/sqrt(Lp)) D [A; 0] = (1/sqrt(s)) S H D [A; 0].
//   H_Lp (Sylvester) factors as a product of butterfly levels over the bits
//   of the row index.  Each pass loads a tile of 2^t rows (rows that differ
//   only in t consecutive index bits) x CB columns into shared memory, runs
//   the t butterfly levels there, and writes it back: log2(Lp)/9 passes over
//   the data instead of log2(Lp).  The first pass applies D while loading
//   (rows >= L read as zero); the last pass writes only the sampled rows.
// Gaussian: Y = G A with G (s x L) of N(0, 1/s) entries from Philox stream 2,
//   generated into the workspace, then a plain GEMM.
#include <algorithm>
#include <type_traits>

#include "tk_internal.cuh"

namespace tk {
namespace {

constexpr int kFwhtThreads = 256;
constexpr int kFwhtMaxBits = 9;

// Tile width: 128 bytes of one row (16 doubles or 32 floats); a power of two,
// so every index below is a shift or a mask.
template <typename TC>
constexpr int fwht_cb() {
  return (int)(128 / sizeof(TC));
}
template <typename TC>
constexpr int fwht_lcb() {
  return sizeof(TC) == 8 ? 4 : 5;
}

template <typename TIn, typename TC, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kFwhtThreads)
    k_fwht_pass(const TIn* src, int64_t ld_src, TC* dst, double* __restrict__ Y,
                const int8_t* __restrict__ signs, const int32_t* __restrict__ rowmap, int64_t L, int64_t cols,
                int b0, int t, int64_t ncb, double scale) {
  constexpr int CB = fwht_cb<TC>(), LCB = fwht_lcb<TC>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* tile = reinterpret_cast<TC*>(smem_raw);
  const int64_t g = blockIdx.x / ncb;
  const int64_t cb = blockIdx.x - g * ncb;
  const int64_t lo = g & ((int64_t(1) << b0) - 1);
  const int64_t hi = g >> b0;
  const int rows_t = 1 << t;
  const int64_t c0 = cb * CB;
  const int tile_elems = rows_t << LCB;
  for (int idx = threadIdx.x; idx < tile_elems; idx += blockDim.x) {
    const int mid = idx >> LCB, c = idx & (CB - 1);
    const int64_t r = (hi << (b0 + t)) | ((int64_t)mid << b0) | lo;
    const int64_t col = c0 + c;
    TC v = TC(0);
    if (col < cols) {
      if (FIRST) {
        if (r < L) v = (TC)src[r * ld_src + col] * (TC)signs[r];
      } else {
        v = (TC)src[r * ld_src + col];
      }
    }
    tile[idx] = v;
  }
  __syncthreads();
  const int pairs = (rows_t >> 1) << LCB;
  for (int lv = 0; lv < t; ++lv) {
    const int h = 1 << lv;
    for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
      const int q = p >> LCB, c = p & (CB - 1);
      const int i = ((q >> lv) << (lv + 1)) | (q & (h - 1));  // rows i and i + h differ in bit lv
      TC* a = tile + (i << LCB) + c;
      TC* b = a + (h << LCB);
      const TC x = *a, y = *b;
      *a = x + y;
      *b = x - y;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < tile_elems; idx += blockDim.x) {
    const int mid = idx >> LCB, c = idx & (CB - 1);
    const int64_t r = (hi << (b0 + t)) | ((int64_t)mid << b0) | lo;
    const int64_t col = c0 + c;
    if (col >= cols) continue;
    if (LAST) {
      const int32_t k = rowmap[r];
      if (k >= 0) Y[(int64_t)k * cols + col] = scale * (double)tile[idx];
    } else {
      dst[r * cols + col] = tile[idx];
    }
  }
}

// The same pass with the butterflies in registers.  A tile is 2^t rows x 32
// columns (t = R1 + 3); warp w, lane c own column c.  Phase 1: thread (w, c)
// loads rows (w << R1) | b, b < 2^R1, straight from global memory (each load
// instruction is one 32-column row segment of the warp) and runs the R1 low
// levels in registers.  One exchange through shared memory regroups the rows
// as (k << R1) | j (k < 8, 2^(R1-3) values of j per warp), the 3 top levels run
// in registers, and the rows go straight back to global memory.  Shared
// memory is written and read once per tile instead of once per level.
template <typename TIn, typename TC, bool FIRST, bool LAST, int R1>
__global__ void __launch_bounds__(256)
    k_fwht_reg(const TIn* src, int64_t ld_src, TC* dst, double* __restrict__ Y, const int8_t* __restrict__ signs,
               const int32_t* __restrict__ rowmap, int64_t L, int64_t cols, int b0, int64_t ncb, double scale) {
  constexpr int T = R1 + 3, NR = 1 << R1, NJ = NR >> 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* tile = reinterpret_cast<TC*>(smem_raw);  // [2^T rows][33] (padded: conflict-free transposed reads)
  const int64_t g = blockIdx.x / ncb;
  const int64_t cb = blockIdx.x - g * ncb;
  const int64_t lo = g & ((int64_t(1) << b0) - 1);
  const int64_t hi = g >> b0;
  const int w = threadIdx.x >> 5, c = threadIdx.x & 31;
  const int64_t col = cb * 32 + c;
  const bool cok = col < cols;
  auto grow = [&](int mid) -> int64_t { return (hi << (b0 + T)) | ((int64_t)mid << b0) | lo; };
  TC v[NR];
#pragma unroll
  for (int b = 0; b < NR; ++b) {
    const int64_t r = grow((w << R1) | b);
    TC x = TC(0);
    if (cok) {
      if (FIRST) {
        if (r < L) x = (TC)src[r * ld_src + col] * (TC)signs[r];
      } else {
        x = (TC)src[r * ld_src + col];
      }
    }
    v[b] = x;
  }
#pragma unroll
  for (int h = 1; h < NR; h <<= 1)
#pragma unroll
    for (int b = 0; b < NR; ++b)
      if (!(b & h)) {
        const TC x = v[b], y = v[b + h];
        v[b] = x + y;
        v[b + h] = x - y;
      }
#pragma unroll
  for (int b = 0; b < NR; ++b) tile[((w << R1) | b) * 33 + c] = v[b];
  __syncthreads();
  // phase 2: rows (k << R1) | j for j = w NJ + i
#pragma unroll
  for (int i = 0; i < NJ; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) v[i * 8 + k] = tile[((k << R1) | (w * NJ + i)) * 33 + c];
#pragma unroll
  for (int i = 0; i < NJ; ++i)
#pragma unroll
    for (int h = 1; h < 8; h <<= 1)
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (!(k & h)) {
          const TC x = v[i * 8 + k], y = v[i * 8 + k + h];
          v[i * 8 + k] = x + y;
          v[i * 8 + k + h] = x - y;
        }
  if (!cok) return;
#pragma unroll
  for (int i = 0; i < NJ; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t r = grow((k << R1) | (w * NJ + i));
      if (LAST) {
        const int32_t q = rowmap[r];
        if (q >= 0) Y[(int64_t)q * cols + col] = scale * (double)v[i * 8 + k];
      } else {
        dst[r * cols + col] = v[i * 8 + k];
      }
    }
}

template <typename TIn, typename TC>
tk_status run_fwht_pass(bool first, bool last, const TIn* srcA, const TC* srcZ, int64_t ld_src, TC* Z, double* Y,
                        const int8_t* signs, const int32_t* rowmap, int64_t L, int64_t Lp, int64_t cols, int b0,
                        int t, double scale, cudaStream_t st) {
  if (t >= 6 && t <= (sizeof(TC) == 4 ? 9 : 8)) {
    const int64_t ncb32 = cdiv(cols, 32);
    const int64_t blocks32 = (Lp >> t) * ncb32;
    const size_t smem32 = sizeof(TC) * (size_t)(1 << t) * 33;
#define TK_FWHT_REG(R, F, LST, SRC)                                                                         \
  do {                                                                                                      \
    auto kern = k_fwht_reg<TIn, TC, F, LST, R>;                                                             \
    TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 72 * 1024));            \
    kern<<<(unsigned)blocks32, 256, smem32, st>>>(SRC, ld_src, Z, Y, signs, rowmap, L, cols, b0, ncb32, scale); \
  } while (0)
#define TK_FWHT_REG_T(R)                                                                   \
  do {                                                                                     \
    if (first && last) TK_FWHT_REG(R, true, true, srcA);                                   \
    else if (first) TK_FWHT_REG(R, true, false, srcA);                                     \
    else if (last) TK_FWHT_REG(R, false, true, reinterpret_cast<const TIn*>(srcZ));        \
    else TK_FWHT_REG(R, false, false, reinterpret_cast<const TIn*>(srcZ));                 \
  } while (0)
    switch (t) {
      case 6: TK_FWHT_REG_T(3); break;
      case 7: TK_FWHT_REG_T(4); break;
      case 8: TK_FWHT_REG_T(5); break;
      default:
        if constexpr (sizeof(TC) == 4) TK_FWHT_REG_T(6);
        break;
    }
#undef TK_FWHT_REG_T
#undef TK_FWHT_REG
    TK_LAUNCH_CHECK();
    return TK_OK;
  }
  const int CB = fwht_cb<TC>();
  const int64_t ncb = cdiv(cols, CB);
  const int64_t groups = Lp >> t;
  const int64_t blocks = groups * ncb;
  const size_t smem = sizeof(TC) * (size_t)(1 << t) * CB;
#define TK_FWHT_LAUNCH(F, LST, SRC)                                                                       \
  do {                                                                                                    \
    auto kern = k_fwht_pass<TIn, TC, F, LST>;                                                             \
    /* one constant cap for every caller (concurrent host threads must not race on it) */                 \
    TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));          \
    kern<<<(unsigned)blocks, kFwhtThreads, smem, st>>>(SRC, ld_src, Z, Y, signs, rowmap, L, cols, b0, t, \
                                                       ncb, scale);                                       \
  } while (0)
  if (first && last) TK_FWHT_LAUNCH(true, true, srcA);
  else if (first) TK_FWHT_LAUNCH(true, false, srcA);
  else if (last) TK_FWHT_LAUNCH(false, true, reinterpret_cast<const TIn*>(srcZ));
  else TK_FWHT_LAUNCH(false, false, reinterpret_cast<const TIn*>(srcZ));
#undef TK_FWHT_LAUNCH
  TK_LAUNCH_CHECK();
  return TK_OK;
}

// ---- SRDCT ---------------------------------------------------------------------
// X = sqrt(Lp/s) S C D [A; 0] with C the orthonormal DCT-II of length Lp (a
// power of two), D and S the SRHT's draws.  The DCT of each column comes from
// one complex FFT of the same length (Makhoul): with v_i = x_2i and
// v_(Lp-1-i) = x_(2i+1) (i < Lp/2) and V = FFT(v),
//   DCT-II(x)_k = Re(exp(-i pi k / (2 Lp)) V_k),  times a_k = sqrt((1 + [k > 0]) / Lp).
// The FFT is radix-2 decimation in frequency: stage j (from the top bit down)
// pairs rows i and i + 2^j and multiplies the difference by
// exp(-2 pi i (i mod 2^j) / 2^(j+1)) = T[(i mod 2^j) 2^(a-1-j)], T a table of
// exp(-2 pi i q / Lp).  Passes run up to 8 stages on a tile of 2^t rows x one
// 128-byte column block (real and imaginary parts in shared memory); the
// first pass loads the reordered, sign-flipped rows of A, the last one leaves
// V_k in row bitrev(k) and evaluates only the sampled k.
constexpr int kFftMaxBits = 8;

template <typename TC>
__global__ void k_fft_twiddles(int64_t Lp, TC* __restrict__ tre, TC* __restrict__ tim) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Lp / 2; q += (int64_t)gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)q / (double)Lp, &sn, &cs);
    tre[q] = (TC)cs;
    tim[q] = (TC)(-sn);
  }
}

template <typename TIn, typename TC, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kFwhtThreads)
    k_fft_pass(const TIn* __restrict__ src, int64_t ld_src, TC* __restrict__ zre, TC* __restrict__ zim,
               double* __restrict__ Y, const int8_t* __restrict__ signs, const int32_t* __restrict__ rowmap,
               const TC* __restrict__ tre, const TC* __restrict__ tim, int64_t L, int a, int64_t cols, int b0, int t,
               int64_t ncb, double scale) {
  constexpr int CB = fwht_cb<TC>(), LCB = fwht_lcb<TC>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* sre = reinterpret_cast<TC*>(smem_raw);
  TC* sim = sre + (CB << t);
  const int64_t Lp = int64_t(1) << a;
  const int64_t g = blockIdx.x / ncb;
  const int64_t cb = blockIdx.x - g * ncb;
  const int64_t lo = g & ((int64_t(1) << b0) - 1);
  const int64_t hi = g >> b0;
  const int rows_t = 1 << t;
  const int64_t c0 = cb * CB;
  const int tile_elems = rows_t << LCB;
  for (int idx = threadIdx.x; idx < tile_elems; idx += blockDim.x) {
    const int mid = idx >> LCB, c = idx & (CB - 1);
    const int64_t r = (hi << (b0 + t)) | ((int64_t)mid << b0) | lo;
    const int64_t col = c0 + c;
    TC vr = TC(0), vi = TC(0);
    if (col < cols) {
      if (FIRST) {
        const int64_t sr = Lp == 1 ? 0 : (r < Lp / 2 ? 2 * r : 2 * (Lp - 1 - r) + 1);  // Makhoul's reordering
        if (sr < L) vr = (TC)src[sr * ld_src + col] * (TC)signs[sr];
      } else {
        vr = zre[r * cols + col];
        vi = zim[r * cols + col];
      }
    }
    sre[idx] = vr;
    sim[idx] = vi;
  }
  __syncthreads();
  const int pairs = (rows_t >> 1) << LCB;
  for (int lv = t - 1; lv >= 0; --lv) {  // global bit j = b0 + lv, top bit first
    const int h = 1 << lv;
    const int j = b0 + lv;
    for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
      const int q = p >> LCB, c = p & (CB - 1);
      const int i = ((q >> lv) << (lv + 1)) | (q & (h - 1));
      const int ia = (i << LCB) + c, ib = ia + (h << LCB);
      const TC ar = sre[ia], ai = sim[ia], br = sre[ib], bi = sim[ib];
      const int64_t tw = ((((int64_t)(i & (h - 1))) << b0) | lo) << (a - 1 - j);
      const TC wr = tre[tw], wi = tim[tw];
      const TC dr = ar - br, di = ai - bi;
      sre[ia] = ar + br;
      sim[ia] = ai + bi;
      sre[ib] = dr * wr - di * wi;
      sim[ib] = dr * wi + di * wr;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < tile_elems; idx += blockDim.x) {
    const int mid = idx >> LCB, c = idx & (CB - 1);
    const int64_t r = (hi << (b0 + t)) | ((int64_t)mid << b0) | lo;
    const int64_t col = c0 + c;
    if (col >= cols) continue;
    if (LAST) {
      const int64_t k = a == 0 ? 0 : (int64_t)(__brevll((unsigned long long)r) >> (64 - a));  // V_k in row bitrev(k)
      const int32_t q = rowmap[k];
      if (q >= 0) {
        double sn, cs;
        sincospi((double)k / (double)(2 * Lp), &sn, &cs);
        const double ak = k == 0 ? sqrt(1.0 / (double)Lp) : sqrt(2.0 / (double)Lp);
        Y[(int64_t)q * cols + col] = scale * ak * (cs * (double)sre[idx] + sn * (double)sim[idx]);
      }
    } else {
      zre[r * cols + col] = sre[idx];
      zim[r * cols + col] = sim[idx];
    }
  }
}

template <typename TIn, typename TC>
tk_status srdct_impl(const TIn* A, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s, double* Y,
                     Arena& ar, cudaStream_t st) {
  const int64_t Lp = next_pow2(L);
  const int a = ilog2(Lp);
  int8_t* signs = ar.take<int8_t>((size_t)Lp);
  int32_t* rowmap = ar.take<int32_t>((size_t)Lp);
  TC* zre = (a > kFftMaxBits) ? ar.take<TC>((size_t)Lp * (size_t)cols) : nullptr;
  TC* zim = (a > kFftMaxBits) ? ar.take<TC>((size_t)Lp * (size_t)cols) : nullptr;
  TC* tre = ar.take<TC>((size_t)std::max<int64_t>(Lp / 2, 1));
  TC* tim = ar.take<TC>((size_t)std::max<int64_t>(Lp / 2, 1));
  if (!ar.ok()) return TK_ENOMEM;
  if (a > 62) return TK_EINVAL;
  TK_TRY(draw_signs_rows(seed, Lp, s, signs, nullptr, rowmap, ar, st));
  if (s == 0 || cols == 0) return TK_OK;
  if (Lp >= 2) {
    k_fft_twiddles<TC><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(Lp / 2, 256), 152 * 32)), 256, 0, st>>>(
        Lp, tre, tim);
    TK_LAUNCH_CHECK();
  }
  const double scale = sqrt((double)Lp / (double)s);
  const int CB = fwht_cb<TC>();
  const int64_t ncb = cdiv(cols, CB);
  int top = a;
  bool first = true;
  do {
    const int b0 = std::max(top - kFftMaxBits, 0);
    const int t = top - b0;
    const bool last = b0 == 0;
    const int64_t blocks = (Lp >> t) * ncb;
    const size_t smem = 2 * sizeof(TC) * (size_t)(1 << t) * CB;
#define TK_FFT_LAUNCH(F, LST)                                                                                   do {                                                                                                            auto kern = k_fft_pass<TIn, TC, F, LST>;                                                                      TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));                  kern<<<(unsigned)blocks, kFwhtThreads, smem, st>>>(A, ld, zre, zim, Y, signs, rowmap, tre, tim, L, a, cols,                                                        b0, t, ncb, scale);                                      } while (0)
    if (first && last) TK_FFT_LAUNCH(true, true);
    else if (first) TK_FFT_LAUNCH(true, false);
    else if (last) TK_FFT_LAUNCH(false, true);
    else TK_FFT_LAUNCH(false, false);
#undef TK_FFT_LAUNCH
    TK_LAUNCH_CHECK();
    first = false;
    top = b0;
  } while (top > 0);
  return TK_OK;
}

template <typename TC>
__global__ void k_gauss_fill(uint64_t seed, int64_t s, int64_t L, double inv_sqrt_s, TC* __restrict__ G) {
  int64_t total = s * L;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += stride)
    G[k] = (TC)gauss_entry(seed, (uint64_t)k, inv_sqrt_s);
}

template <typename T>
__global__ void k_transpose(const T* __restrict__ A, int64_t rows, int64_t cols, int64_t lda, T* __restrict__ AT) {
  __shared__ T tileT[32][33];
  int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tileT[k][threadIdx.x] = A[r * lda + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) AT[c * rows + r] = tileT[threadIdx.x][k];
  }
}

__global__ void k_f64_to_f32(const double* __restrict__ s, float* __restrict__ d, int64_t rows, int64_t cols,
                             int64_t lds, int64_t ldd) {
  int64_t total = rows * cols;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += stride) {
    int64_t r = k / cols, c = k - r * cols;
    d[r * ldd + c] = (float)s[r * lds + c];
  }
}

__global__ void k_f32_to_f64(const float* __restrict__ s, double* __restrict__ d, int64_t total) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += stride) d[k] = (double)s[k];
}

int grid_for(int64_t total, int threads) { return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, threads), 152 * 32)); }

template <typename TIn, typename TC>
tk_status srht_impl(const TIn* A, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s, double* Y,
                    Arena& ar, cudaStream_t st) {
  const int64_t Lp = next_pow2(L);
  const int a = ilog2(Lp);
  int8_t* signs = ar.take<int8_t>((size_t)Lp);
  int32_t* rowmap = ar.take<int32_t>((size_t)Lp);
  TC* Z = (a > (sizeof(TC) == 4 ? kFwhtMaxBits : 8)) ? ar.take<TC>((size_t)Lp * (size_t)cols) : nullptr;  // > 1 pass
  if (!ar.ok()) return TK_ENOMEM;
  TK_TRY(draw_signs_rows(seed, Lp, s, signs, nullptr, rowmap, ar, st));
  if (s == 0 || cols == 0) return TK_OK;
  const double scale = 1.0 / sqrt((double)s);
  // bits per pass: up to 9 (float) or 8 (double, whose register pass holds 32 values); passes of
  // equal size where possible, so that every pass can run in registers (>= 6 bits)
  const int maxb = sizeof(TC) == 4 ? kFwhtMaxBits : 8;
  int npass = (a + maxb - 1) / maxb;
  if (npass == 0) npass = 1;
  int b0 = 0;
  for (int p = 0; p < npass; ++p) {
    int t = (a - b0 + (npass - p) - 1) / (npass - p);  // split the remaining bits evenly
    if (t < 0) t = 0;
    bool first = (p == 0), last = (p == npass - 1);
    TK_TRY((run_fwht_pass<TIn, TC>(first, last, A, Z, first ? ld : cols, Z, Y, signs, rowmap, L, Lp, cols, b0, t,
                                   scale, st)));
    b0 += t;
  }
  return TK_OK;
}

// Split count of the float64 Gaussian sketch product Y (s x cols) = G A:
// enough 64 x 64 output tiles x splits for two CTAs per SM, >= 256 rows each.
int gauss_splits(int64_t L, int64_t cols, int64_t s) {
  const int64_t tiles = cdiv(s, 64) * cdiv(cols, 64);
  if (tiles >= 152) return 1;
  return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(2 * 152, tiles), L / 256));
}

// Y[k] = sum_z part[z][k]
__global__ void k_sum_planes(const double* __restrict__ part, int splits, int64_t total, double* __restrict__ Y) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < splits; ++z) acc += part[(int64_t)z * total + k];
    Y[k] = acc;
  }
}

template <typename TIn, typename TC>
tk_status gauss_impl(const TIn* A, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s, double* Y,
                     Arena& ar, cudaStream_t st) {
  TC* G = ar.take<TC>((size_t)s * (size_t)L);
  TC* Yc = std::is_same<TC, double>::value ? nullptr : ar.take<TC>((size_t)s * (size_t)cols);
  const int splits = std::is_same<TC, double>::value ? gauss_splits(L, cols, s) : 1;
  double* part = splits > 1 ? ar.take<double>((size_t)splits * s * cols) : nullptr;
  if (!ar.ok()) return TK_ENOMEM;
  if (s == 0 || cols == 0) return TK_OK;
  k_gauss_fill<TC><<<grid_for(s * L, 256), 256, 0, st>>>(seed, s, L, 1.0 / sqrt((double)s), G);
  TK_LAUNCH_CHECK();
  if (std::is_same<TC, double>::value) {
    if (splits > 1) {  // few output tiles: split the sum over the long axis, then add the planes
      TK_TRY((gemm_splitk<TC, TIn>(false, false, s, cols, L, G, L, A, ld, part, splits, st)));
      k_sum_planes<<<grid_for(s * cols, 256), 256, 0, st>>>(part, splits, s * cols, Y);
      TK_LAUNCH_CHECK();
    } else {
      TK_TRY((gemm<TC, TIn, double>(false, false, s, cols, L, G, L, A, ld, Y, cols, 1.0, nullptr, nullptr, 0, st)));
    }
  } else {
    TK_TRY((gemm<TC, TIn, TC>(false, false, s, cols, L, G, L, A, ld, Yc, cols, 1.0, nullptr, nullptr, 0, st)));
    k_f32_to_f64<<<grid_for(s * cols, 256), 256, 0, st>>>(reinterpret_cast<const float*>(Yc), Y, s * cols);
    TK_LAUNCH_CHECK();
  }
  return TK_OK;
}

}  // namespace

size_t srht_rows_workspace(int64_t L, int64_t cols, tk_dtype dt, int64_t s) {
  (void)s;
  const int64_t Lp = next_pow2(L);
  Arena a;
  a.take<int8_t>((size_t)Lp);
  a.take<int32_t>((size_t)Lp);
  if (ilog2(Lp) > (dt == TK_F64 ? 8 : kFwhtMaxBits)) a.take<char>((size_t)Lp * (size_t)cols * (dt == TK_F64 ? 8 : 4));
  return a.used + draw_workspace(Lp) + 512;
}

size_t srdct_rows_workspace(int64_t L, int64_t cols, tk_dtype dt, int64_t s) {
  (void)s;
  const int64_t Lp = next_pow2(L);
  const size_t es = dt == TK_F64 ? 8 : 4;
  Arena a;
  a.take<int8_t>((size_t)Lp);
  a.take<int32_t>((size_t)Lp);
  if (ilog2(Lp) > kFftMaxBits) {
    a.take<char>((size_t)Lp * (size_t)cols * es);
    a.take<char>((size_t)Lp * (size_t)cols * es);
  }
  a.take<char>((size_t)std::max<int64_t>(Lp / 2, 1) * es);
  a.take<char>((size_t)std::max<int64_t>(Lp / 2, 1) * es);
  return a.used + draw_workspace(Lp) + 512;
}

tk_status srdct_rows(const void* A, tk_dtype dt, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s,
                     double* Y, Arena& ar, cudaStream_t st) {
  if (dt == TK_F64) return srdct_impl<double, double>((const double*)A, L, cols, ld, seed, s, Y, ar, st);
  return srdct_impl<float, float>((const float*)A, L, cols, ld, seed, s, Y, ar, st);
}

size_t gauss_rows_workspace(int64_t L, int64_t cols, tk_dtype dt, int64_t s) {
  Arena a;
  size_t es = dt == TK_F64 ? 8 : 4;
  a.take<char>((size_t)s * (size_t)L * es);
  if (dt != TK_F64) a.take<char>((size_t)s * (size_t)cols * es);
  const int splits = dt == TK_F64 ? gauss_splits(L, cols, s) : 1;
  if (splits > 1) a.take<double>((size_t)splits * s * cols);
  return a.used + 512;
}

tk_status srht_rows(const void* A, tk_dtype dt, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s,
                    double* Y, Arena& ar, cudaStream_t st) {
  if (dt == TK_F64) return srht_impl<double, double>((const double*)A, L, cols, ld, seed, s, Y, ar, st);
  return srht_impl<float, float>((const float*)A, L, cols, ld, seed, s, Y, ar, st);
}

tk_status gauss_rows(const void* A, tk_dtype dt, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s,
                     double* Y, Arena& ar, cudaStream_t st) {
  if (dt == TK_F64) return gauss_impl<double, double>((const double*)A, L, cols, ld, seed, s, Y, ar, st);
  return gauss_impl<float, float>((const float*)A, L, cols, ld, seed, s, Y, ar, st);
}

tk_status transpose(const void* A, tk_dtype dt, int64_t rows, int64_t cols, int64_t lda, void* AT, cudaStream_t st) {
  if (rows == 0 || cols == 0) return TK_OK;
  dim3 grid((unsigned)cdiv(cols, 32), (unsigned)cdiv(rows, 32));
  dim3 block(32, 8);
  if (grid.y > 65535u) {
    set_error_msg("transpose: too many rows for one launch");
    return TK_EINVAL;
  }
  if (dt == TK_F64) k_transpose<double><<<grid, block, 0, st>>>((const double*)A, rows, cols, lda, (double*)AT);
  else k_transpose<float><<<grid, block, 0, st>>>((const float*)A, rows, cols, lda, (float*)AT);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

tk_status convert_f64_to_f32(const double* src, float* dst, int64_t rows, int64_t cols, int64_t lds, int64_t ldd,
                             cudaStream_t st) {
  if (rows * cols == 0) return TK_OK;
  k_f64_to_f32<<<grid_for(rows * cols, 256), 256, 0, st>>>(src, dst, rows, cols, lds, ldd);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

}  // namespace tk
