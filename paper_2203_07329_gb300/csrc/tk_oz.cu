// Float64-accurate products on the BF16 tensor cores (splitting into exact
// integer slices, in the manner of Ozaki's error-free matrix multiplication).
//
// GB300 issues about two float64 FMA per clock per SM, so the float64 products
// of the mixed form (the Gram matrix, the Cholesky trailing updates, and the
// refinement's r = b - X A^T and A^T r) are bound by that pipe.  Here every
// row of an operand is scaled by a power of two 2^E (E one above the exponent
// of its largest entry, so that 2^(E-2) <= max |x| < 2^(E-1)), rounded to
// nearest at 2^(E-57) (within 2^-55 of the row maximum) and written with
// S = 8 balanced base-128 digits,
//   x 2^-E = sum_p d_p 2^(-7(p+1)),  d_p in [-64, 64],
// taken from the least significant end with carries; each digit is exact in
// BF16.  A product of two digits is an integer of magnitude <= 2^12; the pairs
// (p, q) with p + q = t share one FP32 accumulator ("level" t), and a level
// sum of at most 8 pairs over 256 values of K stays below 2^24, so the tensor
// core's FP32 accumulation is exact.  Every 256 values of K the level sums
// are added, with their weights 2^(-7(t+2)), exactly into two int64
// accumulators per output (levels 0-3 and 4-7), made one double at the
// end (with 4 digits: scaled into FP32 accumulators).  The 28
// pairs with p + q > 7 are dropped: at most 7.1 * 2^-58 of 2^(Ea+Ex), i.e.
// 2^-51 of max|a| max|x| per product when every digit is +-64 (typical digits
// give far less).  The result carries errors of a few float64 units relative
// to the row maxima: the normwise accuracy of a float64 GEMM (the tests check
// it element by element against extended-precision products).  Cut after 4
// digits, the same slices are a round-to-nearest 28-bit representation.
//
// The products run on tcgen05 (kind::f16, M = 128, K = 16; per digit p of the
// big operand one MMA of N = 32 (S - p) over the stacked digit planes of the
// small one), operands brought in by TMA in the 128-byte swizzle layout, the
// level accumulators in tensor memory, double-buffered so that four epilogue
// warps flush one 256-value chunk of K while the MMAs of the next chunk run.
#include <algorithm>
#include <climits>
#include <type_traits>
#include <cuda_bf16.h>

#include "tk_internal.cuh"
#include "tk_tcgen05.cuh"

namespace tk {
namespace {

constexpr int OZ_S = 8;          // slices
constexpr int OZ_LV = OZ_S;      // levels t = p + q in 0..7 kept
constexpr int OZ_KPAD = 64;      // slice rows are padded to a multiple of 64 values of K (one TMA box)

// Exponent marking a row or column with an inf or NaN: its digits are zero
// and every output that uses it is NaN, so non-finite input is reported (the
// LSQR stop tests and the refinement see it) instead of being dropped.
constexpr int OZ_EBAD = 1 << 24;

// max(m, |x|) that turns inf and NaN into +inf (fmax would ignore a NaN).
__device__ __forceinline__ double oz_absmax(double m, double x) {
  const double a = fabs(x);
  return a <= m ? m : (a == a ? a : __longlong_as_double(0x7ff0000000000000ll));
}
// The exponent of a maximum: one above frexp's (0 for 0, OZ_EBAD if not finite).
__device__ __forceinline__ int oz_exponent(double mx) {
  if (!(mx <= 1.7976931348623157e308)) return OZ_EBAD;
  int e = 0;
  if (mx > 0.0) {
    frexp(mx, &e);  // mx = f 2^e, 0.5 <= f < 1
    ++e;            // so mx < 2^(e-1)
  }
  return e;
}

// Exponent E with max_j |row_j| < 2^(E-1) (0 for a zero row); one warp per row.
template <typename T>
__global__ void k_oz_rowexp(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld, int* __restrict__ E) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const int lane = threadIdx.x & 31;
  double mx = 0.0;
  for (int64_t j = lane; j < cols; j += 32) mx = oz_absmax(mx, (double)X[r * ld + j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) E[r] = oz_exponent(mx);
}

// Exponent E with max_r |X[r][c]| < 2^(E-1) per column (0 for a zero column):
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
  for (int64_t r = r0; r < r1; ++r) v = oz_absmax(v, (double)X[r * ld + c]);
  atomicMax(&mx[c], (unsigned long long)__double_as_longlong(v));  // +inf orders above every finite value
}
__global__ void k_oz_colexp(const unsigned long long* __restrict__ mx, int64_t cols, int* __restrict__ E) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  E[c] = oz_exponent(__longlong_as_double((long long)mx[c]));
}

// round(x 2^(56-E)) (|x 2^-E| < 1/2, so |result| <= 2^55) from the bit
// pattern of x: no float64 instruction (GB300 issues those at a fraction of
// the integer rate).  Ties round away from zero.
__device__ __forceinline__ long long oz_fixed(double x, int E) {
  const long long bits = __double_as_longlong(x);
  int ex = (int)((bits >> 52) & 0x7ff);
  long long mant = bits & ((1ll << 52) - 1);
  if (ex) mant |= 1ll << 52;
  else ex = 1;  // subnormal: same scale as the smallest normal exponent
  const int sh = ex - 1019 - E;  // |x| 2^(56-E) = mant 2^sh
  long long u;
  if (sh >= 0) u = mant << sh;  // mant 2^sh < 2^55: sh < 55
  else if (sh > -63) u = (mant + (1ll << (-sh - 1))) >> (-sh);
  else u = 0;
  return bits < 0 ? -u : u;
}
__device__ __forceinline__ long long oz_fixed(float x, int E) {
  const int bits = __float_as_int(x);
  int ex = (bits >> 23) & 0xff;
  long long mant = bits & 0x7fffff;
  if (ex) mant |= 0x800000;
  else ex = 1;
  const int sh = ex - 94 - E;  // |x| 2^(56-E) = mant 2^sh
  long long u;
  if (sh >= 0) u = mant << sh;  // mant 2^sh < 2^55: sh < 55 (subnormal x: small mant)
  else if (sh > -63) u = (mant + (1ll << (-sh - 1))) >> (-sh);
  else u = 0;
  return bits < 0 ? -u : u;
}

// BF16 bits of a small integer (|d| <= 2^8): through the float with the
// 1.5 * 2^23 offset; its low 16 bits are zero, so the top half is exact.
__device__ __forceinline__ unsigned short oz_bf16_bits(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return (unsigned short)(__float_as_uint(f) >> 16);
}

// The 8 balanced base-128 digits of v (|v| <= 2^55): d = ((u + 64) mod 128)
// - 64 from the bottom, carry (u - d) / 128, on two 32-bit halves (the low 28
// bits, then the rest plus the carry); the last carry is the top digit,
// |d_0| <= 64.  bits[p] = BF16 bit pattern of d_p.
__device__ __forceinline__ void oz_digits(long long v, unsigned short (&bits)[OZ_S]) {
  int lo = (int)(v & ((1ll << 28) - 1));
  int hi = (int)(v >> 28);
#pragma unroll
  for (int p = OZ_S - 1; p >= 4; --p) {
    const int d = ((lo + 64) & 127) - 64;
    bits[p] = oz_bf16_bits(d);
    lo = (lo - d) >> 7;
  }
  hi += lo;
#pragma unroll
  for (int p = 3; p >= 1; --p) {
    const int d = ((hi + 64) & 127) - 64;
    bits[p] = oz_bf16_bits(d);
    hi = (hi - d) >> 7;
  }
  bits[0] = oz_bf16_bits(hi);
}

template <typename T>
__device__ __forceinline__ void oz_split(T x, int E, unsigned short (&bits)[OZ_S]) {
  oz_digits(oz_fixed(x, E), bits);
}
__device__ __forceinline__ unsigned oz_pack(unsigned short a, unsigned short b) { return (unsigned)a | ((unsigned)b << 16); }

// Slices of the rows of X with row exponents E: planes out[p][r][c] (row
// stride cols_pad, zero in the padding) with X[r][c] 2^-E[r] = sum_p
// out[p][r][c] 2^(-7(p+1)) to within 2^-57 (rounded to nearest).
// Grid: rows over blockIdx.x (grid-stride) and column chunks of 2 x 256 over
// blockIdx.y; each thread splits two adjacent values (one 4-byte store per plane).
template <typename T>
__global__ void __launch_bounds__(256) k_oz_slice(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                                                  const int* __restrict__ E, int64_t cols_pad, int planes,
                                                  __nv_bfloat16* __restrict__ out) {
  const int64_t plane = rows * cols_pad;
  const int64_t c = ((int64_t)blockIdx.y * blockDim.x + threadIdx.x) * 2;
  if (c >= cols_pad) return;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int e = E[r];
    const T* xr = X + r * ld;
    unsigned short s0[OZ_S], s1[OZ_S];
    oz_split(c < cols ? xr[c] : T(0), e, s0);
    oz_split(c + 1 < cols ? xr[c + 1] : T(0), e, s1);
    unsigned* o = reinterpret_cast<unsigned*>(out + r * cols_pad + c);
#pragma unroll
    for (int p = 0; p < OZ_S; ++p)
      if (p < planes) o[p * (plane / 2)] = oz_pack(s0[p], s1[p]);
  }
}

// Exponents of long rows (cols much larger than rows): E[r] = max over the
// blocks of a row of the exponent of their largest |value| (atomicMax; E
// filled with OZ_EMIN first, then zero rows set to 0).
constexpr int OZ_EMIN = -4096;
__global__ void k_oz_fill_emin(int* __restrict__ E, int64_t rows) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows) E[r] = OZ_EMIN;
}
template <typename T>
__global__ void __launch_bounds__(256) k_oz_rowexp_long(const T* __restrict__ X, int64_t cols, int64_t ld,
                                                        int64_t per_block, int* __restrict__ E) {
  __shared__ double sh[32];
  const int64_t r = blockIdx.y;
  const int64_t c0 = (int64_t)blockIdx.x * per_block;
  const int64_t c1 = c0 + per_block < cols ? c0 + per_block : cols;
  double mx = 0.0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) mx = oz_absmax(mx, (double)X[r * ld + c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, sh[w]);
    if (mx > 0.0) atomicMax(&E[r], oz_exponent(mx));  // OZ_EBAD wins
  }
}
__global__ void k_oz_fix_zero_rows(int* __restrict__ E, int64_t rows) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows && E[r] == OZ_EMIN) E[r] = 0;
}

// Slices of the COLUMNS of X (rows x cols) with column exponents E, stored
// transposed: planes out[p][c][r] (row stride rows_pad, zero in the padding).
// 64 x 32 tiles through shared memory: reads of 32 consecutive columns, and
// per plane 128-byte stores of 64 consecutive rows (two per thread); grid.x
// runs over row tiles, grid.y over column tiles.
template <typename T>
__global__ void __launch_bounds__(256) k_oz_slice_t(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                                                    const int* __restrict__ E, int64_t rows_pad,
                                                    __nv_bfloat16* __restrict__ out) {
  __shared__ T tile[64][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int64_t r0 = (int64_t)blockIdx.x * 64, c0 = (int64_t)blockIdx.y * 32;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = r0 + ty + 8 * i, c = c0 + tx;
    tile[ty + 8 * i][tx] = (r < rows && c < cols) ? X[r * ld + c] : T(0);
  }
  __syncthreads();
  const int64_t plane = cols * rows_pad;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int cc = ty + 8 * i;
    const int64_t c = c0 + cc, r = r0 + 2 * tx;
    if (c < cols && r < rows_pad) {  // rows_pad is a multiple of 64: r + 1 < rows_pad too
      const int e = E[c];
      unsigned short s0[OZ_S], s1[OZ_S];
      oz_split(tile[2 * tx][cc], e, s0);
      oz_split(tile[2 * tx + 1][cc], e, s1);
      unsigned* o = reinterpret_cast<unsigned*>(out + c * rows_pad + r);
#pragma unroll
      for (int p = 0; p < OZ_S; ++p) o[p * (plane / 2)] = oz_pack(s0[p], s1[p]);
    }
  }
}

// ---- the product on tcgen05 ---------------------------------------------------
// D[r][l] = sum_k P[r][k] Q[l][k] from the first S digit planes of P (rows x
// K, row exponents EP) and of Q (M x K, row exponents EQ), both K-major.
// S = 8: float64 accuracy (levels added exactly into int64 accumulators, one
// rounding at the end); S = 4: the 28-bit rounded operands, float32 accuracy
// (levels flushed into float32).
// CTA: 128 rows of P x 32 rows of Q x one K split (blockIdx.z).
//   warp 0 (one lane): TMA producer -- per 64 values of K the S planes of Q
//     (4 KiB each) into a 2-slot ring, then the S planes of P one by one
//     (16 KiB each) into an 8-slot ring;
//   warp 1 (one lane): MMA issuer -- for plane p of P, D_(p+q) += P_p Q_q^T
//     for every q <= S-1-p as one MMA of N = 32 (S - p) (4 of K = 16); the
//     level accumulators of a chunk of 256 values of K sit in one of two
//     tensor-memory buffers;
//   warp 2: allocates / frees the 2 S 32 tensor-memory columns;
//   warps 4-7: epilogue -- per chunk, read the S levels (lanes 32(w-4) ..),
//     add them into 32 accumulators per row, release the buffer; at the end
//     write the result: MODE 0 R[l][r] = b[r] - D (float64); MODE 1
//     partial[z][l][r] = D (float64); MODE 2 U[l][r] = D + coef[l] U[l][r]
//     (float32 U; coef == nullptr: U = D).
// Every mbarrier wait is bounded; a wait that gives up sets *err and the
// roles stop.
constexpr int OT_M = 128;
constexpr int OT_N = 32;
constexpr int OT_KB = 64;
constexpr int OT_CHUNK = 256;
constexpr int OT_KB_PER_CHUNK = OT_CHUNK / OT_KB;
constexpr int64_t OT_MAX_KPS = int64_t(1) << 27;  // values of K per split that the int64 level sums hold exactly
constexpr uint32_t OT_P_BYTES = OT_M * OT_KB * 2;   // 16 KiB

// CTA shapes (tensor memory: 2 buffers x S levels x NT columns <= 512):
//   S = 8, NT = 32 (float64-accurate passes): one CTA per SM, an 8-slot ring of P planes;
//   S = 4, NT = 32 (float32 LSQR products, <= 32 lambda): 4 slots and 256 columns, so two
//     CTAs share an SM and one streams while the other starts up or flushes its last chunk;
//   S = 4, NT = 64 (more than 32 lambda): one CTA per SM over 64 lambda, so the digit planes
//     of the big operand are read once for 64 lambda instead of once per 32.
template <int S, int NT>
struct OtCfg {
  static constexpr bool WIDE = S == OZ_S || NT == 64;
  static constexpr int PST = WIDE ? 8 : 4;
  static constexpr int CTAS_PER_SM = WIDE ? 1 : 2;
  static constexpr uint32_t QS_BYTES = NT * OT_KB * 2;  // one digit plane of the small operand
};

template <int S, int NT>
struct OtSmem {
  static constexpr int PST = OtCfg<S, NT>::PST;
  uint8_t p[PST][OT_P_BYTES];
  uint8_t q[2][S * OtCfg<S, NT>::QS_BYTES];
  uint64_t p_full[PST];
  uint64_t p_empty[PST];
  uint64_t q_full[2];
  uint64_t q_empty[2];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t mma_drain;  // error path: completes when every MMA the CTA issued is done
  uint32_t tmem_base;
};

template <int S, int MODE, int NT>
__global__ void __launch_bounds__(256, OtCfg<S, NT>::CTAS_PER_SM)
    k_oz_tc(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmQ,
            const int* __restrict__ EP, const int* __restrict__ EQ, int64_t rows, int M, int64_t K, int64_t kps,
            const double* __restrict__ b, void* __restrict__ out, int64_t ldo, const double* __restrict__ coef,
            int upper_only, int* __restrict__ err) {
  using Acc = typename std::conditional<S == OZ_S, double, float>::type;
  constexpr uint32_t TMEM_COLS = 2 * S * NT;
  constexpr uint32_t QS_BYTES = OtCfg<S, NT>::QS_BYTES;
  constexpr uint32_t Q_BYTES = S * QS_BYTES;
  extern __shared__ __align__(1024) uint8_t ot_raw[];
  OtSmem<S, NT>& Sm = *reinterpret_cast<OtSmem<S, NT>*>((reinterpret_cast<uintptr_t>(ot_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * OT_M;
  const int l0 = (int)blockIdx.y * NT;
  // a symmetric product (P = Q) needs out[l][r] for l <= r only
  if (upper_only && l0 > r0 + OT_M - 1) return;
  const int64_t kbeg = (int64_t)blockIdx.z * kps;
  const int64_t kend = K < kbeg + kps ? K : kbeg + kps;
  const int nkb = kend > kbeg ? (int)((kend - kbeg + OT_KB - 1) / OT_KB) : 0;
  const int nch = (nkb + OT_KB_PER_CHUNK - 1) / OT_KB_PER_CHUNK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OtCfg<S, NT>::PST; ++s) {
      mbar_init(&Sm.p_full[s], 1);
      mbar_init(&Sm.p_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&Sm.q_full[s], 1);
      mbar_init(&Sm.q_empty[s], 1);
      mbar_init(&Sm.acc_full[s], 1);
      mbar_init(&Sm.acc_empty[s], 128);
    }
    mbar_init(&Sm.mma_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&Sm.tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = Sm.tmem_base;

  if (warp == 0 && lane == 0) {
    int g = 0, gq = 0;  // loads issued into the P ring and the Q ring
    bool live = true;
    for (int kb = 0; kb < nkb && live; ++kb) {
      const int kc = (int)(kbeg + (int64_t)kb * OT_KB);
      const int qs = kb & 1;
      if (!mbar_wait(&Sm.q_empty[qs], ((uint32_t)(kb >> 1) & 1u) ^ 1u, err)) break;
      mbar_expect_tx(&Sm.q_full[qs], Q_BYTES);
      for (int p = 0; p < S; ++p) tma_load_3d(&tmQ, &Sm.q_full[qs], Sm.q[qs] + p * QS_BYTES, kc, l0, p);
      ++gq;
      for (int p = 0; p < S; ++p, ++g) {
        const int ps = g % OtCfg<S, NT>::PST;
        if (!mbar_wait(&Sm.p_empty[ps], ((uint32_t)(g / OtCfg<S, NT>::PST) & 1u) ^ 1u, err)) {
          live = false;
          break;
        }
        mbar_expect_tx(&Sm.p_full[ps], OT_P_BYTES);
        tma_load_3d(&tmP, &Sm.p_full[ps], Sm.p[ps], kc, (int)r0, p);
      }
    }
    if (*(volatile int*)err) {  // gave up: no bulk copy may still be landing when the CTA exits
      tma_drain_ring(Sm.p_full, OtCfg<S, NT>::PST, g);
      tma_drain_ring(Sm.q_full, 2, gq);
    }
  } else if (warp == 1 && lane == 0) {
    int g = 0;
    bool live = true;
    for (int c = 0; c < nch && live; ++c) {
      const int bsel = c & 1, use = c >> 1;
      if (use > 0 && !mbar_wait(&Sm.acc_empty[bsel], (uint32_t)(use - 1) & 1u, err)) break;
      tc_fence_after();
      const uint32_t dbase = tmem + (uint32_t)(bsel * S * NT);
      const int kb0 = OT_KB_PER_CHUNK * c;
      const int kb_end = nkb < kb0 + OT_KB_PER_CHUNK ? nkb : kb0 + OT_KB_PER_CHUNK;
      for (int kb = kb0; kb < kb_end && live; ++kb) {
        const int qs = kb & 1;
        if (!mbar_wait(&Sm.q_full[qs], (uint32_t)(kb >> 1) & 1u, err)) {
          live = false;
          break;
        }
        tc_fence_after();
        const uint32_t qa = smem_u32(Sm.q[qs]);
        for (int p = 0; p < S; ++p, ++g) {
          const int ps = g % OtCfg<S, NT>::PST;
          if (!mbar_wait(&Sm.p_full[ps], (uint32_t)(g / OtCfg<S, NT>::PST) & 1u, err)) {
            live = false;
            break;
          }
          tc_fence_after();
          // the planes Q_0 .. Q_(S-1-p) lie one after another (NT rows each), and the levels
          // p .. S-1 are consecutive NT-column blocks of the buffer: all pairs (p, q) are one
          // MMA with N = NT (S - p) whose column block q lands on level p + q
          const uint64_t pd = sdesc_sw128(smem_u32(Sm.p[ps]));
          const uint64_t qd = sdesc_sw128(qa);
          const uint32_t idesc = idesc_bf16(OT_M, NT * (S - p));
          const uint32_t d = dbase + (uint32_t)(p * NT);
#pragma unroll
          for (int k = 0; k < OT_KB / 16; ++k) {
            // the first MMA of a chunk (p = 0) overwrites every level of the buffer
            const uint32_t acc = (kb == kb0 && p == 0 && k == 0) ? 0u : 1u;
            tc_mma_bf16(d, pd + 2ull * k, qd + 2ull * k, idesc, acc);
          }
          tc_commit(&Sm.p_empty[ps]);
        }
        if (live) tc_commit(&Sm.q_empty[qs]);
      }
      if (live) tc_commit(&Sm.acc_full[bsel]);
    }
    if (*(volatile int*)err) {  // gave up: wait for the MMAs issued before tensor memory is freed
      tc_commit(&Sm.mma_drain);
      mbar_drain(&Sm.mma_drain, 0u);
    }
  } else if (warp >= 4) {
    const int ew = warp - 4;
    // S = 8 (float64-accurate): the chunk's 8 exact level sums (|L_t| <= (t+1) 2^20, so L0 128 + L1 and
    // the like fit an int) are added exactly into two int64 accumulators per column, hi += L0 2^21 +
    // L1 2^14 + L2 2^7 + L3 and lo likewise from L4 .. L7 (value = hi 2^-35 + lo 2^-63; each under 2^44 per
    // chunk, so exact for K <= 2^27 per split), 8 columns at a time -- integer work, off GB300's slow float64
    // pipe -- and turned into one double at the end.  S = 4: float32 accumulators.
    Acc acc[S == OZ_S ? 1 : NT];
    long long hacc[S == OZ_S ? NT : 1], lacc[S == OZ_S ? NT : 1];
#pragma unroll
    for (int j = 0; j < (S == OZ_S ? 1 : NT); ++j) acc[j] = Acc(0);
#pragma unroll
    for (int j = 0; j < (S == OZ_S ? NT : 1); ++j) hacc[j] = lacc[j] = 0;
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
      const int bsel = c & 1, use = c >> 1;
      if (!mbar_wait(&Sm.acc_full[bsel], (uint32_t)use & 1u, err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(bsel * S * NT);
      if constexpr (S == OZ_S) {
#pragma unroll
        for (int g = 0; g < NT / 8; ++g) {
          uint32_t v[OZ_S][8];
#pragma unroll
          for (int t = 0; t < OZ_S; ++t) tmem_ld8_nowait(base + (uint32_t)(t * NT + 8 * g), v[t]);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            int L[OZ_S];
#pragma unroll
            for (int t = 0; t < OZ_S; ++t) L[t] = __float2int_rz(__uint_as_float(v[t][j]));  // exact integers
            hacc[8 * g + j] += (long long)(L[0] * 128 + L[1]) * 16384 + (L[2] * 128 + L[3]);
            lacc[8 * g + j] += (long long)(L[4] * 128 + L[5]) * 16384 + (L[6] * 128 + L[7]);
          }
        }
      } else {
#pragma unroll 1
        for (int t = S - 1; t >= 0; --t) {  // smallest level first
#pragma unroll
          for (int h = 0; h < NT / 32; ++h) {
            uint32_t v[32];
            tmem_ld32_nowait(base + (uint32_t)(t * NT + 32 * h), v);
            tmem_wait_ld();
            const float sc = __int_as_float((127 - 7 * (t + 2)) << 23);  // 2^(-7(t+2)), exact
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[32 * h + j] = fmaf(__uint_as_float(v[j]), sc, acc[32 * h + j]);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&Sm.acc_empty[bsel]);
    }
    const int64_t r = r0 + ew * 32 + lane;
    if (ok && r < rows) {
      const int er = EP[r];
      const double br = MODE == 0 ? b[r] : 0.0;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int l = l0 + j;
        if (l < M) {
          const int eq = EQ[l];
          double d;
          if constexpr (S == OZ_S) d = fma((double)lacc[j], 0x1p-63, (double)hacc[j] * 0x1p-35);
          else d = (double)acc[j];
          const double v = (er >= OZ_EBAD || eq >= OZ_EBAD) ? __longlong_as_double(0x7ff8000000000000ll)
                                                            : ldexp(d, er + eq);
          if (MODE == 0) {
            static_cast<double*>(out)[(int64_t)l * ldo + r] = br - v;
          } else if (MODE == 1) {
            static_cast<double*>(out)[((int64_t)blockIdx.z * M + l) * ldo + r] = v;
          } else {
            float* u = static_cast<float*>(out) + (int64_t)l * ldo + r;
            *u = coef ? (float)(v + coef[l] * (double)*u) : (float)v;
          }
        }
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// 3D map over the slice planes (K fastest, then rows, then the plane index),
// box = 64 values of K x box_rows x 1 plane, 128-byte swizzle.
tk_status make_slice_map(CUtensorMap* map, const void* base, int64_t rows, int64_t kp, uint32_t box_rows,
                         int planes) {
  EncodeTiledFn fn;
  TK_TRY(encode_fn(&fn));
  const cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)rows * kp * 2};
  const cuuint32_t box[3] = {(cuuint32_t)OT_KB, box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error_msg("cuTensorMapEncodeTiled rejected the slice layout");
    return TK_ECUDA;
  }
  return TK_OK;
}

// P: planesP digit planes of rows x K, Q: planesQ planes of M x K (both K
// rounded up to 64); S digits of each are used.
// The lambda-tile width of a product with M rows of the small operand: 64 for the
// LSQR products (S = 4) over more than 32 lambda, else 32.
constexpr int oz_tile_n(int S, int64_t M) { return (S != OZ_S && M > 32) ? 64 : 32; }

template <int S, int MODE, int NT>
tk_status launch_oz_tc_nt(const CUtensorMap& mP, const void* Qs, const int* EP, int64_t rows, const int* EQ, int M,
                          int planesQ, int64_t kp, int64_t kps, int sp, const double* b, void* out, int64_t ldo,
                          const double* coef, int* err, cudaStream_t st, int upper_only) {
  CUtensorMap mQ;
  TK_TRY(make_slice_map(&mQ, Qs, M, kp, NT, planesQ));
  const size_t smem = sizeof(OtSmem<S, NT>) + 1024;
  TK_CUDA(cudaFuncSetAttribute(k_oz_tc<S, MODE, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const dim3 grid((unsigned)cdiv(rows, OT_M), (unsigned)cdiv(M, NT), (unsigned)sp);
  k_oz_tc<S, MODE, NT><<<grid, 256, smem, st>>>(mP, mQ, EP, EQ, rows, M, kp, kps, b, out, ldo, coef, upper_only, err);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

template <int S, int MODE>
tk_status launch_oz_tc(const void* Ps, const int* EP, int64_t rows, int planesP, const void* Qs, const int* EQ, int M,
                       int planesQ, int64_t K, int splits, const double* b, void* out, int64_t ldo,
                       const double* coef, int* err, cudaStream_t st, int upper_only = 0) {
  const int64_t kp = cdiv(K, OZ_KPAD) * OZ_KPAD;
  if (rows > INT32_MAX || kp > INT32_MAX || M > 65535 * OT_N) {
    set_error_msg("emulated product: dimensions exceed the 32-bit TMA coordinates");
    return TK_EINVAL;
  }
  CUtensorMap mP;
  TK_TRY(make_slice_map(&mP, Ps, rows, kp, OT_M, planesP));
  const int64_t kps = cdiv(cdiv(K, splits), OT_CHUNK) * OT_CHUNK;  // whole chunks per split
  const int sp = (int)cdiv(K, kps);
  if (S == OZ_S && kps > OT_MAX_KPS) {  // the exact int64 level accumulators of a split
    set_error_msg("emulated product: more than 2^27 values of K in one split");
    return TK_EINVAL;
  }
  if (oz_tile_n(S, M) == 64) {
    if constexpr (S != OZ_S)
      TK_TRY((launch_oz_tc_nt<S, MODE, 64>(mP, Qs, EP, rows, EQ, M, planesQ, kp, kps, sp, b, out, ldo, coef, err, st,
                                           upper_only)));
  } else {
    TK_TRY((launch_oz_tc_nt<S, MODE, 32>(mP, Qs, EP, rows, EQ, M, planesQ, kp, kps, sp, b, out, ldo, coef, err, st,
                                         upper_only)));
  }
  if (MODE == 1 && sp < splits) {  // the caller sums `splits` planes: the unused ones are zero
    double* o = static_cast<double*>(out);
    TK_CUDA(cudaMemsetAsync(o + (int64_t)sp * M * ldo, 0, sizeof(double) * (size_t)(splits - sp) * M * ldo, st));
  }
  return TK_OK;
}

// ---- Cholesky trailing update -------------------------------------------------
// Right-looking blocked Cholesky (upper, R^T R = C + lambda I), 64-row block
// step kb: with the row panel P = R[kb rows, columns > kb] (64 x w) already
// solved, the trailing upper triangle T -= P^T P.  The panel's columns are
// sliced with one exponent per column (the output index), stored K-major
// (planes [lambda][p][column][64]); one CTA then forms a 128 x 64 tile of
// P^T P for one lambda from all 8 + 8 slice planes at once (K = 64: a single
// chunk, exact in FP32), flushes the 8 levels into float64 and subtracts the
// scaled result from T through shared memory (coalesced).

// Panel slices of block row kb for every lambda (grid: column tiles of 32 x
// lambda).  Rows c >= w of the slice planes are not written.
__global__ void __launch_bounds__(256) k_oz_panel_slice(const double* __restrict__ R, int64_t ldr, int64_t rstride,
                                                        int64_t np, int kb, __nv_bfloat16* __restrict__ out,
                                                        int* __restrict__ EC) {
  __shared__ double tile[64][33];
  __shared__ int ex[32];
  const int l = blockIdx.y;
  const int64_t c0 = (int64_t)(kb + 1) * 64, w = np - c0;
  const int64_t ct = (int64_t)blockIdx.x * 32;
  const double* Rl = R + (int64_t)l * rstride + (int64_t)kb * 64 * ldr + c0;
  for (int idx = threadIdx.x; idx < 64 * 32; idx += blockDim.x) {
    const int k = idx >> 5, cc = idx & 31;
    const int64_t c = ct + cc;
    tile[k][cc] = c < w ? Rl[(int64_t)k * ldr + c] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double mx = 0.0;
    for (int k = 0; k < 64; ++k) mx = oz_absmax(mx, tile[k][threadIdx.x]);
    const int e = oz_exponent(mx);
    ex[threadIdx.x] = e;
    const int64_t c = ct + threadIdx.x;
    if (c < w) EC[(int64_t)l * np + c] = e;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 64 * 32; idx += blockDim.x) {
    const int cc = idx >> 6, k = idx & 63;
    const int64_t c = ct + cc;
    if (c < w) {
      unsigned short sl[OZ_S];
      oz_split(tile[k][cc], ex[cc], sl);
      unsigned short* o = reinterpret_cast<unsigned short*>(out);
#pragma unroll
      for (int p = 0; p < OZ_S; ++p) o[(((int64_t)l * OZ_S + p) * np + c) * 64 + k] = sl[p];
    }
  }
}

constexpr int CS_M = 128;                        // rows of a CTA's slab
constexpr int CS_N = 32;                         // columns of one tile
constexpr int CS_TILES = 8;                      // column tiles per CTA
constexpr uint32_t CS_P_BYTES = CS_M * 64 * 2;   // 16 KiB per digit plane of the slab
constexpr uint32_t CS_Q_BYTES = CS_N * 64 * 2;   // 4 KiB per digit plane of a tile
constexpr uint32_t CS_TMEM_COLS = 2 * OZ_LV * CS_N;  // two buffers of 8 levels x 32 columns

struct CsSmem {
  uint8_t p[OZ_S][CS_P_BYTES];
  uint8_t q[2][OZ_S * CS_Q_BYTES];
  int ecol[CS_TILES * CS_N];  // the column exponents of the CTA's tiles
  uint64_t p_full;
  uint64_t q_full[2];
  uint64_t q_empty[2];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t mma_drain;  // error path: completes when every MMA the CTA issued is done
  uint32_t tmem_base;
};

// A level sum of K = 64 products (|L| <= 8 * 64 * 64 * 64 = 2^21) as an
// int: the float's integer read back through the 1.5 * 2^23 offset (exact for
// |L| < 2^22).
__device__ __forceinline__ int level_int(uint32_t bits) {
  return __float_as_int(__fadd_rn(__uint_as_float(bits), 12582912.0f)) - 0x4B400000;
}

// 2^e as a double (e within the normal range).
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// v 2^s as a double, built from the integer's bits with integer instructions
// only (GB300's float64 pipe is the bottleneck of the update's epilogue):
// exact for |v| < 2^53.  *ok = false when the result would not be a normal
// double (the caller then takes the float64 route).
__device__ __forceinline__ double i53_scaled(long long v, int s, bool* ok) {
  if (v == 0) return 0.0;
  const unsigned long long sg = v < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int p = 63 - __clzll((long long)a);  // a in [2^p, 2^(p+1)), p <= 52
  const int ex = p + s + 1023;
  if (ex < 1 || ex > 2046) {
    *ok = false;
    return 0.0;
  }
  const unsigned long long mant = (a << (52 - p)) & ((1ull << 52) - 1);
  return __longlong_as_double((long long)(sg | ((unsigned long long)ex << 52) | mant));
}

// Grid: (row slabs of 128, chunks of 8 column tiles of 32, lambda) over the
// w x w trailing block.  Slab i0 needs the tiles j0 >= i0 (j >= i); a CTA
// whose chunk holds none exits at once.  The slab's digit planes are loaded
// once; the tiles stream through a 2-slot ring and two tensor-memory buffers,
// so the flush and the update of one tile overlap the products of the next.
// Flush: the 8 exact level sums are combined in int64 by Horner,
// hi = ((L0 128 + L1) 128 + L2) 128 + L3 and lo likewise from L4..L7 (both
// below 2^43), and the tile value is hi 2^-35 + lo 2^-63 (exact products of
// exact integers), scaled by 2^(E_i + E_j).
__global__ void __launch_bounds__(384, 1)
    k_oz_syrk(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmQ,
              const int* __restrict__ EC, int64_t np, int kb, double* __restrict__ R, int64_t ldr, int64_t rstride,
              int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t cs_raw[];
  CsSmem& S = *reinterpret_cast<CsSmem*>((reinterpret_cast<uintptr_t>(cs_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.z;
  const int64_t c0 = (int64_t)(kb + 1) * 64, w = np - c0;
  const int i0 = (int)blockIdx.x * CS_M;
  const int t_first = i0 / CS_N + (int)blockIdx.y * CS_TILES;
  const int t_all = (int)(w / CS_N);
  const int nt = t_all - t_first < CS_TILES ? t_all - t_first : CS_TILES;
  if (nt <= 0) return;

  if (threadIdx.x == 0) {
    mbar_init(&S.p_full, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S.q_full[s], 1);
      mbar_init(&S.q_empty[s], 1);
      mbar_init(&S.acc_full[s], 1);
      mbar_init(&S.acc_empty[s], 256);
    }
    mbar_init(&S.mma_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(CS_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0 && lane == 0) {
    mbar_expect_tx(&S.p_full, OZ_S * CS_P_BYTES);
    for (int p = 0; p < OZ_S; ++p) tma_load_3d(&tmP, &S.p_full, S.p[p], 0, i0, l * OZ_S + p);
    int gq = 0;  // tiles issued into the Q ring
    for (int t = 0; t < nt; ++t) {
      const int s = t & 1;
      if (!mbar_wait(&S.q_empty[s], ((uint32_t)(t >> 1) & 1u) ^ 1u, err)) break;
      mbar_expect_tx(&S.q_full[s], OZ_S * CS_Q_BYTES);
      const int j0 = (t_first + t) * CS_N;
      for (int p = 0; p < OZ_S; ++p) tma_load_3d(&tmQ, &S.q_full[s], S.q[s] + p * CS_Q_BYTES, 0, j0, l * OZ_S + p);
      ++gq;
    }
    if (*(volatile int*)err) {  // gave up: no bulk copy may still be landing when the CTA exits
      mbar_drain(&S.p_full, 0u);
      tma_drain_ring(S.q_full, 2, gq);
    }
  } else if (warp == 1 && lane == 0) {
    if (mbar_wait(&S.p_full, 0u, err)) {
      for (int t = 0; t < nt; ++t) {
        const int s = t & 1;
        if (!mbar_wait(&S.q_full[s], (uint32_t)(t >> 1) & 1u, err)) break;
        if (t >= 2 && !mbar_wait(&S.acc_empty[s], (uint32_t)((t >> 1) - 1) & 1u, err)) break;
        tc_fence_after();
        const uint64_t qd = sdesc_sw128(smem_u32(S.q[s]));
        const uint32_t dbase = tmem + (uint32_t)(s * OZ_LV * CS_N);
        for (int p = 0; p < OZ_S; ++p) {
          // planes Q_0 .. Q_(7-p) are contiguous: one MMA of N = 32 (8 - p) onto levels p .. 7
          const uint64_t pd = sdesc_sw128(smem_u32(S.p[p]));
          const uint32_t idesc = idesc_bf16(CS_M, CS_N * (OZ_S - p));
          const uint32_t d = dbase + (uint32_t)(p * CS_N);
#pragma unroll
          for (int k = 0; k < 4; ++k) tc_mma_bf16(d, pd + 2ull * k, qd + 2ull * k, idesc, (p == 0 && k == 0) ? 0u : 1u);
        }
        tc_commit(&S.q_empty[s]);
        tc_commit(&S.acc_full[s]);
      }
    }
    if (*(volatile int*)err) {  // gave up: wait for the MMAs issued before tensor memory is freed
      tc_commit(&S.mma_drain);
      mbar_drain(&S.mma_drain, 0u);
    }
  } else if (warp >= 4) {
    // 8 epilogue warps: warp w reads tensor-memory lanes 32 (w % 4) .. (the rows), and the two warps
    // of a lane quarter split each tile's 32 columns: warps 4-7 the first 16, warps 8-11 the last 16
    const int ew = warp & 3, half = (warp - 4) >> 2;
    const int64_t i = i0 + ew * 32 + lane;
    const int* El = EC + (int64_t)l * np;
    const int ei = i < w ? El[i] : 0;
    double* Trow = R + (int64_t)l * rstride + (c0 + i) * ldr + c0;
    // the exponents of the CTA's columns, once, in shared memory (the epilogue warps only)
    for (int c = (int)threadIdx.x - 128; c < CS_TILES * CS_N; c += 256) {
      const int64_t col = (int64_t)t_first * CS_N + c;
      S.ecol[c] = col < w ? El[col] : 0;
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    // the thread's 16 columns of a tile in 2 groups of 8; per group the 8 levels of the 8 columns are
    // read from tensor memory and the exact integers hi = L0 2^21 + L1 2^14 + L2 2^7 + L3 and lo (L4 ..
    // L7 likewise) formed as (L0 128 + L1) 2^14 + (L2 128 + L3) -- the same integers as a Horner
    // chain, |L0 128 + L1| < 2^30
    constexpr int G = 8;
    for (int t = 0; t < nt; ++t) {
      const int s = t & 1;
      const int64_t j0 = (int64_t)(t_first + t) * CS_N + half * 2 * G;
      // T of the thread's 16 columns first: their loads do not wait for the products
      double tv[2][G];
#pragma unroll
      for (int gi = 0; gi < 2; ++gi)
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int64_t col = j0 + gi * G + j;
          tv[gi][j] = (i < w && col < w && col >= i) ? Trow[col] : 0.0;
        }
      if (!mbar_wait(&S.acc_full[s], (uint32_t)(t >> 1) & 1u, err)) break;
      tc_fence_after();
      const uint32_t base =
          tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(s * OZ_LV * CS_N) + (uint32_t)(half * 2 * G);
#pragma unroll
      for (int gi = 0; gi < 2; ++gi) {
        const int64_t jg = j0 + gi * G;
        uint32_t v[OZ_LV][G];
#pragma unroll
        for (int lv = 0; lv < OZ_LV; ++lv) tmem_ld8_nowait(base + (uint32_t)(lv * CS_N + gi * G), v[lv]);
        tmem_wait_ld();
        if (gi == 1) {
          tc_fence_before();
          mbar_arrive(&S.acc_empty[s]);  // every level of the thread's columns is in registers
        }
        if (i < w) {
#pragma unroll
          for (int j = 0; j < G; ++j) {
            if (jg + j < w && jg + j >= i) {
              const int ej = S.ecol[t * CS_N + half * 2 * G + gi * G + j];
              const int e = ei + ej;
              if (ei >= OZ_EBAD || ej >= OZ_EBAD) {  // a row or column marked non-finite: NaN (its digits are zero)
                Trow[jg + j] = __longlong_as_double(0x7ff8000000000000ll);
                continue;
              }
              const int a0 = level_int(v[0][j]) * 128 + level_int(v[1][j]);
              const int a1 = level_int(v[2][j]) * 128 + level_int(v[3][j]);
              const int b0 = level_int(v[4][j]) * 128 + level_int(v[5][j]);
              const int b1 = level_int(v[6][j]) * 128 + level_int(v[7][j]);
              const long long hi = (long long)a0 * 16384 + a1, lo = (long long)b0 * 16384 + b1;
              // (hi 2^-35 + lo 2^-63) 2^e with the two scaled terms built exactly from the integers'
              // bits; the sum and the subtraction are the only float64 operations (the same rounding
              // as scaling the rounded sum, since a power of two scales exactly)
              bool ok = true;
              const double shi = i53_scaled(hi, e - 35, &ok), slo = i53_scaled(lo, e - 63, &ok);
              if (ok) {
                Trow[jg + j] = tv[gi][j] - (shi + slo);
              } else {  // a scaled term outside the normal range: through the float64 pipe
                const double vhi = (double)hi * 0x1p-35, vlo = (double)lo * 0x1p-63;  // exact
                Trow[jg + j] = tv[gi][j] - (vhi + vlo) * (e >= -1022 && e <= 1023 ? pow2d(e) : ldexp(1.0, e));
              }
            }
          }
        }
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CS_TMEM_COLS) : "memory");
  }
}


// ---- the two products of an LSQR step, fused over one read of A -----------------
// One LSQR step of the mixed form needs U' = W A^T + c .* U (m values per lambda)
// and then G = U' A (n values per lambda).  The second product of a band of rows
// needs the first product over the band's whole rows, so a band must be held
// between the two.  Here a cluster of CL CTAs (CL a power of two <= 8) owns one
// band of 128 rows at a time, CTA q the columns [q cpc, (q + 1) cpc) of it (cpc <=
// 256, so the CTA's slab of the 4 digit planes is at most 256 KiB):
//   P1  the CTA's part of W A^T for the band (K = its columns) on tcgen05 into one
//       of two tensor-memory buffers; W's digits stay in shared memory throughout;
//   X1  the CL partials are added through distributed shared memory: CTA q adds
//       the rows [q 128/CL, (q + 1) 128/CL) in rank order, forms U' = v + c U for
//       them (written to U), and stores u' = U' 2^(E_r - E_max) (the row scale of
//       A's digits moved onto U') into every CTA's copy of the band's u';
//   X2  every CTA digitizes the band's u' (4 digits, one exponent per lambda) into
//       the B operand of
//   P2  G_q += A_slab^T u' on tcgen05, the A operand read MN-major from the same
//       digit planes, read again (from L2: a few microseconds after P1's read).
// The producer issues the next band's P1 loads before this band's P2 loads, so A
// streams from memory while the epilogue exchanges and digitizes.  Each CTA keeps
// its columns' G in registers across all the bands its cluster processes, and
// writes one partial plane per cluster at the end.  The exchange uses mbarriers in
// distributed shared memory with bounded waits; every CTA reaches the cluster
// barrier before exit, so no CTA leaves while another may still read or write its
// shared memory.
constexpr int FU_M = 128;   // band rows
constexpr int FU_NT = 32;   // lambda
constexpr int FU_RS = 3;    // ring slots of one 128-column chunk of one digit plane (2 TMA boxes)
constexpr int FU_S = 4;     // digits (the float32 LSQR products)
constexpr uint32_t FU_SLOT = 2 * OT_P_BYTES;                 // 32 KiB
constexpr uint32_t FU_QBOX = FU_NT * 64 * 2;                 // 4 KiB: 32 rows x 64 values of one plane
constexpr uint32_t FU_QCH = 2 * FU_S * FU_QBOX;              // 32 KiB: 128 K x 4 planes
constexpr uint32_t FU_TMEM_COLS = 512;                       // P1: 2 x 128, P2: 2 x 128

struct FuSmem {
  uint8_t ring[FU_RS][FU_SLOT];
  uint8_t wq[2][FU_QCH];      // W digits of chunk c (resident): [64-K box][plane][32 rows][128 B]
  uint8_t q2[FU_QCH];         // u' digits: [64-row chunk][plane][32 lambda][128 B]
  float pbuf[FU_NT * FU_M];   // P1 partial, [lambda][row]
  float ub[FU_NT * FU_M];     // u' of the band, [lambda][row]
  uint32_t umax[4][FU_NT];    // per warp: max |u'| bits per lambda
  int ea[FU_M];
  int eu[FU_NT];
  int ew[FU_NT];
  float psc[FU_NT];           // 2^(E_max + E_u) of the band, per lambda (the P2 scale)
  int emax4[4];
  uint64_t ring_full[FU_RS], ring_empty[FU_RS], w_full;
  uint64_t p1_full[2], p1_empty[2], q2_full, q2_empty, p2_full[2], p2_empty[2];
  uint64_t pb_full, pb_empty, ub_full, ub_empty;
  uint64_t mma_drain;
  uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t nclusters_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// shared::cluster address of `p` (a shared variable of this CTA) in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t dsmem_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void dsmem_arrive(uint32_t bar_cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster_addr) : "memory");
}
// generic pointer to `p` (a shared array of this CTA) in CTA `rank` of the cluster: plain loads and
// stores through it, which the compiler may batch (ordered after the acquiring waits, which clobber memory)
template <typename T>
__device__ __forceinline__ T* peer_ptr(T* p, uint32_t rank) {
  return static_cast<T*>(__cluster_map_shared_rank(static_cast<void*>(p), rank));
}
// bounded wait with cluster-scope acquire (data written by other CTAs before their arrive is visible)
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* b, uint32_t parity, int* err) {
  uint64_t t0 = 0;
  for (uint32_t i = 0; i < (1u << 26); ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (i >= 256) __nanosleep(32);
    if ((i & 255u) == 255u) {
      if (*(volatile int*)err) return false;
      const uint64_t t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > kWaitBudgetNs) break;
    }
  }
  atomicExch(err, 1);
  return false;
}
// true on every one of the 128 epilogue threads iff v is true on all of them (named barrier 1): the
// epilogue takes every exit together, so no thread is left waiting at a named barrier
__device__ __forceinline__ bool epi_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 128, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// K-major operand, 128-byte swizzle: byte offset of element (row, k) in a box of 64 values per row
__device__ __forceinline__ uint32_t sw128_off(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) + ((k & 7) << 1));
}
// MN-major 128-byte-swizzled operand: LBO = distance between 64-element blocks along M, SBO = between
// 8-row blocks along K
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t saddr, uint32_t lbo_bytes) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// 2^e as a float (0 below the normal range, inf above)
__device__ __forceinline__ float pow2f(int e) {
  return e < -126 ? 0.f : (e > 127 ? __int_as_float(0x7f800000) : __int_as_float((127 + e) << 23));
}

// The 4 balanced base-128 digits of x 2^-E rounded to 28 bits (|x| < 2^E): the value
// v = round(x 2^(28 - E)) (exact scaling in float64, one rounding) written as
// d0 2^21 + d1 2^14 + d2 2^7 + d3 with d1..d3 in [-64, 63].
__device__ __forceinline__ void oz_split4(float x, int E, unsigned short (&bits)[4]) {
  int v = (int)__double2ll_rn((double)x * pow2d(28 - E));
#pragma unroll
  for (int p = 3; p >= 1; --p) {
    const int d = ((v + 64) & 127) - 64;
    bits[p] = oz_bf16_bits(d);
    v = (v - d) >> 7;
  }
  bits[0] = oz_bf16_bits(v);
}

__global__ void __launch_bounds__(256, 1)
    k_oz_fused(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW,
               const int* __restrict__ EA, const int* __restrict__ EW, int64_t m, int64_t n, int count, int cpc,
               float* __restrict__ U, int64_t ldu, const double* __restrict__ coef, double* __restrict__ partial,
               int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t fu_raw[];
  FuSmem& S = *reinterpret_cast<FuSmem*>((reinterpret_cast<uintptr_t>(fu_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t q = cluster_rank();
  int cl_size;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(cl_size));
  const int64_t bands = (m + FU_M - 1) / FU_M;
  const int64_t zc = cluster_id_x(), ncl = nclusters_x();
  const int nb = zc < bands ? (int)((bands - 1 - zc) / ncl + 1) : 0;  // bands of this cluster
  const int nch = cpc / 128;       // 128-column chunks of this CTA (1 or 2)
  const int col0 = (int)q * cpc;   // this CTA's first column
  const int row_lo = (int)q * (FU_M / cl_size), nrows = FU_M / cl_size;  // this CTA's rows in X1

  if (threadIdx.x == 0) {
    for (int s = 0; s < FU_RS; ++s) {
      mbar_init(&S.ring_full[s], 1);
      mbar_init(&S.ring_empty[s], 1);
    }
    mbar_init(&S.w_full, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S.p1_full[s], 1);
      mbar_init(&S.p1_empty[s], 128);
      mbar_init(&S.p2_full[s], 1);
      mbar_init(&S.p2_empty[s], 128);
    }
    mbar_init(&S.q2_full, 1);
    mbar_init(&S.q2_empty, 1);
    mbar_init(&S.pb_full, cl_size);
    mbar_init(&S.pb_empty, cl_size);
    mbar_init(&S.ub_full, cl_size);
    mbar_init(&S.ub_empty, cl_size);
    mbar_init(&S.mma_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < FU_NT) S.ew[threadIdx.x] = threadIdx.x < count ? EW[threadIdx.x] : 0;
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(FU_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync_all();  // every CTA's barriers are initialized before any remote arrive
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: W once; then P1(band 0), and per band i: P1(band i + 1), P2(band i) -- the
    // same 4 planes x nch chunks of A each time
    int g = 0;
    mbar_expect_tx(&S.w_full, (uint32_t)nch * FU_QCH);
    for (int c = 0; c < nch; ++c)
      for (int kb = 0; kb < 2; ++kb)
        for (int p = 0; p < FU_S; ++p)
          tma_load_3d(&tmW, &S.w_full, S.wq[c] + (kb * FU_S + p) * FU_QBOX, col0 + 128 * c + 64 * kb, 0, p);
    auto load_band = [&](int j) -> bool {
      const int r0 = (int)((zc + (int64_t)j * ncl) * FU_M);
      for (int c = 0; c < nch; ++c) {
        const int k0 = col0 + 128 * c;
        for (int p = 0; p < FU_S; ++p, ++g) {
          const int s = g % FU_RS;
          if (!mbar_wait(&S.ring_empty[s], ((uint32_t)(g / FU_RS) & 1u) ^ 1u, err)) return false;
          mbar_expect_tx(&S.ring_full[s], FU_SLOT);
          tma_load_3d(&tmA, &S.ring_full[s], S.ring[s], k0, r0, p);
          tma_load_3d(&tmA, &S.ring_full[s], S.ring[s] + OT_P_BYTES, k0 + 64, r0, p);
        }
      }
      return true;
    };
    bool live = nb == 0 || load_band(0);
    for (int i = 0; i < nb && live; ++i) {
      if (i + 1 < nb) live = load_band(i + 1);
      if (live) live = load_band(i);
    }
    if (*(volatile int*)err) {
      tma_drain_ring(S.ring_full, FU_RS, g);
      mbar_drain(&S.w_full, 0u);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    int g = 0, T = 0;
    bool live = mbar_wait(&S.w_full, 0u, err);
    tc_fence_after();
    // P1 of the cluster's j-th band into tensor-memory buffer j & 1
    auto p1 = [&](int j) -> bool {
      const int buf = j & 1;
      if (j >= 2 && !mbar_wait(&S.p1_empty[buf], (uint32_t)(((j - 2) >> 1) & 1), err)) return false;
      tc_fence_after();
      for (int c = 0; c < nch; ++c) {
        for (int p = 0; p < FU_S; ++p, ++g) {
          const int s = g % FU_RS;
          if (!mbar_wait(&S.ring_full[s], (uint32_t)(g / FU_RS) & 1u, err)) return false;
          tc_fence_after();
          const uint32_t idesc = idesc_bf16(FU_M, FU_NT * (FU_S - p));
#pragma unroll
          for (int ks = 0; ks < 8; ++ks) {  // K = 128 columns: 4 steps in each 64-column box
            const uint32_t box = (uint32_t)(ks >> 2), kk = (uint32_t)(ks & 3);
            const uint64_t ad = sdesc_sw128(smem_u32(S.ring[s]) + box * OT_P_BYTES) + 2ull * kk;
            const uint64_t bd = sdesc_sw128(smem_u32(S.wq[c]) + box * FU_S * FU_QBOX) + 2ull * kk;
            const uint32_t acc = (c == 0 && p == 0 && ks == 0) ? 0u : 1u;
            tc_mma_bf16(tmem + 128u * (uint32_t)buf + (uint32_t)(p * FU_NT), ad, bd, idesc, acc);
          }
          tc_commit(&S.ring_empty[s]);
        }
      }
      tc_commit(&S.p1_full[buf]);
      return true;
    };
    if (live && nb > 0) live = p1(0);
    for (int i = 0; i < nb && live; ++i) {
      if (i + 1 < nb && !p1(i + 1)) break;
      // P2: wait for the band's u' digits
      if (!mbar_wait(&S.q2_full, (uint32_t)(i & 1), err)) break;
      tc_fence_after();
      for (int c = 0; c < nch && live; ++c, ++T) {
        const int bsel = T & 1, use = T >> 1;
        if (use > 0 && !mbar_wait(&S.p2_empty[bsel], (uint32_t)((use - 1) & 1), err)) {
          live = false;
          break;
        }
        tc_fence_after();
        const uint32_t dbase = tmem + 256u + 128u * (uint32_t)bsel;
        for (int p = 0; p < FU_S; ++p, ++g) {
          const int s = g % FU_RS;
          if (!mbar_wait(&S.ring_full[s], (uint32_t)(g / FU_RS) & 1u, err)) {
            live = false;
            break;
          }
          tc_fence_after();
          // A operand = the slab's columns (M) x the band's rows (K), MN-major; transpose bit 15
          const uint32_t idesc = idesc_bf16(FU_M, FU_NT * (FU_S - p)) | (1u << 15);
#pragma unroll
          for (int ks = 0; ks < 8; ++ks) {  // K = 128 band rows: 16 rows (2 KiB) per step
            const uint64_t ad = sdesc_mn_sw128(smem_u32(S.ring[s]) + (uint32_t)ks * 2048u, OT_P_BYTES);
            const uint64_t bd =
                sdesc_sw128(smem_u32(S.q2) + (uint32_t)(ks >> 2) * FU_S * FU_QBOX) + 2ull * (uint32_t)(ks & 3);
            tc_mma_bf16(dbase + (uint32_t)(p * FU_NT), ad, bd, idesc, (p == 0 && ks == 0) ? 0u : 1u);
          }
          tc_commit(&S.ring_empty[s]);
        }
        if (live) tc_commit(&S.p2_full[bsel]);
      }
      if (live) tc_commit(&S.q2_empty);  // the band's u' digits are no longer read
    }
    if (*(volatile int*)err) {
      tc_commit(&S.mma_drain);
      mbar_drain(&S.mma_drain, 0u);
    }
  } else if (warp >= 4) {
    // ---- epilogue warps (thread e = TMEM lane e: a band row in P1, X2; a column in P2)
    const int e = (int)threadIdx.x - 128, ew = warp - 4;
    float gacc[2][FU_NT];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int l = 0; l < FU_NT; ++l) gacc[c][l] = 0.f;
    bool ok = true;
    int T = 0;
    // P2 of the previous band: G of this CTA's columns += A_slab^T u', the levels weighted by
    // 2^(-7 (t + 2)), the sum by 2^(E_max + E_u) (S.psc, still the previous band's)
    auto p2_read = [&]() -> bool {
#pragma unroll
      for (int c = 0; c < 2; ++c) {  // nch <= 2, unrolled so that gacc stays in registers
        if (c >= nch) break;
        const int bsel = T & 1, use = T >> 1;
        ++T;
        if (!epi_all(mbar_wait(&S.p2_full[bsel], (uint32_t)(use & 1), err))) return false;
        tc_fence_after();
        const uint32_t base = tmem + ((uint32_t)(ew * 32) << 16) + 256u + 128u * (uint32_t)bsel;
        float lev[FU_NT];
#pragma unroll
        for (int l = 0; l < FU_NT; ++l) lev[l] = 0.f;
#pragma unroll 1
        for (int t = FU_S - 1; t >= 0; --t) {
          uint32_t v[32];
          tmem_ld32_nowait(base + (uint32_t)(t * FU_NT), v);
          tmem_wait_ld();
          const float lw = __int_as_float((127 - 7 * (t + 2)) << 23);  // the level weight 2^(-7 (t + 2))
#pragma unroll
          for (int l = 0; l < FU_NT; ++l) lev[l] = fmaf(__uint_as_float(v[l]), lw, lev[l]);
        }
        tc_fence_before();
        mbar_arrive(&S.p2_empty[bsel]);
#pragma unroll
        for (int l = 0; l < FU_NT; ++l) gacc[c][l] = fmaf(lev[l], S.psc[l], gacc[c][l]);
      }
      return true;
    };
    int ea_next = nb > 0 && zc * FU_M + e < m ? EA[zc * FU_M + e] : 0;
    for (int i = 0; i < nb && ok; ++i) {
      const int64_t r0 = (zc + (int64_t)i * ncl) * FU_M;
      // the band's row exponents and their maximum over the finite rows (the next band's loaded ahead)
      const int ea_e = ea_next;
      {
        const int64_t rn = r0 + ncl * FU_M + e;
        ea_next = i + 1 < nb && rn < m ? EA[rn] : 0;
      }
      S.ea[e] = ea_e;
      const int wm = __reduce_max_sync(0xffffffffu, (r0 + e < m && ea_e < OZ_EBAD) ? ea_e : INT_MIN);
      if (lane == 0) S.emax4[ew] = wm;
      epi_sync();
      int eamax = max(max(S.emax4[0], S.emax4[1]), max(S.emax4[2], S.emax4[3]));
      if (eamax == INT_MIN) eamax = 0;
      // P1 partial of this CTA's columns, row e of the band
      const int buf = i & 1;
      if (!epi_all(mbar_wait(&S.p1_full[buf], (uint32_t)((i >> 1) & 1), err))) {
        ok = false;
        break;
      }
      tc_fence_after();
      float acc[FU_NT];
#pragma unroll
      for (int l = 0; l < FU_NT; ++l) acc[l] = 0.f;
      const uint32_t lb = tmem + ((uint32_t)(ew * 32) << 16) + 128u * (uint32_t)buf;
#pragma unroll 1
      for (int t = FU_S - 1; t >= 0; --t) {
        uint32_t v[32];
        tmem_ld32_nowait(lb + (uint32_t)(t * FU_NT), v);
        tmem_wait_ld();
        const float sc = __int_as_float((127 - 7 * (t + 2)) << 23);
#pragma unroll
        for (int l = 0; l < FU_NT; ++l) acc[l] = fmaf(__uint_as_float(v[l]), sc, acc[l]);
      }
      tc_fence_before();
      mbar_arrive(&S.p1_empty[buf]);
      // my partial may be overwritten once every CTA has read the previous band's
      if (!epi_all(i == 0 || mbar_wait_cluster(&S.pb_empty, (uint32_t)((i - 1) & 1), err))) {
        ok = false;
        break;
      }
#pragma unroll
      for (int l = 0; l < FU_NT; ++l) S.pbuf[l * FU_M + e] = acc[l];
      epi_sync();
      if (e == 0) {
        asm volatile("fence.acq_rel.cluster;" ::: "memory");
        for (int r = 0; r < cl_size; ++r) dsmem_arrive(dsmem_addr(&S.pb_full, (uint32_t)r));
      }
      // the previous band's P2 while the peers' partials arrive
      if (i > 0 && !p2_read()) {
        ok = false;
        break;
      }
      // X1: my rows of the band (4 at a time), summed over the cluster in rank order; U' = v + c U;
      // u' into every CTA
      if (!epi_all(mbar_wait_cluster(&S.pb_full, (uint32_t)(i & 1), err) &&
                   (i == 0 || mbar_wait_cluster(&S.ub_empty, (uint32_t)((i - 1) & 1), err)))) {
        ok = false;
        break;
      }
      const int nq = nrows / 4;
      for (int v = e; v < FU_NT * nq; v += 128) {
        const int l = v / nq, row = row_lo + 4 * (v % nq);
        float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int r = 0; r < cl_size; ++r) {
          const float4 t4 = *reinterpret_cast<const float4*>(peer_ptr(S.pbuf, (uint32_t)r) + l * FU_M + row);
          s4.x += t4.x;
          s4.y += t4.y;
          s4.z += t4.z;
          s4.w += t4.w;
        }
        const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
        float up[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int64_t grow = r0 + row + k;
          up[k] = 0.f;
          if (grow < m && l < count) {
            const int er = S.ea[row + k], eq = S.ew[l];
            const int es = er + eq;
            const double val = (er >= OZ_EBAD || eq >= OZ_EBAD) ? __longlong_as_double(0x7ff8000000000000ll)
                               : (es >= -1022 && es <= 1023) ? (double)sv[k] * pow2d(es)
                                                             : ldexp((double)sv[k], es);
            float* u = U + (int64_t)l * ldu + grow;
            const float un = coef ? (float)(val + coef[l] * (double)*u) : (float)val;
            *u = un;
            up[k] = er >= OZ_EBAD ? un : un * pow2f(er - eamax);
          }
        }
        const float4 u4 = make_float4(up[0], up[1], up[2], up[3]);
        for (int r = 0; r < cl_size; ++r)
          *reinterpret_cast<float4*>(peer_ptr(S.ub, (uint32_t)r) + l * FU_M + row) = u4;
      }
      epi_sync();
      if (e == 0) {
        asm volatile("fence.acq_rel.cluster;" ::: "memory");
        for (int r = 0; r < cl_size; ++r) {
          dsmem_arrive(dsmem_addr(&S.pb_empty, (uint32_t)r));
          dsmem_arrive(dsmem_addr(&S.ub_full, (uint32_t)r));
        }
      }
      // X2: the band's u' digits (4, one exponent per lambda) into the B operand of P2; thread e = row
      if (!epi_all(mbar_wait_cluster(&S.ub_full, (uint32_t)(i & 1), err) &&
                   (i == 0 || mbar_wait(&S.q2_empty, (uint32_t)((i - 1) & 1), err)))) {
        ok = false;
        break;
      }
#pragma unroll 4
      for (int l = 0; l < FU_NT; ++l) {
        const uint32_t b = __float_as_uint(fabsf(S.ub[l * FU_M + e]));  // non-finite: >= 0x7f800000
        const uint32_t mx = __reduce_max_sync(0xffffffffu, b);
        if (lane == 0) S.umax[ew][l] = mx;
      }
      epi_sync();
      if (e < FU_NT) {
        const uint32_t mx = max(max(S.umax[0][e], S.umax[1][e]), max(S.umax[2][e], S.umax[3][e]));
        const int eu = mx >= 0x7f800000u ? OZ_EBAD : oz_exponent((double)__uint_as_float(mx));
        S.eu[e] = eu;
        S.psc[e] = eu >= OZ_EBAD ? __int_as_float(0x7fc00000) : pow2f(eamax + eu);
      }
      epi_sync();
      {
        uint8_t* base = S.q2 + (e >> 6) * FU_S * FU_QBOX;
#pragma unroll 4
        for (int l = 0; l < FU_NT; ++l) {
          const int eu = S.eu[l];
          unsigned short bits[FU_S];
          oz_split4(eu >= OZ_EBAD ? 0.f : S.ub[l * FU_M + e], eu >= OZ_EBAD ? 0 : eu, bits);
#pragma unroll
          for (int p = 0; p < FU_S; ++p)
            *reinterpret_cast<unsigned short*>(base + p * FU_QBOX + sw128_off(l, e & 63)) = bits[p];
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core reads
      epi_sync();
      if (e == 0) {
        mbar_arrive(&S.q2_full);
        asm volatile("fence.acq_rel.cluster;" ::: "memory");
        for (int r = 0; r < cl_size; ++r) dsmem_arrive(dsmem_addr(&S.ub_empty, (uint32_t)r));
      }
    }
    // the last band's P2
    if (ok && nb > 0) ok = p2_read();
    // this cluster's partial plane of G: partial[z][l][col]
    if (ok) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c >= nch) break;
        const int64_t col = col0 + 128 * c + e;
        if (col < n) {
#pragma unroll
          for (int l = 0; l < FU_NT; ++l)
            if (l < count) partial[((int64_t)zc * count + l) * n + col] = (double)gacc[c][l];
        }
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  cluster_sync_all();  // no CTA leaves while a peer may still use its shared memory
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FU_TMEM_COLS) : "memory");
  }
}

}  // namespace

size_t oz_slices_bytes(int64_t rows, int64_t cols, int planes) {
  return sizeof(__nv_bfloat16) * (size_t)planes * (size_t)rows * (size_t)(cdiv(cols, OZ_KPAD) * OZ_KPAD);
}

tk_status oz_prepare(const void* X, tk_dtype dt, int64_t rows, int64_t cols, int64_t ld, void* slices, int* E,
                     cudaStream_t st, int planes) {
  if (rows == 0 || cols == 0) return TK_OK;
  const int64_t kp = cdiv(cols, OZ_KPAD) * OZ_KPAD;
  const bool f64 = dt == TK_F64;
  if (cols >= 16384 && rows <= 65535) {
    // few long rows (the residuals of the normal-equation pass): blocks of 8192 values per row
    const int64_t per = 8192;
    k_oz_fill_emin<<<(unsigned)cdiv(rows, 256), 256, 0, st>>>(E, rows);
    TK_LAUNCH_CHECK();
    const dim3 g((unsigned)cdiv(cols, per), (unsigned)rows);
    if (f64) k_oz_rowexp_long<double><<<g, 256, 0, st>>>((const double*)X, cols, ld, per, E);
    else k_oz_rowexp_long<float><<<g, 256, 0, st>>>((const float*)X, cols, ld, per, E);
    TK_LAUNCH_CHECK();
    k_oz_fix_zero_rows<<<(unsigned)cdiv(rows, 256), 256, 0, st>>>(E, rows);
  } else {
    const unsigned gr = (unsigned)cdiv(rows, 8);
    if (f64) k_oz_rowexp<double><<<gr, 256, 0, st>>>((const double*)X, rows, cols, ld, E);
    else k_oz_rowexp<float><<<gr, 256, 0, st>>>((const float*)X, rows, cols, ld, E);
  }
  TK_LAUNCH_CHECK();
  const int64_t chunks = cdiv(kp, 512);  // 256 threads x 2 values
  if (chunks > 65535) {
    set_error_msg("emulated float64 product: rows too long for the slicing grid");
    return TK_EINVAL;
  }
  const dim3 gs((unsigned)std::min<int64_t>(rows, std::max<int64_t>(1, 152 * 16 / chunks)), (unsigned)chunks);
  __nv_bfloat16* out = static_cast<__nv_bfloat16*>(slices);
  if (f64) k_oz_slice<double><<<gs, 256, 0, st>>>((const double*)X, rows, cols, ld, E, kp, planes, out);
  else k_oz_slice<float><<<gs, 256, 0, st>>>((const float*)X, rows, cols, ld, E, kp, planes, out);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

size_t oz_colmax_bytes(int64_t cols) { return sizeof(unsigned long long) * (size_t)std::max<int64_t>(cols, 1); }

tk_status oz_prepare_cols(const void* X, tk_dtype dt, int64_t rows, int64_t cols, int64_t ld, void* slices, int* E,
                          void* colmax, cudaStream_t st) {
  if (rows == 0 || cols == 0) return TK_OK;
  const int64_t rp = cdiv(rows, OZ_KPAD) * OZ_KPAD;
  unsigned long long* mx = static_cast<unsigned long long*>(colmax);
  TK_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * (size_t)cols, st));
  // about 4 CTAs of 256 columns per SM, each over a band of rows
  const int64_t cb = cdiv(cols, 256);
  const int64_t bands = std::max<int64_t>(1, std::min<int64_t>(cdiv(4 * 152, cb), cdiv(rows, 64)));
  const int64_t rows_per = cdiv(rows, bands);
  const dim3 gm((unsigned)cb, (unsigned)cdiv(rows, rows_per));
  if (cdiv(cols, 32) > 65535) {
    set_error_msg("emulated float64 product: too many columns for the slicing grid");
    return TK_EINVAL;
  }
  const dim3 gt((unsigned)cdiv(rp, 64), (unsigned)cdiv(cols, 32));
  __nv_bfloat16* out = static_cast<__nv_bfloat16*>(slices);
  if (dt == TK_F64) k_oz_colmax<double><<<gm, 256, 0, st>>>((const double*)X, rows, cols, ld, rows_per, mx);
  else k_oz_colmax<float><<<gm, 256, 0, st>>>((const float*)X, rows, cols, ld, rows_per, mx);
  TK_LAUNCH_CHECK();
  k_oz_colexp<<<(unsigned)cb, 256, 0, st>>>(mx, cols, E);
  TK_LAUNCH_CHECK();
  if (dt == TK_F64) k_oz_slice_t<double><<<gt, dim3(32, 8), 0, st>>>((const double*)X, rows, cols, ld, E, rp, out);
  else k_oz_slice_t<float><<<gt, dim3(32, 8), 0, st>>>((const float*)X, rows, cols, ld, E, rp, out);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

tk_status oz_residual(const void* Aslices, const int* EA, int64_t m, int64_t n, const void* Xslices, const int* EX,
                      int64_t M, const double* b, double* R, int64_t ldr, int* err, cudaStream_t st) {
  if (m == 0 || M == 0) return TK_OK;
  return launch_oz_tc<OZ_S, 0>(Aslices, EA, m, OZ_S, Xslices, EX, (int)M, OZ_S, n, 1, b, R, ldr, nullptr, err, st);
}

// Split count of a split-K digit product with `tiles` output tiles: the fewest
// waves (1..8) whose last wave is at least 97 % full, so that no SM idles
// through a ragged last wave (e.g. 64 tiles x 5 splits on 304 slots ran 1.05
// waves); at least 256 values of K per split.
int oz_normal_splits(int64_t m, int64_t n, int64_t M, int S) {
  const int nt = oz_tile_n(S, M);
  const int ctas_per_sm = (S == OZ_S || nt == 64) ? 1 : 2;
  const int64_t tiles = std::max<int64_t>(1, cdiv(n, OT_M) * cdiv(M, nt));
  const int64_t slots = 152 * (int64_t)ctas_per_sm;
  const int64_t maxs = std::max<int64_t>(1, cdiv(m, OT_CHUNK));
  int64_t best = 1;
  double best_eff = -1.0;
  for (int64_t w = 1; w <= 8; ++w) {
    const int64_t sp = std::min<int64_t>(cdiv(w * slots, tiles), maxs);
    const int64_t ctas = tiles * sp;
    const double eff = (double)ctas / (double)(cdiv(ctas, slots) * slots);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = sp;
    }
    if (eff >= 0.97 || sp == maxs) break;
  }
  return (int)std::max<int64_t>({int64_t(1), best, cdiv(m, OT_MAX_KPS)});  // at most 2^27 values of K per split
}

tk_status oz_normal(const void* AslicesT, const int* EC, int64_t m, int64_t n, const double* R, int64_t ldr,
                    int64_t M, void* Rslices, int* EX, double* partial, int splits, int* err, cudaStream_t st) {
  if (M == 0 || n == 0) return TK_OK;
  TK_TRY(oz_prepare(R, TK_F64, M, m, ldr, Rslices, EX, st));
  return launch_oz_tc<OZ_S, 1>(AslicesT, EC, n, OZ_S, Rslices, EX, (int)M, OZ_S, m, splits, nullptr, partial, n,
                               nullptr, err, st);
}

tk_status oz_lsqr_aw(const void* Aslices, const int* EA, int64_t m, int64_t n, const float* W, int64_t ldw, int count,
                     void* Wslices, int* EW, float* U, int64_t ldu, const double* coef, int* err, cudaStream_t st) {
  if (m == 0 || count == 0) return TK_OK;
  TK_TRY(oz_prepare(W, TK_F32, count, n, ldw, Wslices, EW, st, OZ_LSQR_DIGITS));
  return launch_oz_tc<OZ_LSQR_DIGITS, 2>(Aslices, EA, m, OZ_S, Wslices, EW, count, OZ_LSQR_DIGITS, n, 1, nullptr, U,
                                         ldu, coef, err, st);
}

tk_status oz_lsqr_atu(const void* AslicesT, const int* EC, int64_t m, int64_t n, const float* U, int64_t ldu,
                      int count, void* Uslices, int* EU, double* partial, int splits, int* err, cudaStream_t st) {
  if (n == 0 || count == 0) return TK_OK;
  TK_TRY(oz_prepare(U, TK_F32, count, m, ldu, Uslices, EU, st, OZ_LSQR_DIGITS));
  return launch_oz_tc<OZ_LSQR_DIGITS, 1>(AslicesT, EC, n, OZ_S, Uslices, EU, count, OZ_LSQR_DIGITS, m, splits,
                                         nullptr, partial, n, nullptr, err, st);
}

// Cluster shape of the fused step for n columns: CL CTAs (a power of two, at most 8, so that each
// CTA's share of a band's 128 rows is a multiple of 4) of cpc columns (a multiple of 128, at most
// 256); CL = 0 when n is beyond 8 x 256.
static void fused_shape(int64_t n, int* CL, int* cpc) {
  const int64_t n64 = cdiv(n, OZ_KPAD) * OZ_KPAD;
  const int64_t need = std::max<int64_t>(1, cdiv(n64, 256));
  int cl = 1;
  while (cl < need && cl < 8) cl *= 2;
  const int c = (int)(cdiv(n64, (int64_t)cl * 128) * 128);
  *CL = c <= 256 ? cl : 0;
  *cpc = c;
}

bool oz_fused_supported(int64_t m, int64_t n, int count) {
  int cl = 0, cpc = 0;
  fused_shape(n, &cl, &cpc);
  return cl > 0 && count >= 1 && count <= FU_NT && m >= 1 && m <= INT32_MAX;
}

tk_status oz_lsqr_fused(const void* Aslices, const int* EA, int64_t m, int64_t n, const float* W, int64_t ldw,
                        int count, void* Wslices, int* EW, float* U, int64_t ldu, const double* coef, double* partial,
                        int max_planes, int* planes, int* err, cudaStream_t st) {
  int CL = 0, cpc = 0;
  fused_shape(n, &CL, &cpc);
  if (!oz_fused_supported(m, n, count) || max_planes < 1) {
    set_error_msg("fused LSQR step: unsupported shape");
    return TK_EINVAL;
  }
  const int64_t n64 = cdiv(n, OZ_KPAD) * OZ_KPAD;
  TK_TRY(oz_prepare(W, TK_F32, count, n, ldw, Wslices, EW, st, OZ_LSQR_DIGITS));
  CUtensorMap mA, mW;
  TK_TRY(make_slice_map(&mA, Aslices, m, n64, OT_M, OZ_S));
  TK_TRY(make_slice_map(&mW, Wslices, count, n64, FU_NT, OZ_LSQR_DIGITS));
  const size_t smem = sizeof(FuSmem) + 1024;
  TK_CUDA(cudaFuncSetAttribute(k_oz_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // one wave of resident clusters, each looping over its bands (no second wave)
  static int cached[9] = {0};
  if (!cached[CL]) {
    cfg.gridDim = dim3((unsigned)((152 / CL) * CL), 1, 1);
    int nc = 0;
    TK_CUDA(cudaOccupancyMaxActiveClusters(&nc, k_oz_fused, &cfg));
    cached[CL] = nc > 0 ? nc : 1;
  }
  const int64_t bands = cdiv(m, FU_M);
  const int ncl = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)cached[CL], bands, (int64_t)max_planes}));
  cfg.gridDim = dim3((unsigned)(ncl * CL), 1, 1);
  TK_CUDA(cudaLaunchKernelEx(&cfg, k_oz_fused, mA, mW, EA, (const int*)EW, m, n, count, cpc, U, ldu, coef, partial,
                             err));
  TK_LAUNCH_CHECK();
  *planes = ncl;
  return TK_OK;
}

size_t oz_gram_workspace(int64_t r, int64_t c) {
  Arena a;
  a.take<char>(oz_slices_bytes(c, r));
  a.take<int>(c);
  a.take<char>(oz_colmax_bytes(c));
  return a.used + 256;
}

tk_status oz_gram(const double* Y, int64_t r, int64_t c, double* C, void* work, size_t bytes, int* err,
                  cudaStream_t st) {
  if (c == 0) return TK_OK;
  if (r == 0) {
    TK_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * (size_t)c * c, st));
    return TK_OK;
  }
  Arena a;
  a.base = static_cast<char*>(work);
  a.cap = bytes;
  void* Ys = a.take<char>(oz_slices_bytes(c, r));
  int* E = a.take<int>(c);
  void* mx = a.take<char>(oz_colmax_bytes(c));
  if (!a.ok()) return TK_ENOMEM;
  TK_TRY(oz_prepare_cols(Y, TK_F64, r, c, c, Ys, E, mx, st));
  return launch_oz_tc<OZ_S, 1>(Ys, E, c, OZ_S, Ys, E, (int)c, OZ_S, r, 1, nullptr, C, c, nullptr, err, st, 1);
}

size_t oz_chol_workspace(int64_t np, int N) {
  Arena a;
  a.take<__nv_bfloat16>((size_t)N * OZ_S * np * 64);
  a.take<int>((size_t)N * np);
  return a.used + 256;
}

tk_status oz_chol_begin(double* R, int64_t ldr, int64_t rstride, int N, int64_t np, void* work, size_t bytes,
                        int* err, OzCholPlan* plan, cudaStream_t st) {
  if (np % 64 || (int64_t)N * OZ_S > 65535 || np > INT32_MAX) {
    set_error_msg("emulated Cholesky: unsupported order or lambda count");
    return TK_EINVAL;
  }
  Arena a;
  a.base = static_cast<char*>(work);
  a.cap = bytes;
  const size_t sb = sizeof(__nv_bfloat16) * (size_t)N * OZ_S * np * 64;
  plan->slices = a.take<__nv_bfloat16>((size_t)N * OZ_S * np * 64);
  plan->EC = a.take<int>((size_t)N * np);
  if (!a.ok()) return TK_ENOMEM;
  plan->R = R;
  plan->ldr = ldr;
  plan->rstride = rstride;
  plan->N = N;
  plan->np = np;
  plan->err = err;
  // rows of the slice planes beyond a step's panel width are read by the
  // edge tiles (their products are discarded): keep them finite
  TK_CUDA(cudaMemsetAsync(plan->slices, 0, sb, st));
  EncodeTiledFn fn;
  TK_TRY(encode_fn(&fn));
  const cuuint64_t dims[3] = {64, (cuuint64_t)np, (cuuint64_t)N * OZ_S};
  const cuuint64_t strides[2] = {128, (cuuint64_t)np * 128};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int which = 0; which < 2; ++which) {
    const cuuint32_t box[3] = {64, which == 0 ? (cuuint32_t)CS_M : (cuuint32_t)CS_N, 1};
    CUresult r = fn(which == 0 ? &plan->mP : &plan->mQ, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, plan->slices, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error_msg("cuTensorMapEncodeTiled rejected the panel slice layout");
      return TK_ECUDA;
    }
  }
  TK_CUDA(cudaFuncSetAttribute(k_oz_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(CsSmem) + 1024)));
  return TK_OK;
}

tk_status oz_chol_step(const OzCholPlan& plan, int kb, cudaStream_t st) {
  const int64_t w = plan.np - (int64_t)(kb + 1) * 64;
  if (w <= 0) return TK_OK;
  __nv_bfloat16* sl = static_cast<__nv_bfloat16*>(plan.slices);
  k_oz_panel_slice<<<dim3((unsigned)cdiv(w, 32), (unsigned)plan.N), 256, 0, st>>>(plan.R, plan.ldr, plan.rstride,
                                                                                   plan.np, kb, sl, plan.EC);
  TK_LAUNCH_CHECK();
  const dim3 grid((unsigned)cdiv(w, CS_M), (unsigned)cdiv(w / CS_N, CS_TILES), (unsigned)plan.N);
  k_oz_syrk<<<grid, 384, sizeof(CsSmem) + 1024, st>>>(plan.mP, plan.mQ, plan.EC, plan.np, kb, plan.R, plan.ldr,
                                                     plan.rstride, plan.err);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

}  // namespace tk
