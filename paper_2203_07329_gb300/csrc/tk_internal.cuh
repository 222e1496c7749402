// Internal declarations shared by the CUDA translation units of libtikhonov.
// Nothing here is part of the C ABI (include/tikhonov.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <algorithm>
#include <vector>

#include "tikhonov.h"

namespace tk {

// ---------------------------------------------------------------- errors --
void set_error(cudaError_t e, const char* file, int line);
void set_error_msg(const char* msg);

#define TK_CUDA(x)                                 \
  do {                                             \
    cudaError_t e__ = (x);                         \
    if (e__ != cudaSuccess) {                      \
      ::tk::set_error(e__, __FILE__, __LINE__);    \
      return TK_ECUDA;                             \
    }                                              \
  } while (0)

// Every kernel launch of the library is followed by TK_LAUNCH_CHECK(), which
// also counts it (tk_launch_count()).
void count_launch();
void count_launches(size_t n);  // n kernels of a replayed graph
#define TK_LAUNCH_CHECK()   \
  do {                      \
    ::tk::count_launch();   \
    TK_CUDA(cudaGetLastError()); \
  } while (0)

#define TK_TRY(x)                  \
  do {                             \
    tk_status s__ = (x);           \
    if (s__ != TK_OK) return s__;  \
  } while (0)

// Per-lambda status order: the worse of two statuses is kept.
inline int severity(tk_status s) {
  switch (s) {
    case TK_OK: return 0;
    case TK_ENOCONV: return 1;
    case TK_ENUMERIC: return 2;
    case TK_ENOTSPD: return 3;
    default: return 4;
  }
}
inline tk_status worse(tk_status a, tk_status b) { return severity(b) > severity(a) ? b : a; }

// Stop rule of the mixed form's refinement after round `round` produced a
// correction of norm dn (the previous one pd; the first correction is x
// itself) on x of norm xn: done when the correction is below tol ||x||, when
// the next correction predicted from the observed contraction, dn * (dn / pd),
// is below tol ||x|| / 10, when the corrections stopped halving (x sits at the
// float64 floor of the residual), or when dn is not finite.
inline bool refine_done(int round, double dn, double pd, double xn, double tol) {
  if (!(dn == dn) || dn > 1e300) return true;
  if (dn <= tol * xn) return true;
  if (round >= 1 && pd > 0.0 && pd < 1e300 && dn * (dn / pd) <= 0.1 * tol * xn) return true;
  return round >= 2 && dn > 0.5 * pd;
}

// ------------------------------------------------------------ workspace --
// Bump allocator over a caller-provided device buffer (256-byte aligned
// slices).  With base == nullptr it only measures.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    if (!base) return nullptr;
    return reinterpret_cast<T*>(base + off);
  }
  bool ok() const { return base == nullptr || used <= cap; }
};

inline int64_t next_pow2(int64_t m) {
  int64_t p = 1;
  while (p < m) p <<= 1;
  return p;
}
inline int ilog2(int64_t p) {
  int a = 0;
  while ((int64_t(1) << a) < p) ++a;
  return a;
}
__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// --------------------------------------------------- Philox4x32-10 (GPU) --
// Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten
// rounds of two 32x32 multiplies; the key advances by the Weyl constants
// after each round.  Counter = (index lo, index hi, stream, 0), key = seed.
__device__ __forceinline__ uint4 philox(uint64_t index, uint32_t stream, uint64_t seed) {
  uint32_t x0 = (uint32_t)index, x1 = (uint32_t)(index >> 32), x2 = stream, x3 = 0u;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t h0 = __umulhi(0xD2511F53u, x0), l0 = 0xD2511F53u * x0;
    uint32_t h1 = __umulhi(0xCD9E8D57u, x2), l1 = 0xCD9E8D57u * x2;
    uint32_t y0 = h1 ^ x1 ^ k0, y2 = h0 ^ x3 ^ k1;
    x0 = y0; x1 = l1; x2 = y2; x3 = l0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(x0, x1, x2, x3);
}

enum : uint32_t { STREAM_SIGNS = 0, STREAM_KEYS = 1, STREAM_GAUSS = 2, STREAM_SPARSE = 4 };

// Gaussian entry k of an embedding with N(0, 1/s) entries: Philox call k/4 of
// stream 2, Box-Muller on word pairs (w0, w1) and (w2, w3).
__device__ __forceinline__ double gauss_entry(uint64_t seed, uint64_t k, double inv_sqrt_s) {
  uint4 w = philox(k >> 2, STREAM_GAUSS, seed);
  int lane = (int)(k & 3u);
  uint32_t a = (lane < 2) ? w.x : w.z;
  uint32_t b = (lane < 2) ? w.y : w.w;
  double u1 = ((double)a + 1.0) * 2.3283064365386962890625e-10;
  double u2 = (double)b * 2.3283064365386962890625e-10;
  double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return ((lane & 1) ? r * sn : r * cs) * inv_sqrt_s;
}

// -------------------------------------------------------------- reduce --
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread gets the result.  `sh` needs 32 entries.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  T t = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  T r = sh[0];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------ profiler --
bool prof_enabled();
int prof_begin(int phase, cudaStream_t st);
// bytes: the operation's own (each operand once, A in the caller's dtype); impl_bytes: what the
// implementation moves (digit planes, copies), < 0 = the same
void prof_end(int tok, cudaStream_t st, double flops, double bytes, double impl_bytes = -1.0);

// --------------------------------------------------------- launchers -----
// Draws (tk_draw.cu)
size_t draw_workspace(int64_t mp);
tk_status draw_signs_rows(uint64_t seed, int64_t mp, int64_t s, int8_t* signs, int64_t* rows, int32_t* rowmap,
                          Arena& ar, cudaStream_t st);

// Sketches (tk_sketch.cu).  Y = X A (s x cols) of the "long axis first"
// layout: the transform runs along the rows of a (L x cols) matrix with
// row stride ld.  Output Y is s x cols float64.
tk_status srht_rows(const void* A, tk_dtype dt, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s,
                    double* Y, Arena& ar, cudaStream_t st);
size_t srht_rows_workspace(int64_t L, int64_t cols, tk_dtype dt, int64_t s);
tk_status gauss_rows(const void* A, tk_dtype dt, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s,
                     double* Y, Arena& ar, cudaStream_t st);
size_t gauss_rows_workspace(int64_t L, int64_t cols, tk_dtype dt, int64_t s);
// SRDCT (tk_sketch.cu): X = sqrt(Lp/s) S C D [I; 0], C the orthonormal DCT-II of length Lp.
tk_status srdct_rows(const void* A, tk_dtype dt, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s,
                     double* Y, Arena& ar, cudaStream_t st);
size_t srdct_rows_workspace(int64_t L, int64_t cols, tk_dtype dt, int64_t s);
// Sparse embedding (tk_sparse.cu): one signed entry per column of X (s x L).
constexpr int64_t kSparseMaxS = int64_t(1) << 22;
tk_status sparse_rows(const void* A, tk_dtype dt, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s,
                      double* Y, Arena& ar, cudaStream_t st);
size_t sparse_rows_workspace(int64_t L, int64_t cols, int64_t s);
// the draws and the rows sorted by bucket (ascending row within a bucket) on their own, for parity tests
tk_status sparse_draw_sorted(uint64_t seed, int64_t L, int64_t s, int32_t* h, int8_t* sign, int32_t* order,
                             int32_t* start, Arena& ar, cudaStream_t st);
tk_status transpose(const void* A, tk_dtype dt, int64_t rows, int64_t cols, int64_t lda, void* AT,
                    cudaStream_t st);
tk_status convert_f64_to_f32(const double* src, float* dst, int64_t rows, int64_t cols, int64_t lds, int64_t ldd,
                             cudaStream_t st);

// Tensor-core BF16 Gaussian sketch (tk_tc.cu): Y (s x n) = G A, A m x n.
size_t tc_sketch_workspace(int64_t m, int64_t n, int64_t s);
tk_status tc_gauss_sketch(const void* A, tk_dtype dt, int64_t m, int64_t n, int64_t lda, uint64_t seed, int64_t s,
                          double* Y, Arena& ar, cudaStream_t st);

// Tensor-core LSQR products (tk_tc.cu), float32 operands, 3-term TF32 split.
size_t tc_lmaj_workspace(int N_cap, int64_t K);
tk_status tc_lmaj_product(bool update, const float* X, int64_t rows, int64_t K, int64_t ldx, const float* L,
                          int64_t ldl, int N, float* U, int64_t ldu, const double* coef, double* partial, int splits,
                          void* scratch, cudaStream_t st);
tk_status tc_lmaj_check(void* scratch, int N, int64_t K, cudaStream_t st);

// Measured GEMM choices (tk_tune.cu): key = operand types (0 float, 1
// double), transposes, split-K or not, M (rounded up to a power of two), N, K.
struct GemmKey {
  int ta = 0, tb = 0, tc = 0, transA = 0, transB = 0, split = 0;
  int64_t M = 0, N = 0, K = 0;
};
struct TuneChoice {
  int cfg = -1;    // tile configuration index of the generic kernel (-1: the fixed rule)
  int splits = 0;  // split count of a split-K product (0: the caller's)
};
int64_t tune_bucket(int64_t M);
bool tune_lookup(GemmKey k, TuneChoice* out);
void tune_store(GemmKey k, TuneChoice c);
size_t tune_size();
size_t tune_describe(char* buf, size_t len);
void tune_clear();
template <typename T>
constexpr int dtype_code() {
  return sizeof(T) == 8 ? 1 : 0;
}

// Float64-accurate products on the BF16 tensor cores (tk_oz.cu).  The rows of
// X (rows x cols, row stride ld) are split into 8 exact BF16 slice planes
// (row stride cols rounded up to 64) with row exponents E (oz_prepare), or the
// columns of X into planes of X^T with column exponents (oz_prepare_cols:
// slices bytes oz_slices_bytes(cols, rows), E: cols ints, colmax:
// oz_colmax_bytes(cols)).  *err (device) is set if a pipeline wait timed out.
constexpr int OZ_LSQR_DIGITS = 4;  // digits of the float32-accurate LSQR products
size_t oz_slices_bytes(int64_t rows, int64_t cols, int planes = 8);
tk_status oz_prepare(const void* X, tk_dtype dt, int64_t rows, int64_t cols, int64_t ld, void* slices, int* E,
                     cudaStream_t st, int planes = 8);
size_t oz_colmax_bytes(int64_t cols);
tk_status oz_prepare_cols(const void* X, tk_dtype dt, int64_t rows, int64_t cols, int64_t ld, void* slices, int* E,
                          void* colmax, cudaStream_t st);
// R[l][i] = b[i] - sum_k X[l][k] A[i][k] from the row slices of A (m x n) and
// of X (M x n).
tk_status oz_residual(const void* Aslices, const int* EA, int64_t m, int64_t n, const void* Xslices, const int* EX,
                      int64_t M, const double* b, double* R, int64_t ldr, int* err, cudaStream_t st);
// The normal-equation pass: partial[z][l][j] (z < splits; unused planes zero)
// of sum_i A[i][j] R[l][i], from the column slices of A (oz_prepare_cols) and
// R (M x m, row stride ldr); Rslices: oz_slices_bytes(M, m), EX: M ints.
int oz_normal_splits(int64_t m, int64_t n, int64_t M, int S = 8);  // S: digits of the product (4 or 8)
// Cholesky of C + lambda I (chol_shifted) with the trailing updates on the
// tensor cores: oz_chol_begin prepares the slice buffers and tensor maps
// (work: oz_chol_workspace(np, N) bytes), oz_chol_step(kb) replaces the
// float64 update of block step kb.
struct OzCholPlan {
  CUtensorMap mP;
  CUtensorMap mQ;
  double* R = nullptr;
  int64_t ldr = 0, rstride = 0, np = 0;
  int N = 0;
  void* slices = nullptr;
  int* EC = nullptr;
  int* err = nullptr;
};
size_t oz_chol_workspace(int64_t np, int N);
tk_status oz_chol_begin(double* R, int64_t ldr, int64_t rstride, int N, int64_t np, void* work, size_t bytes,
                        int* err, OzCholPlan* plan, cudaStream_t st);
tk_status oz_chol_step(const OzCholPlan& plan, int kb, cudaStream_t st);
// The two float32 LSQR products from the first 4 digits of the slices of A
// (the 28-bit rounded A) and of the lambda-major vectors, sliced here
// (Wslices / Uslices: oz_slices_bytes(count, n or m, 4); EW / EU: count ints):
//   aw:  U[l][i] = sum_k W[l][k] A[i][k] + coef[l] U[l][i]  (coef may be null);
//   atu: partial[z][l][j] = sum_{i in split z} U[l][i] A[i][j].
tk_status oz_lsqr_aw(const void* Aslices, const int* EA, int64_t m, int64_t n, const float* W, int64_t ldw, int count,
                     void* Wslices, int* EW, float* U, int64_t ldu, const double* coef, int* err, cudaStream_t st);
// The two products of one LSQR step fused over one read of A's row-exponent digit planes (count <= 32,
// n <= 2048): U <- W A^T + coef .* U in place, and partial[z] (z < *planes <= max_planes; count x n
// float64 planes) whose sum is U A for the new U.  Wslices / EW as oz_lsqr_aw.
bool oz_fused_supported(int64_t m, int64_t n, int count);
tk_status oz_lsqr_fused(const void* Aslices, const int* EA, int64_t m, int64_t n, const float* W, int64_t ldw,
                        int count, void* Wslices, int* EW, float* U, int64_t ldu, const double* coef, double* partial,
                        int max_planes, int* planes, int* err, cudaStream_t st);
tk_status oz_lsqr_atu(const void* AslicesT, const int* EC, int64_t m, int64_t n, const float* U, int64_t ldu,
                      int count, void* Uslices, int* EU, double* partial, int splits, int* err, cudaStream_t st);
// Float32 LSQR products for at most 16 lambda from the float32 A (m x n, row
// stride lda): aw: C[l][i] = sum_k W[l][k] A[i][k] (+ beta[l] C[l][i]; beta may
// be null), W (count x n) held in shared memory (lm_small_aw_supported);
// atu: partial[z][l][j] (z < splits, count x n planes) whose sum is U A.
bool lm_small_aw_supported(int64_t n, int count);
tk_status lm_small_aw(const float* A, int64_t lda, int64_t m, int64_t n, const float* W, int64_t ldw, int count,
                      float* C, int64_t ldc, const double* beta, cudaStream_t st);
int lm_small_atu_splits(int64_t m, int64_t n);
tk_status lm_small_atu(const float* A, int64_t lda, int64_t m, int64_t n, const float* U, int64_t ldu, int count,
                       double* partial, int splits, cudaStream_t st);
// C = Y^T Y (Y: r x c float64, row stride c), the upper triangle (j >= i) of
// C (c x c) written, float64-accurate; work: oz_gram_workspace(r, c) bytes.
size_t oz_gram_workspace(int64_t r, int64_t c);
tk_status oz_gram(const double* Y, int64_t r, int64_t c, double* C, void* work, size_t bytes, int* err,
                  cudaStream_t st);
tk_status oz_normal(const void* AslicesT, const int* EC, int64_t m, int64_t n, const double* R, int64_t ldr,
                    int64_t M, void* Rslices, int* EX, double* partial, int splits, int* err, cudaStream_t st);

// Dense kernels (tk_dense.cu)
template <typename TA, typename TB, typename TC>
tk_status gemm(bool transA, bool transB, int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda, const TB* B,
               int64_t ldb, TC* C, int64_t ldc, double alpha, const double* beta_row, const TC* Cin,
               int64_t ldcin, cudaStream_t st);
template <typename TA, typename TB>
tk_status gemm_splitk(bool transA, bool transB, int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda,
                      const TB* B, int64_t ldb, double* partial, int splits, cudaStream_t st);
int splitk_count(int64_t M, int64_t N, int64_t K);
// The split count a split-K product of this shape runs with: the measured one
// (<= cap) when tk_autotune() recorded it, else cap (the buffer's capacity).
template <typename TA, typename TB>
int splitk_tuned(int64_t M, int64_t N, int64_t K, int cap);
// Times the candidate tile shapes (and split counts <= split_cap when partial
// is set) of one product shape on the stream and records the fastest.
template <typename TA, typename TB, typename TC>
tk_status tune_gemm(bool transA, bool transB, int64_t M, int64_t N, int64_t K, const TA* A, int64_t lda, const TB* B,
                    int64_t ldb, TC* C, int64_t ldc, double alpha, const double* beta_row, const TC* Cin,
                    int64_t ldcin, int split_cap, double* partial, cudaStream_t st);
// Gram matrix C = Y^T Y, upper triangle only (what the Cholesky reads).
// scratch (optional, gram_scratch_bytes(r, c)): split-K partials when the
// upper triangle has few 64 x 64 tiles (a small n).
size_t gram_scratch_bytes(int64_t r, int64_t c);
tk_status gram_upper(const double* Y, int64_t r, int64_t c, double* C, void* scratch, size_t scratch_bytes,
                     cudaStream_t st);

size_t chol_workspace(int64_t n, int N);
// BP2 (tk_qr.cu, Section 4.1): R_l from a Householder QR of [Y; sqrt(l) I] for every lambda (diag > 0, identity
// padding up to np); info as chol_shifted (NaN: negative).
size_t bp2_workspace(int64_t s, int64_t n, int N);
tk_status bp2_factor(const double* Y, int64_t s, int64_t n, const double* lam_dev, int N, double* R, int64_t np,
                     int64_t ldr, int64_t rstride, int* info_dev, void* work, size_t bytes, cudaStream_t st);
tk_status chol_shifted(const double* C, int64_t n, const double* lambdas_dev, int N, double* R, int64_t ldr,
                       int64_t rstride, int* info_dev, Arena& ar, cudaStream_t st, const OzCholPlan* oz = nullptr);

// M = R^-1 (upper) and Mt = M^T (lower), arithmetic in T, for N factors R
// (float64, padded order np = ceil(n/64)*64, row stride ldr, matrix stride
// rstride); M and Mt: N x np x np, row stride np.
template <typename T>
tk_status tri_inverse(const double* R, int64_t n, int64_t ldr, int64_t rstride, int N, T* M, T* Mt, cudaStream_t st);
// out_k = M_l in_k (or Mt_l in_k when transposed) for slots k < count,
// l = idx[k] (idx null: l = k); in/out vectors of length n at stride ldx
// (out must not overlap in).
template <typename T>
tk_status trmv_batched(bool transposed, int64_t n, const T* M, const T* Mt, int64_t ldm, int64_t mstride,
                       const int* idx, const T* in, T* out, int64_t ldx, int count, cudaStream_t st);

// Batched triangular solves on slots: vector of slot j is X + j*ldx (length
// n); its factor is R + idx[j]*rstride (row stride ldr, upper triangular).
// pbuf (float64, count x n) enables the grid-wide column sweep for n > 512;
// with pbuf == nullptr one CTA solves each slot.  Xin may equal X.
template <typename TR, typename TX>
tk_status trsv_batched(bool transposed, int64_t n, const TR* R, int64_t ldr, int64_t rstride, const int* idx,
                       const TX* Xin, TX* X, int64_t ldx, int count, double* pbuf, cudaStream_t st);

// Low rank (tk_lowrank.cu)
size_t svd_workspace(int64_t s, int64_t n);
// Many one-sided Jacobi SVDs at once (grouped batch): every round of the
// circle schedule is one launch over the pairs of all matrices still rotating.
struct SvdJob {
  const double* Y = nullptr;  // s x n (read only)
  int64_t s = 0, n = 0;
  double* sigma = nullptr;    // s, descending
  double* V = nullptr;        // n x s
  void* scratch = nullptr;    // svd_workspace(s, n) bytes
  size_t scratch_bytes = 0;
  int sweeps = 0;             // out
  double* W = nullptr;        // carved from scratch
  double* nrm = nullptr;
  int* perm = nullptr;
};
size_t svd_grouped_workspace(const std::vector<SvdJob>& jobs);
tk_status jacobi_svd_grouped(std::vector<SvdJob>& jobs, void* work, size_t work_bytes, cudaStream_t st);
tk_status jacobi_svd(const double* Y, int64_t s, int64_t n, double* sigma, double* V, int* sweeps_host, Arena& ar,
                     cudaStream_t st);

}  // namespace tk
