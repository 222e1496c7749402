// BP2 preconditioner (Section 4.1): for every lambda_l, the R factor of a QR
// decomposition of the partly exact sketch
//   B_l = [Y; sqrt(lambda_l) I_n]   ((s + n) x n,  Y = X A),
// in place of Algorithm 1's chol(Y^T Y + lambda_l I).  In exact arithmetic the
// two are the same factor (up to row signs); BP2 never forms Y^T Y, and each
// lambda costs a QR of an (s + n) x n matrix instead of an n x n Cholesky.
//
// Householder QR, one column at a time, all lambda per launch: B_l is kept
// column-major (each column contiguous, s + n values) so that a reflector and
// the columns it acts on are read as contiguous vectors.  Per column k:
//   k_hh_vec:   ||B_l[k:, k]||, alpha = -sign(b_kk) ||.||, v = B_l[k:, k] - alpha e_k
//               (stored in place), tau = 2 / v^T v = 1 / (nrm (nrm + |b_kk|));
//   k_hh_apply: B_l[k:, j] -= tau (v^T B_l[k:, j]) v for every j > k.
// R_l[i][j] = B_l[i, j] for j >= i, with row i scaled by sign(alpha_i) so that
// diag(R) > 0; the padding up to np holds the identity (as the Cholesky
// factors do).  A zero column records k + 1 in info[l] (TK_ENOTSPD), a NaN
// -(k + 1) (TK_ENUMERIC).
#include "tk_internal.cuh"

namespace tk {
namespace {

constexpr int kQrThreads = 256;

__global__ void k_qr_init(const double* __restrict__ Y, int64_t s, int64_t n, const double* __restrict__ lam,
                          double* __restrict__ B, int* __restrict__ info) {
  const int l = blockIdx.y;
  const int64_t M = s + n;
  double* Bl = B + (int64_t)l * n * M;
  const double sl = sqrt(lam[l]);
  if (blockIdx.x == 0 && threadIdx.x == 0) info[l] = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * M; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / M, i = e - j * M;
    Bl[e] = i < s ? Y[i * n + j] : (i - s == j ? sl : 0.0);
  }
}

// One block per lambda: the reflector of column k.
__global__ void __launch_bounds__(kQrThreads) k_hh_vec(double* __restrict__ B, int64_t s, int64_t n, int64_t k,
                                                       double* __restrict__ tau, double* __restrict__ alpha,
                                                       int* __restrict__ info) {
  __shared__ double sh[32];
  const int l = blockIdx.x;
  const int64_t M = s + n;
  double* col = B + ((int64_t)l * n + k) * M;
  double acc = 0.0;
  for (int64_t i = k + threadIdx.x; i < M; i += blockDim.x) acc = fma(col[i], col[i], acc);
  const double nrm = sqrt(block_sum(acc, sh));
  if (threadIdx.x == 0) {
    const double bkk = col[k];
    if (!(nrm > 0.0)) {  // zero column, or NaN
      if (info[l] == 0) info[l] = (nrm != nrm) ? -(int)(k + 1) : (int)(k + 1);
      tau[l] = 0.0;
      alpha[(int64_t)l * n + k] = nrm != nrm ? nrm : 1.0;
    } else {
      const double a = bkk > 0.0 ? -nrm : nrm;
      col[k] = bkk - a;  // v_k; the rest of v is the column below the diagonal
      tau[l] = 1.0 / (nrm * (nrm + fabs(bkk)));
      alpha[(int64_t)l * n + k] = a;
    }
  }
}

// Grid (trailing columns, lambda): one block per column j > k applies the reflector.
__global__ void __launch_bounds__(kQrThreads) k_hh_apply(double* __restrict__ B, int64_t s, int64_t n, int64_t k,
                                                         const double* __restrict__ tau) {
  __shared__ double sh[32];
  const int l = blockIdx.y;
  const int64_t j = k + 1 + blockIdx.x;
  if (j >= n) return;
  const int64_t M = s + n;
  const double* v = B + ((int64_t)l * n + k) * M;
  double* c = B + ((int64_t)l * n + j) * M;
  double acc = 0.0;
  for (int64_t i = k + threadIdx.x; i < M; i += blockDim.x) acc = fma(v[i], c[i], acc);
  const double d = block_sum(acc, sh) * tau[l];
  for (int64_t i = k + threadIdx.x; i < M; i += blockDim.x) c[i] = fma(-d, v[i], c[i]);
}

// R_l (row-major, row stride ldr, matrix stride rstride, np x np): the upper
// triangle of the reduced B_l with row signs making diag(R) > 0, identity on
// the padding, zeros below the diagonal.
__global__ void k_qr_extract(const double* __restrict__ B, int64_t s, int64_t n, int64_t np,
                             const double* __restrict__ alpha, double* __restrict__ R, int64_t ldr, int64_t rstride) {
  const int l = blockIdx.y;
  const int64_t M = s + n;
  const double* Bl = B + (int64_t)l * n * M;
  double* Rl = R + (int64_t)l * rstride;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < np * np; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / np, j = e - i * np;
    double v = 0.0;
    if (i < n && j < n) {
      if (j > i) {
        const double a = alpha[(int64_t)l * n + i];
        v = a < 0.0 ? -Bl[j * M + i] : Bl[j * M + i];
      } else if (j == i) {
        v = fabs(alpha[(int64_t)l * n + i]);
      }
    } else if (i == j) {
      v = 1.0;
    }
    Rl[i * ldr + j] = v;
  }
}

}  // namespace

size_t bp2_workspace(int64_t s, int64_t n, int N) {
  Arena a;
  a.take<double>((size_t)N * n * (s + n));
  a.take<double>((size_t)N);
  a.take<double>((size_t)N * n);
  return a.used + 512;
}

tk_status bp2_factor(const double* Y, int64_t s, int64_t n, const double* lam_dev, int N, double* R, int64_t np,
                     int64_t ldr, int64_t rstride, int* info_dev, void* work, size_t bytes, cudaStream_t st) {
  if (N == 0 || n == 0) return TK_OK;
  if (n - 1 > 65535 || N > 65535) {
    set_error_msg("BP2: more than 65536 columns or lambdas");
    return TK_EINVAL;
  }
  Arena a;
  a.base = static_cast<char*>(work);
  a.cap = bytes;
  double* B = a.take<double>((size_t)N * n * (s + n));
  double* tau = a.take<double>((size_t)N);
  double* alpha = a.take<double>((size_t)N * n);
  if (!a.ok()) return TK_ENOMEM;
  const int64_t M = s + n;
  const unsigned gi = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(n * M, 256), 152 * 8));
  k_qr_init<<<dim3(gi, (unsigned)N), 256, 0, st>>>(Y, s, n, lam_dev, B, info_dev);
  TK_LAUNCH_CHECK();
  for (int64_t k = 0; k < n; ++k) {
    k_hh_vec<<<N, kQrThreads, 0, st>>>(B, s, n, k, tau, alpha, info_dev);
    if (k + 1 < n) k_hh_apply<<<dim3((unsigned)(n - 1 - k), (unsigned)N), kQrThreads, 0, st>>>(B, s, n, k, tau);
    TK_LAUNCH_CHECK();
  }
  const unsigned ge = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(np * np, 256), 152 * 8));
  k_qr_extract<<<dim3(ge, (unsigned)N), 256, 0, st>>>(B, s, n, np, alpha, R, ldr, rstride);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

}  // namespace tk
