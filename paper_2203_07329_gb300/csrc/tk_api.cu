// C ABI of libtikhonov: argument checks, workspace planning and the order of
// the steps of Algorithms 1, 2 and 3 (and the mixed-precision refinement
// around Algorithm 1).  Every numerical step runs in the kernels of the other
// translation units; this file only sequences them.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "tk_group.cuh"
#include "tk_lsqr.cuh"

namespace tk {

thread_local char g_err[512] = "";

void set_error(cudaError_t e, const char* file, int line) {
  snprintf(g_err, sizeof g_err, "%s (%s:%d)", cudaGetErrorString(e), file, line);
}
void set_error_msg(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

namespace {

tk_status einval(const char* msg) {
  set_error_msg(msg);
  return TK_EINVAL;
}


// ---------------------------------------------------------------- plan -----
struct Plan {
  int64_t m = 0, n = 0, lda = 0;
  tk_dtype dt = TK_F64;
  bool under = false;
  int64_t L = 0, c = 0;  // long and short dimension
  int64_t s = 0;
  int64_t np = 0;        // Cholesky order padded to the 64 tile
  int N = 0, N_cap = 0;
  tk_opts o{};
  bool mixed = false, lowrank = false;
  bool qr = false;        // BP2: R from a QR of [Y; sqrt(l) I] instead of chol(Y^T Y + l I)
  bool lsqr_tc = false;  // tensor-core float32 LSQR products (3-term TF32)
  bool lsqr_oz = false;  // float32 LSQR products from the 4-digit slices of A
  bool lsqr_fused = false;  // ... both products of a step in one kernel
  bool prep_only = false;  // grouped batch: build the preconditioner only
  bool inv64 = false;      // float64 form: explicit float64 R^-1 (small factors)
};

constexpr int64_t kMaxShort = 8192;
constexpr int64_t kMaxLong = (int64_t(1) << 30);

tk_status check_opts(const tk_opts* o) {
  if (!o) return einval("options pointer is NULL");
  if (o->sketch != TK_SKETCH_SRHT && o->sketch != TK_SKETCH_GAUSS && o->sketch != TK_SKETCH_SPARSE &&
      o->sketch != TK_SKETCH_SRDCT)
    return einval("unknown sketch kind");
  if (o->precond != TK_PRECOND_CHOL && o->precond != TK_PRECOND_LOWRANK && o->precond != TK_PRECOND_QR)
    return einval("unknown preconditioner");
  if (o->precision != TK_PREC_FP64 && o->precision != TK_PREC_MIXED) return einval("unknown precision");
  if (o->schedule != TK_SCHED_BATCHED && o->schedule != TK_SCHED_ONE_AT_A_TIME) return einval("unknown schedule");
  if (o->lsqr_tc < 0 || o->lsqr_tc > 3) return einval("lsqr_tc must be 0, 1, 2 or 3");
  if (!(o->tol > 0.0) || !std::isfinite(o->tol)) return einval("tol must be a positive finite number");
  if (o->maxiter < 1) return einval("maxiter must be >= 1");
  if (o->s < 0) return einval("sketch size s must be >= 0");
  if (o->precond == TK_PRECOND_LOWRANK && !(o->alpha >= 1.0 && std::isfinite(o->alpha)))
    return einval("alpha must be >= 1");
  if (o->precision == TK_PREC_MIXED) {
    if (o->max_refine < 1) return einval("max_refine must be >= 1");
    if (!(o->inner_tol > 0.0) || !(o->refine_tol > 0.0)) return einval("inner_tol and refine_tol must be > 0");
  }
  return TK_OK;
}

tk_status make_plan(const tk_problem* p, int N, const tk_opts* o, Plan& P) {
  if (!p) return einval("problem pointer is NULL");
  TK_TRY(check_opts(o));
  if (p->m < 1 || p->n < 1) return einval("m and n must be >= 1");
  if (p->lda < p->n) return einval("lda must be >= n");
  if (p->dtype != TK_F64 && p->dtype != TK_F32) return einval("unknown dtype");
  if (N < 0) return einval("N must be >= 0");
  P.m = p->m;
  P.n = p->n;
  P.lda = p->lda;
  P.dt = p->dtype;
  P.under = p->m < p->n;
  P.L = std::max(p->m, p->n);
  P.c = std::min(p->m, p->n);
  if (P.c > kMaxShort) return einval("min(m, n) above 8192 is not supported");
  if (P.L > kMaxLong) return einval("max(m, n) above 2^30 is not supported");
  P.o = *o;
  P.N = N;
  P.mixed = o->precision == TK_PREC_MIXED;
  P.lowrank = o->precond == TK_PRECOND_LOWRANK;
  P.qr = o->precond == TK_PRECOND_QR;
  if (P.under && P.mixed) return einval("the mixed-precision form is built for m >= n");
  if (P.under && P.qr) return einval("the BP2 (QR) preconditioner is built for m >= n");
  if (P.under && o->x0) return einval("the warm start x0 is supported for m >= n (Algorithms 1 and 3)");
  int64_t s = o->s;
  // the sparse embedding needs more rows for the same distortion (Theorem 3.5: s grows with sd^2)
  if (s == 0) s = P.lowrank ? P.c : std::min<int64_t>((o->sketch == TK_SKETCH_SPARSE ? 16 : 4) * P.c, P.L);
  if ((o->sketch == TK_SKETCH_SRHT || o->sketch == TK_SKETCH_SRDCT) && s > next_pow2(P.L))
    return einval("SRHT / SRDCT sketch size exceeds the padded length");
  if (o->sketch == TK_SKETCH_SPARSE && s > kSparseMaxS) return einval("sparse sketch size above 2^22");
  if (P.lowrank && s > P.c) s = P.c;  // alpha * sd <= n (Algorithm 3); a full-size sketch is still exact
  P.s = s;
  P.np = cdiv(P.c, 64) * 64;
  P.N_cap = (o->schedule == TK_SCHED_ONE_AT_A_TIME) ? 1 : std::max(N, 1);
  // the tensor-core products need 16-byte aligned float32 rows of A, A^T and
  // the lambda-major vectors; other shapes keep the SIMT float32 products
  // small float64 factors: an explicit inverse costs N n^3/3 flops once and
  // turns each preconditioner apply into one launch (substitution on a
  // factor of order <= 512 runs in a single CTA per lambda)
  P.inv64 = !P.mixed && !P.lowrank && !P.under && P.c <= 512;
  P.lsqr_tc = P.mixed && o->lsqr_tc == 1 && P.N_cap <= 64 && !P.under && P.m % 4 == 0 && P.n % 4 == 0 &&
              (P.dt == TK_F64 || P.lda % 4 == 0);
  P.lsqr_oz = P.mixed && (o->lsqr_tc == 2 || o->lsqr_tc == 3) && o->emulate_fp64 && !P.under;
  P.lsqr_fused = P.lsqr_oz && o->lsqr_tc == 3;
  return TK_OK;
}

// Device buffers of one solve, carved from the caller's workspace.
struct Bufs {
  double* lam = nullptr;
  int* ids = nullptr;
  int* info = nullptr;
  double* ones = nullptr;
  double* Y = nullptr;
  void* AT = nullptr;
  float* A32 = nullptr;
  float* AT32 = nullptr;
  double* A64 = nullptr;
  double* C = nullptr;
  double* R = nullptr;
  float* Minv = nullptr;   // mixed: R^-1 in float32 (N x np x np)
  float* Mtinv = nullptr;  // mixed: R^-T in float32
  double* Minv64 = nullptr;   // float64 form, small factors: R^-1
  double* Mtinv64 = nullptr;  // and R^-T
  double* sig = nullptr;
  double* lrV = nullptr;
  double* lrS = nullptr;
  float* lrV32 = nullptr;
  float* lrS32 = nullptr;
  int64_t* ranks = nullptr;
  double* sd = nullptr;
  double* D = nullptr;
  double* Xa = nullptr;
  double* G = nullptr;
  double* Rres = nullptr;
  double* part = nullptr;
  double* nrm = nullptr;
  void* Aoz = nullptr;      // mixed, emulate_fp64: BF16 slices of A and their row exponents
  int* EA = nullptr;
  void* Xoz = nullptr;      // ... and of the lambda rows of x
  int* EX = nullptr;
  void* AozC = nullptr;     // ... the column-scaled slices of A, their column exponents
  int* EC = nullptr;
  void* colmax = nullptr;
  int* oz_err = nullptr;    // set by a timed-out wait of the emulated products
  void* Roz = nullptr;      // ... and of the residuals (normal-equation pass)
  int* ER = nullptr;
  char* scratch = nullptr;  // sketch scratch
  size_t scratch_bytes = 0;
  char* svd = nullptr;      // SVD scratch (low rank)
  size_t svd_bytes = 0;
  Lsqr<double> e64;
  Lsqr<float> e32;
  int splits = 1;
};

// The mixed form's Gaussian sketch of an overdetermined A runs on the tensor
// cores (BF16 operands, FP32 accumulation); every other sketch is SIMT.
bool tc_sketch(const Plan& P) { return P.mixed && P.o.sketch == TK_SKETCH_GAUSS && !P.under; }

// The mixed form with emulate_fp64 forms its Gram matrix from exact slices on
// the tensor cores (float64 accuracy).
bool emulated_gram(const Plan& P) { return P.mixed && P.o.emulate_fp64 && !P.lowrank && !P.qr; }

size_t sketch_scratch(const Plan& P) {
  tk_dtype dt = P.mixed ? TK_F32 : P.dt;
  if (tc_sketch(P)) return tc_sketch_workspace(P.L, P.c, P.s);
  if (P.o.sketch == TK_SKETCH_SRHT) return srht_rows_workspace(P.L, P.c, dt, P.s);
  if (P.o.sketch == TK_SKETCH_SPARSE) return sparse_rows_workspace(P.L, P.c, P.s);
  if (P.o.sketch == TK_SKETCH_SRDCT) return srdct_rows_workspace(P.L, P.c, dt, P.s);
  return gauss_rows_workspace(P.L, P.c, dt, P.s);
}

// `a` holds what the LSQR phase reads (lambda, A copies, the float32
// preconditioner, the LSQR and refinement state), `t` what only the
// preconditioner build needs (sketch, Gram, float64 factors, SVD); a single
// solve passes the same arena twice.  prep_only (grouped batch) skips the
// LSQR and refinement state, which the grouped engine owns.
void carve(const Plan& P, Arena& a, Arena& t, Bufs& B) {
  const int N = std::max(P.N, 1);
  // grouped low-rank problems: the SVD runs later over all problems at once,
  // so the sketch and the SVD buffers outlive the build
  Arena& ty = (P.prep_only && P.lowrank) ? a : t;
  B.lam = a.take<double>(N);
  B.ids = a.take<int>(N);
  B.info = a.take<int>(N);
  B.ones = a.take<double>(N);
  B.Y = ty.take<double>((size_t)P.s * P.c);
  if (P.under) B.AT = t.take<char>((size_t)P.m * P.n * (P.dt == TK_F64 ? 8 : 4));
  if (P.mixed && P.dt == TK_F64) B.A32 = a.take<float>((size_t)P.m * P.n);
  if (P.lsqr_tc) B.AT32 = a.take<float>((size_t)P.m * P.n);
  if (!P.mixed && P.dt == TK_F32) B.A64 = a.take<double>((size_t)P.m * P.n);
  if (!P.lowrank) {
    B.C = t.take<double>((size_t)P.c * P.c);
    B.R = (P.mixed ? t : a).take<double>((size_t)N * P.np * P.np);
    if (P.mixed) {
      B.Minv = a.take<float>((size_t)N * P.np * P.np);
      B.Mtinv = a.take<float>((size_t)N * P.np * P.np);
    }
    if (P.inv64) {
      B.Minv64 = a.take<double>((size_t)N * P.np * P.np);
      B.Mtinv64 = a.take<double>((size_t)N * P.np * P.np);
    }
  } else {
    B.sig = ty.take<double>((size_t)P.s);
    B.lrV = (P.mixed ? ty : a).take<double>((size_t)P.c * P.s);
    B.lrS = (P.mixed ? ty : a).take<double>((size_t)N * P.s);
    B.ranks = ty.take<int64_t>(N);
    B.sd = ty.take<double>(N);
    B.svd_bytes = svd_workspace(P.s, P.c);
    B.svd = ty.take<char>(B.svd_bytes);
    if (P.mixed) {
      B.lrV32 = a.take<float>((size_t)P.c * P.s);
      B.lrS32 = a.take<float>((size_t)N * P.s);
    }
  }
  if (P.mixed && P.o.emulate_fp64) B.oz_err = a.take<int>(4);
  if (P.mixed && !P.prep_only && P.o.emulate_fp64) {
    B.Aoz = a.take<char>(oz_slices_bytes(P.m, P.n));
    B.EA = a.take<int>(P.m);
    B.Xoz = a.take<char>(oz_slices_bytes(N, P.n));
    B.EX = a.take<int>(N);
    B.AozC = a.take<char>(oz_slices_bytes(P.n, P.m));  // A^T, column exponents
    B.EC = a.take<int>(P.n);
    B.colmax = a.take<char>(oz_colmax_bytes(P.n));
    B.Roz = a.take<char>(oz_slices_bytes(N, P.m));
    B.ER = a.take<int>(N);
  }
  if (!P.mixed && P.o.x0 && !P.prep_only) {  // warm start: [b - A x0; -sqrt(l) x0] per lambda
    B.Xa = a.take<double>((size_t)N * P.n);
    B.G = a.take<double>((size_t)N * P.n);
    B.Rres = a.take<double>((size_t)N * P.m);
  }
  if (P.mixed && !P.prep_only) {
    B.splits = splitk_count(N, P.n, P.m);
    // the emulated A^T r wants the most splits when the fewest lambdas remain
    if (P.o.emulate_fp64) B.splits = std::max(B.splits, oz_normal_splits(P.m, P.n, 1));
    B.D = a.take<double>((size_t)N * P.n);
    B.Xa = a.take<double>((size_t)N * P.n);
    B.G = a.take<double>((size_t)N * P.n);
    B.Rres = a.take<double>((size_t)N * P.m);
    B.part = a.take<double>((size_t)B.splits * N * P.n);
    B.nrm = a.take<double>((size_t)3 * N);
  }
  // the sketch's scratch is free again when the Gram matrix (or the BP2 factorization) is formed
  size_t sc = std::max(sketch_scratch(P), P.lowrank ? size_t(0) : gram_scratch_bytes(P.s, P.c));
  if (P.qr) sc = std::max(sc, bp2_workspace(P.s, P.c, N));
  if (emulated_gram(P)) sc = std::max({sc, oz_gram_workspace(P.s, P.c), oz_chol_workspace(P.np, N)});
  B.scratch_bytes = sc;
  B.scratch = t.take<char>(sc);
  if (P.prep_only) return;
  const int64_t lr_s = P.lowrank ? P.s : 0;
  if (P.mixed) {
    B.e32.m = P.m; B.e32.n = P.n; B.e32.N_cap = P.N_cap; B.e32.under = false; B.e32.lr_s = lr_s;
    B.e32.tc = P.lsqr_tc;
    B.e32.oz = P.lsqr_oz;
    B.e32.oz_fused = P.lsqr_fused;
    B.e32.carve(a);
  } else {
    B.e64.m = P.m; B.e64.n = P.n; B.e64.N_cap = P.N_cap; B.e64.under = P.under; B.e64.lr_s = lr_s;
    B.e64.carve(a);
  }
}

size_t plan_bytes(const Plan& P) {
  Arena a;
  Bufs B;
  carve(P, a, a, B);
  return a.used + 4096;
}
// the two parts of a prep_only plan: (kept for the LSQR phase, build scratch)
std::pair<size_t, size_t> plan_bytes_split(const Plan& P) {
  Arena a, t;
  Bufs B;
  carve(P, a, t, B);
  return {a.used + 4096, t.used + 4096};
}

// ------------------------------------------------------- small kernels ----
__global__ void k_fill(double* x, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}
__global__ void k_bcast(const double* __restrict__ b, int64_t m, double* __restrict__ out, int rows) {
  const int r = blockIdx.y;
  if (r >= rows) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    out[(int64_t)r * m + i] = b[i];
}
__global__ void k_gather_x(const double* __restrict__ X, int64_t n, const int* __restrict__ ids, double* __restrict__ Xa) {
  const int k = blockIdx.y;
  const int l = ids[k];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    Xa[(int64_t)k * n + j] = X[(int64_t)l * n + j];
}
// g_k = sum_z partial - lambda_l x_l  (float64 normal-equation residual
// A^T (b - A x) - lambda x of the k-th listed lambda); nrm[3k] = ||g_k||
__global__ void k_ne_finish(const double* __restrict__ part, int splits, int count, int64_t n,
                            const int* __restrict__ ids, const double* __restrict__ lam, const double* __restrict__ Xa,
                            double* __restrict__ G, double* __restrict__ nrm) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  const double lv = lam[ids[k]];
  const int64_t plane = (int64_t)count * n;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    double g = 0.0;
    for (int z = 0; z < splits; ++z) g += part[z * plane + (int64_t)k * n + j];
    g = fma(-lv, Xa[(int64_t)k * n + j], g);
    G[(int64_t)k * n + j] = g;
    acc = fma(g, g, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) nrm[3 * k] = sqrt(acc);
}
// X_l += D_l ; nrm[3k+1] = ||D_l||, nrm[3k+2] = ||X_l|| (after the update)
__global__ void k_refine_update(double* __restrict__ X, const double* __restrict__ D, int64_t n,
                                const int* __restrict__ ids, double* __restrict__ nrm) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  const int l = ids[k];
  double dd = 0.0, xx = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    double d = D[(int64_t)l * n + j];
    double x = X[(int64_t)l * n + j] + d;
    X[(int64_t)l * n + j] = x;
    dd = fma(d, d, dd);
    xx = fma(x, x, xx);
  }
  dd = block_sum(dd, sh);
  xx = block_sum(xx, sh);
  if (threadIdx.x == 0) {
    nrm[3 * k + 1] = sqrt(dd);
    nrm[3 * k + 2] = sqrt(xx);
  }
}
// G_k = -lambda_l x0_l for the k-th listed lambda l (the lower block of the
// warm start's right-hand side, scaled as Lsqr::run expects: bbot / sqrt(l))
__global__ void k_neg_lam_rows(const double* __restrict__ Xa, int64_t n, const int* __restrict__ ids,
                               const double* __restrict__ lam, double* __restrict__ G) {
  const int k = blockIdx.y;
  const double lv = lam[ids[k]];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    G[(int64_t)k * n + j] = -lv * Xa[(int64_t)k * n + j];
}
__global__ void k_f64_to_f32_flat(const double* __restrict__ s, float* __restrict__ d, int64_t total) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (float)s[i];
}
__global__ void k_widen(const float* __restrict__ s, int64_t rows, int64_t cols, int64_t lds, double* __restrict__ d) {
  const int64_t total = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / cols, c = i - r * cols;
    d[i] = (double)s[r * lds + c];
  }
}
inline int gsz(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), 152 * 32)); }
inline dim3 rgrid(int64_t len, int rows) {
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(len, 256), 64)), (unsigned)rows);
}

// ----------------------------------------------------------- sketch -------
// Y (s x c): the sketch along the long axis (A for m >= n, A^T for m < n).
tk_status do_sketch(const Plan& P, const void* A_sk, tk_dtype dt_sk, int64_t ld_sk, Bufs& B, cudaStream_t st) {
  const void* src = A_sk;
  int64_t ld = ld_sk;
  if (P.under) {
    TK_TRY(transpose(A_sk, dt_sk, P.m, P.n, ld_sk, B.AT, st));
    src = B.AT;
    ld = P.m;
  }
  Arena sa;
  sa.base = B.scratch;
  sa.cap = B.scratch_bytes;
  if (tc_sketch(P)) return tc_gauss_sketch(src, dt_sk, P.L, P.c, ld, P.o.seed, P.s, B.Y, sa, st);
  if (P.o.sketch == TK_SKETCH_SRHT) return srht_rows(src, dt_sk, P.L, P.c, ld, P.o.seed, P.s, B.Y, sa, st);
  if (P.o.sketch == TK_SKETCH_SPARSE) return sparse_rows(src, dt_sk, P.L, P.c, ld, P.o.seed, P.s, B.Y, sa, st);
  if (P.o.sketch == TK_SKETCH_SRDCT) return srdct_rows(src, dt_sk, P.L, P.c, ld, P.o.seed, P.s, B.Y, sa, st);
  return gauss_rows(src, dt_sk, P.L, P.c, ld, P.o.seed, P.s, B.Y, sa, st);
}

// ------------------------------------------------------ low rank ----------
// Algorithm 3 steps 5 and 7 after the SVD of the sketch: sd_i and the ranks
// s_i, the diagonals S_i, the float32 copies for the mixed form; every lambda
// has a preconditioner.
tk_status lowrank_finish(const LowRankParts& L, tk_info* inf, std::vector<int>& ok_ids, cudaStream_t st) {
  TK_TRY(lowrank_ranks_dev(L.sig, L.s, L.lam, L.N, L.alpha, L.sd, L.ranks, st));
  TK_TRY(lowrank_diag_dev<double>(L.sig, L.s, L.lam, L.ranks, L.N, L.lrS, st));
  std::vector<int64_t> hr(L.N);
  TK_CUDA(cudaMemcpyAsync(hr.data(), L.ranks, sizeof(int64_t) * L.N, cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  ok_ids.clear();
  for (int i = 0; i < L.N; ++i) {
    inf[i].rank = hr[i];
    ok_ids.push_back(i);
  }
  if (L.lrV32) {
    k_f64_to_f32_flat<<<gsz(L.c * L.s), 256, 0, st>>>(L.lrV, L.lrV32, L.c * L.s);
    k_f64_to_f32_flat<<<gsz((int64_t)L.N * L.s), 256, 0, st>>>(L.lrS, L.lrS32, (int64_t)L.N * L.s);
    TK_LAUNCH_CHECK();
  }
  return TK_OK;
}

// ------------------------------------------------------------ solve -------
// A sweep of several solves over one workspace (the L-curve's second sweep):
// the workspace is carved for N_plan lambdas whatever this solve's N, and with
// `reuse` the previous solve's float32 copy of A, sketch, Gram matrix (or SVD
// of the sketch) and digit planes of A are taken as they are.
struct SweepCtx {
  int N_plan = 0;
  bool reuse = false;
};

// With gp (grouped batch) only the preconditioner is built: `work` receives
// what the grouped LSQR reads, `scratch` the build-only buffers, and gp the
// pointers and the lambdas that have a preconditioner.
tk_status solve_impl(const tk_problem* p, const double* lambdas, int N, const tk_opts* o, void* work,
                     size_t work_bytes, cudaStream_t st, double* X, tk_info* info, GroupProblem* gp = nullptr,
                     void* scratch = nullptr, size_t scratch_bytes = 0, const SweepCtx* sw = nullptr) {
  Plan P;
  TK_TRY(make_plan(p, sw ? std::max(N, sw->N_plan) : N, o, P));
  const bool reuse = sw && sw->reuse;
  P.prep_only = gp != nullptr;
  if (N == 0) return TK_OK;
  if (!lambdas) return einval("lambdas pointer is NULL");
  for (int i = 0; i < N; ++i)
    if (!(lambdas[i] > 0.0) || !std::isfinite(lambdas[i])) return einval("every lambda must be a positive finite number");
  if (!p->A || !p->b || !X) return einval("A, b and X must be non-NULL");
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  Arena t;
  t.base = (char*)scratch;
  t.cap = scratch_bytes;
  Bufs B;
  if (!gp) {
    const size_t need = plan_bytes(P);
    if (!work || work_bytes < need) {
      set_error_msg("workspace smaller than tk_workspace_size()");
      return TK_ENOMEM;
    }
    carve(P, a, a, B);
  } else {
    carve(P, a, t, B);
  }
  if (!a.ok() || !t.ok()) {
    set_error_msg("workspace smaller than the solve needs");
    return TK_ENOMEM;
  }

  std::vector<tk_info> inf(N);
  for (auto& x : inf) {
    memset(&x, 0, sizeof(x));
    x.status = TK_OK;
  }
  TK_CUDA(cudaMemcpyAsync(B.lam, lambdas, sizeof(double) * N, cudaMemcpyHostToDevice, st));
  k_fill<<<1, 256, 0, st>>>(B.ones, N, 1.0);
  TK_LAUNCH_CHECK();

  // compute-precision copies of A
  const void* A_sk = p->A;
  tk_dtype dt_sk = P.dt;
  int64_t ld_sk = P.lda;
  const double* A64 = (P.dt == TK_F64) ? (const double*)p->A : nullptr;
  const float* A32 = (P.dt == TK_F32) ? (const float*)p->A : nullptr;
  int64_t lda64 = P.lda, lda32 = P.lda;
  if (P.mixed && P.dt == TK_F64) {
    if (!reuse) {
      const int tok = prof_begin(TK_PHASE_SLICE, st);  // a copy of A made once per solve, like the digit planes
      TK_TRY(convert_f64_to_f32((const double*)p->A, B.A32, P.m, P.n, P.lda, P.n, st));
      prof_end(tok, st, 0.0, 12.0 * P.m * P.n);
    }
    A32 = B.A32;
    lda32 = P.n;
  }
  if (!P.mixed && P.dt == TK_F32) {
    // the plain float64 path on float32 data: widen A once (exact)
    if (!reuse) k_widen<<<gsz(P.m * P.n), 256, 0, st>>>((const float*)p->A, P.m, P.n, P.lda, B.A64);
    TK_LAUNCH_CHECK();
    A64 = B.A64;
    lda64 = P.n;
    A_sk = B.A64;
    dt_sk = TK_F64;
    ld_sk = P.n;
  }
  if (P.mixed) {
    A_sk = A32;
    dt_sk = TK_F32;
    ld_sk = lda32;
  }

  // ---- step 1-2: draw X and sketch Y = XA (or A X)
  if (!reuse) {
    const double es = dt_sk == TK_F64 ? 8.0 : 4.0;
    const double Lp = (double)next_pow2(P.L);
    const double fl = P.o.sketch == TK_SKETCH_SRHT    ? Lp * std::log2(Lp) * P.c
                      : P.o.sketch == TK_SKETCH_SRDCT ? 5.0 * Lp * std::log2(Lp) * P.c
                      : P.o.sketch == TK_SKETCH_SPARSE ? (double)P.L * P.c
                                                       : 2.0 * P.s * P.L * P.c;
    int tok = prof_begin(TK_PHASE_SKETCH, st);
    TK_TRY(do_sketch(P, A_sk, dt_sk, ld_sk, B, st));
    prof_end(tok, st, fl, es * P.L * P.c + 8.0 * P.s * P.c);
  }

  // ---- steps 3-4 (Cholesky) or 4-7 (low rank)
  std::vector<int> ok_ids;
  if (!P.lowrank) {
    int tok = -1;
    if (emulated_gram(P)) TK_CUDA(cudaMemsetAsync(B.oz_err, 0, sizeof(int), st));
    if (!reuse && !P.qr) {
      tok = prof_begin(TK_PHASE_GRAM, st);
      if (emulated_gram(P)) {  // the Cholesky reads only j >= i
        TK_TRY(oz_gram(B.Y, P.s, P.c, B.C, B.scratch, B.scratch_bytes, B.oz_err, st));
      } else {
        TK_TRY(gram_upper(B.Y, P.s, P.c, B.C, B.scratch, B.scratch_bytes, st));
      }
      prof_end(tok, st, (double)P.s * P.c * (P.c + 1), 8.0 * (P.s * P.c + P.c * (P.c + 1) / 2));
    }
    Arena none;
    OzCholPlan ozp;  // the trailing updates on the tensor cores (the Gram scratch is free again)
    if (P.qr) {  // BP2 (Section 4.1): a QR of the (s + n) x n partly exact sketch per lambda
      tok = prof_begin(TK_PHASE_CHOLESKY, st);
      TK_TRY(bp2_factor(B.Y, P.s, P.c, B.lam, N, B.R, P.np, P.np, P.np * P.np, B.info, B.scratch, B.scratch_bytes,
                        st));
      const double M = (double)(P.s + P.c);
      prof_end(tok, st, (double)N * (2.0 * M * P.c * P.c - 2.0 * P.c * P.c * (double)P.c / 3.0),
               8.0 * N * (M * P.c + P.c * P.c / 2.0));
    } else if (emulated_gram(P)) {  // chol_shifted times its float64 and tensor-core parts itself
      TK_TRY(oz_chol_begin(B.R, P.np, P.np * P.np, N, P.np, B.scratch, B.scratch_bytes, B.oz_err, &ozp, st));
      TK_TRY(chol_shifted(B.C, P.c, B.lam, N, B.R, P.np, P.np * P.np, B.info, none, st, &ozp));
    } else {
      tok = prof_begin(TK_PHASE_CHOLESKY, st);
      TK_TRY(chol_shifted(B.C, P.c, B.lam, N, B.R, P.np, P.np * P.np, B.info, none, st));
      prof_end(tok, st, (double)N * P.c * P.c * P.c / 3.0, 8.0 * N * P.c * P.c);
    }
    std::vector<int> hinfo(N);
    TK_CUDA(cudaMemcpyAsync(hinfo.data(), B.info, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    int gerr = 0;
    if (emulated_gram(P)) TK_CUDA(cudaMemcpyAsync(&gerr, B.oz_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TK_CUDA(cudaStreamSynchronize(st));
    if (gerr) {
      set_error_msg("emulated float64 Gram matrix: a pipeline wait timed out");
      return TK_ETIMEOUT;
    }
    for (int i = 0; i < N; ++i) {
      if (hinfo[i] != 0) inf[i].status = hinfo[i] < 0 ? TK_ENUMERIC : TK_ENOTSPD;  // negative: NaN pivot
      else ok_ids.push_back(i);
    }
    if (P.mixed) {
      // the float32 LSQR applies R^-1 and R^-T as explicit float32 matrices
      tok = prof_begin(TK_PHASE_TRINV, st);
      TK_TRY(tri_inverse<float>(B.R, P.c, P.np, P.np * P.np, N, B.Minv, B.Mtinv, st));
      prof_end(tok, st, (double)N * P.c * P.c * P.c / 3.0, 4.0 * N * P.np * P.np * 3.0);
    }
    if (P.inv64) {
      tok = prof_begin(TK_PHASE_TRINV, st);
      TK_TRY(tri_inverse<double>(B.R, P.c, P.np, P.np * P.np, N, B.Minv64, B.Mtinv64, st));
      prof_end(tok, st, (double)N * P.c * P.c * P.c / 3.0, 8.0 * N * P.np * P.np * 3.0);
    }
  } else if (!gp) {
    Arena sa;
    sa.base = B.svd;
    sa.cap = B.svd_bytes;
    int sweeps = 0;
    if (!reuse) {  // sigma and V of the sketch are kept from the previous solve of the sweep
      int tok = prof_begin(TK_PHASE_SVD, st);
      TK_TRY(jacobi_svd(B.Y, P.s, P.c, B.sig, B.lrV, &sweeps, sa, st));
      prof_end(tok, st, 3.5 * sweeps * (double)P.s * P.s * P.c, 8.0 * P.s * P.c);
    }
    LowRankParts L{P.s, P.c, N, P.o.alpha, B.lam, B.sig, B.sd, B.ranks, B.lrV, B.lrS,
                   P.mixed ? B.lrV32 : nullptr, P.mixed ? B.lrS32 : nullptr};
    TK_TRY(lowrank_finish(L, inf.data(), ok_ids, st));
  }
  if (P.o.x0)  // warm start (problem (1.2) from x0): rows of lambdas without a preconditioner keep x0
    TK_CUDA(cudaMemcpyAsync(X, P.o.x0, sizeof(double) * (size_t)N * P.n, cudaMemcpyDeviceToDevice, st));
  else
    TK_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)N * P.n, st));
  if (gp) {
    gp->m = P.m;
    gp->n = P.n;
    gp->A32 = A32;
    gp->lda32 = lda32;
    gp->Af = p->A;
    gp->f64 = P.dt == TK_F64;
    gp->ldaf = P.lda;
    gp->b = p->b;
    gp->lam = B.lam;
    gp->X = X;
    gp->lowrank = P.lowrank;
    gp->Mi = B.Minv;
    gp->Mti = B.Mtinv;
    gp->np = P.np;
    gp->lrV = B.lrV32;
    gp->lrS = B.lrS32;
    gp->lr_s = P.lowrank ? P.s : 0;
    gp->inner_tol = P.o.inner_tol;
    gp->maxiter = P.o.maxiter;
    gp->max_refine = P.o.max_refine;
    gp->refine_tol = P.o.refine_tol;
    gp->emulate = P.o.emulate_fp64 ? 1 : 0;
    gp->ok_ids = ok_ids;
    if (P.lowrank) {  // the SVD and the ranks follow over all problems at once
      gp->lr_parts = LowRankParts{P.s, P.c, N, P.o.alpha, B.lam, B.sig, B.sd, B.ranks, B.lrV, B.lrS,
                                  B.lrV32, B.lrS32};
      gp->svd_Y = B.Y;
      gp->svd_scratch = B.svd;
      gp->svd_bytes = B.svd_bytes;
    }
    for (int i = 0; i < N; ++i) gp->inf[i] = inf[i];
    TK_CUDA(cudaStreamSynchronize(st));  // the build scratch is reused by the lane's next problem
    return TK_OK;
  }
  const int nok = (int)ok_ids.size();
  if (nok > 0) TK_CUDA(cudaMemcpyAsync(B.ids, ok_ids.data(), sizeof(int) * nok, cudaMemcpyHostToDevice, st));

  // ---- LSQR for every lambda (step 5-6 / 8-9)
  std::vector<LsqrResult> res;
  if (!P.mixed) {
    Lsqr<double>& e = B.e64;
    e.A = A64; e.lda = lda64; e.st = st; e.atol = e.btol = P.o.tol; e.maxiter = P.o.maxiter;
    e.a_es = P.dt == TK_F64 ? 8.0 : 4.0;
    if (!P.lowrank) {
      e.prec_kind = TK_PRECOND_CHOL; e.R = B.R; e.ldr = P.np; e.rstride = P.np * P.np;
      if (P.inv64) { e.Mi = B.Minv64; e.Mti = B.Mtinv64; e.ldm = P.np; e.mstride = P.np * P.np; }
    } else {
      e.prec_kind = TK_PRECOND_LOWRANK; e.lrV = B.lrV; e.lrS = B.lrS;
    }
    if (P.o.x0 && nok > 0) {
      // x = x0 + d with d = argmin ||B d - [b - A x0; -sqrt(l) x0]|| (B = [A; sqrt(l) I]): the same
      // minimiser of problem (1.2); LSQR adds d onto X, which holds x0
      k_gather_x<<<rgrid(P.n, nok), 256, 0, st>>>(X, P.n, B.ids, B.Xa);
      k_bcast<<<rgrid(P.m, nok), 256, 0, st>>>(p->b, P.m, B.Rres, nok);
      TK_LAUNCH_CHECK();
      TK_TRY((gemm<double, double, double>(false, true, nok, P.m, P.n, B.Xa, P.n, A64, lda64, B.Rres, P.m, -1.0,
                                           B.ones, B.Rres, P.m, st)));
      k_neg_lam_rows<<<rgrid(P.n, nok), 256, 0, st>>>(B.Xa, P.n, B.ids, B.lam, B.G);
      TK_LAUNCH_CHECK();
      if (P.o.schedule == TK_SCHED_BATCHED) {
        TK_TRY(e.run(B.Rres, P.m, B.G, P.n, B.ids, B.lam, nok, X, P.n, true, res));
      } else {
        for (int k = 0; k < nok; ++k)
          TK_TRY(e.run(B.Rres + (int64_t)k * P.m, 0, B.G + (int64_t)k * P.n, 0, B.ids + k, B.lam, 1, X, P.n, true,
                       res));
      }
    } else if (P.o.schedule == TK_SCHED_BATCHED) {
      TK_TRY(e.run(p->b, 0, nullptr, 0, B.ids, B.lam, nok, X, P.n, false, res));
    } else {
      for (int k = 0; k < nok; ++k) TK_TRY(e.run(p->b, 0, nullptr, 0, B.ids + k, B.lam, 1, X, P.n, false, res));
    }
    for (const auto& r : res) {
      tk_info& q = inf[r.lam_idx];
      q.iters += r.iters;
      q.istop = r.istop;
      q.rnorm = r.rnorm;
      q.arnorm = r.arnorm;
      if (r.istop == 7) q.status = worse(q.status, TK_ENOCONV);
      if (r.istop == 5) q.status = worse(q.status, TK_ENUMERIC);
    }
  } else {
    // ---- mixed: FP32 LSQR on corrections; the float64 pass forms r = b - A x
    //      and g = A^T r - lambda x (the normal-equation check), and the
    //      correction d solves min ||B d - [0; g/sqrt(l)]||, x <- x + d.
    Lsqr<float>& e = B.e32;
    e.A = A32; e.lda = lda32; e.st = st; e.atol = e.btol = P.o.inner_tol; e.maxiter = P.o.maxiter;
    e.a_es = P.dt == TK_F64 ? 8.0 : 4.0;
    if (P.lsqr_tc && ((uintptr_t)A32 % 16) == 0) {
      TK_TRY(transpose(A32, TK_F32, P.m, P.n, lda32, B.AT32, st));  // float32 A^T for the A^T U product
      e.AT = B.AT32;
    } else {
      e.tc = false;  // unaligned base address: SIMT float32 products
    }
    if (!P.lowrank) {
      e.prec_kind = TK_PRECOND_CHOL; e.Mi = B.Minv; e.Mti = B.Mtinv; e.ldm = P.np; e.mstride = P.np * P.np;
    } else {
      e.prec_kind = TK_PRECOND_LOWRANK; e.lrV = B.lrV32; e.lrS = B.lrS32;
    }
    std::vector<int> act = ok_ids;
    std::vector<double> hn(3 * std::max(N, 1));
    std::vector<double> prev_dn(std::max(N, 1), INFINITY);
    if (P.o.emulate_fp64 && !act.empty()) {  // A is split once (by rows and by columns); x, r on every pass
      if (!reuse) {
        const int tok = prof_begin(TK_PHASE_SLICE, st);
        TK_TRY(oz_prepare(p->A, P.dt, P.m, P.n, P.lda, B.Aoz, B.EA, st));
        TK_TRY(oz_prepare_cols(p->A, P.dt, P.m, P.n, P.lda, B.AozC, B.EC, B.colmax, st));
        prof_end(tok, st, 0.0, 2.0 * ((P.dt == TK_F64 ? 16.0 : 8.0) * P.m * P.n + 16.0 * P.m * P.n));
      }
      TK_CUDA(cudaMemsetAsync(B.oz_err, 0, sizeof(int), st));
      if (P.lsqr_oz) {  // the LSQR products read the first 4 digits of the same slices
        e.oz_A = B.Aoz; e.oz_EA = B.EA; e.oz_AT = B.AozC; e.oz_EAT = B.EC; e.oz_err = B.oz_err;
      }
    }
    for (int round = 0; round < P.o.max_refine && !act.empty(); ++round) {
      const int cnt = (int)act.size();
      TK_CUDA(cudaMemcpyAsync(B.ids, act.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, st));
      res.clear();
      if (round == 0 && !P.o.x0) {  // from x = 0 the first correction is the solution of [b; 0]
        if (P.o.schedule == TK_SCHED_BATCHED) TK_TRY(e.run(p->b, 0, nullptr, 0, B.ids, B.lam, cnt, B.D, P.n, false, res));
        else
          for (int k = 0; k < cnt; ++k) TK_TRY(e.run(p->b, 0, nullptr, 0, B.ids + k, B.lam, 1, B.D, P.n, false, res));
      } else {
        // FP64 pass: Rres = b - Xa A^T, G = Rres A - lambda Xa
        k_gather_x<<<rgrid(P.n, cnt), 256, 0, st>>>(X, P.n, B.ids, B.Xa);
        if (!P.o.emulate_fp64) k_bcast<<<rgrid(P.m, cnt), 256, 0, st>>>(p->b, P.m, B.Rres, cnt);
        TK_LAUNCH_CHECK();
        const double ea = P.dt == TK_F64 ? 8.0 : 4.0;
        const double fl = 2.0 * cnt * P.m * P.n;
        int tok = prof_begin(TK_PHASE_RES64, st);
        if (P.o.emulate_fp64) {
          TK_TRY(oz_prepare(B.Xa, TK_F64, cnt, P.n, P.n, B.Xoz, B.EX, st));
          TK_TRY(oz_residual(B.Aoz, B.EA, P.m, P.n, B.Xoz, B.EX, cnt, p->b, B.Rres, P.m, B.oz_err, st));
        } else if (P.dt == TK_F64) {
          TK_TRY((gemm<double, double, double>(false, true, cnt, P.m, P.n, B.Xa, P.n, A64, lda64, B.Rres, P.m, -1.0,
                                               B.ones, B.Rres, P.m, st)));
        } else {
          TK_TRY((gemm<double, float, double>(false, true, cnt, P.m, P.n, B.Xa, P.n, A32, lda32, B.Rres, P.m, -1.0,
                                              B.ones, B.Rres, P.m, st)));
        }
        prof_end(tok, st, fl, ea * P.m * P.n + 8.0 * (2.0 * cnt * P.m + cnt * P.n),
                 (P.o.emulate_fp64 ? 16.0 : ea) * P.m * P.n + 8.0 * (2.0 * cnt * P.m + cnt * P.n));
        tok = prof_begin(TK_PHASE_NE64, st);
        int sp;
        if (P.o.emulate_fp64) {
          sp = std::min(B.splits, oz_normal_splits(P.m, P.n, cnt));
          TK_TRY(oz_normal(B.AozC, B.EC, P.m, P.n, B.Rres, P.m, cnt, B.Roz, B.ER, B.part, sp, B.oz_err, st));
        } else {
          sp = P.dt == TK_F64 ? splitk_tuned<double, double>(cnt, P.n, P.m, B.splits)
                              : splitk_tuned<double, float>(cnt, P.n, P.m, B.splits);
          if (P.dt == TK_F64)
            TK_TRY((gemm_splitk<double, double>(false, false, cnt, P.n, P.m, B.Rres, P.m, A64, lda64, B.part, sp, st)));
          else
            TK_TRY((gemm_splitk<double, float>(false, false, cnt, P.n, P.m, B.Rres, P.m, A32, lda32, B.part, sp, st)));
        }
        prof_end(tok, st, fl, ea * P.m * P.n + 8.0 * (cnt * P.m + (double)sp * cnt * P.n),
                 (P.o.emulate_fp64 ? 16.0 : ea) * P.m * P.n + 8.0 * (cnt * P.m + (double)sp * cnt * P.n));
        k_ne_finish<<<cnt, 256, 0, st>>>(B.part, sp, cnt, P.n, B.ids, B.lam, B.Xa, B.G, B.nrm);
        TK_LAUNCH_CHECK();
        // correction: min ||B d - [0; g/sqrt(l)]||, whose normal equations are
        // (A^T A + l I) d = g; the right-hand side shrinks with the error of x.
        if (P.o.schedule == TK_SCHED_BATCHED) {
          TK_TRY(e.run(nullptr, 0, B.G, P.n, B.ids, B.lam, cnt, B.D, P.n, false, res));
        } else {
          for (int k = 0; k < cnt; ++k)
            TK_TRY(e.run(nullptr, 0, B.G + (int64_t)k * P.n, P.n, B.ids + k, B.lam, 1, B.D, P.n, false, res));
        }
      }
      k_refine_update<<<cnt, 256, 0, st>>>(X, B.D, P.n, B.ids, B.nrm);
      TK_LAUNCH_CHECK();
      TK_CUDA(cudaMemcpyAsync(hn.data(), B.nrm, sizeof(double) * 3 * cnt, cudaMemcpyDeviceToHost, st));
      int oz_err = 0;
      if (P.o.emulate_fp64 && (round > 0 || P.o.x0 || P.lsqr_oz))
        TK_CUDA(cudaMemcpyAsync(&oz_err, B.oz_err, sizeof(int), cudaMemcpyDeviceToHost, st));
      TK_CUDA(cudaStreamSynchronize(st));
      if (oz_err) {
        set_error_msg("emulated float64 product: a pipeline wait timed out");
        return TK_ETIMEOUT;
      }
      for (const auto& r : res) {
        tk_info& q = inf[r.lam_idx];
        q.iters += r.iters;
        q.istop = r.istop;
        q.rnorm = r.rnorm;
        q.arnorm = r.arnorm;
        if (r.istop == 5) q.status = worse(q.status, TK_ENUMERIC);
      }
      std::vector<int> next;
      for (int k = 0; k < cnt; ++k) {
        tk_info& q = inf[act[k]];
        q.refine_steps += 1;
        const bool checked = round > 0 || P.o.x0;  // this round formed g = A^T (b - A x) - l x
        if (checked) q.ne_norm = hn[3 * k];
        const double dn = hn[3 * k + 1], xn = hn[3 * k + 2];
        if (!std::isfinite(dn) || !std::isfinite(xn) || (checked && !std::isfinite(hn[3 * k])))
          q.status = worse(q.status, TK_ENUMERIC);  // refine_done stops on it; the status says why
        const bool done = refine_done(round, dn, prev_dn[act[k]], xn, P.o.refine_tol);
        prev_dn[act[k]] = dn;
        if (!done) next.push_back(act[k]);
      }
      act.swap(next);
    }
    for (int l : act) inf[l].status = worse(inf[l].status, TK_ENOCONV);
  }
  tk_status worst = TK_OK;
  for (int i = 0; i < N; ++i) worst = worse(worst, inf[i].status);
  if (info)
    for (int i = 0; i < N; ++i) info[i] = inf[i];
  TK_CUDA(cudaStreamSynchronize(st));
  return worst;
}

// ------------------------------------------------------------ L-curve -----
// Section 4.3: the points (||A x_i - b||, ||x_i||) of every lambda_i on a
// log-log plot, the regularization parameter of choice at the corner.  The
// corner is the point of largest curvature of P(t) = ln ||A x - b||,
// Q(t) = ln ||x|| in t = ln lambda (Hansen's reading; the paper does not say
// how the corner is found), with three-point differences on the sampled grid.

// rn[k] = ||R_k|| (row k of R, length m), xn[k] = ||X_k|| (length n); one block per row.
__global__ void k_lc_norms(const double* __restrict__ R, int64_t m, const double* __restrict__ X, int64_t n,
                           double* __restrict__ rn, double* __restrict__ xn) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  double rr = 0.0, xx = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    const double v = R[(int64_t)k * m + i];
    rr = fma(v, v, rr);
  }
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = X[(int64_t)k * n + j];
    xx = fma(v, v, xx);
  }
  rr = block_sum(rr, sh);
  xx = block_sum(xx, sh);
  if (threadIdx.x == 0) {
    rn[k] = sqrt(rr);
    xn[k] = sqrt(xx);
  }
}

// Curvature on the ascending grid lam[0..N): kappa[0] = kappa[N-1] = 0; the
// corner is the first largest interior kappa (*corner = -1 if N < 3).  With
// nr > 0, also the second sweep: nr parameters log-spaced strictly between the
// corner's neighbours.  One thread: N is a few dozen.
__global__ void k_lc_curvature(const double* __restrict__ lam, const double* __restrict__ rn,
                               const double* __restrict__ xn, int N, double* __restrict__ kappa,
                               int* __restrict__ corner, int nr, double* __restrict__ next) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < N; ++i) kappa[i] = 0.0;
  if (N < 3) {
    *corner = -1;
    return;
  }
  int best = 1;
  for (int k = 1; k < N - 1; ++k) {
    const double t0 = log(lam[k - 1]), t1 = log(lam[k]), t2 = log(lam[k + 1]);
    const double h1 = t1 - t0, h2 = t2 - t1;
    const double p0 = log(rn[k - 1]), p1 = log(rn[k]), p2 = log(rn[k + 1]);
    const double q0 = log(xn[k - 1]), q1 = log(xn[k]), q2 = log(xn[k + 1]);
    // derivatives of the quadratic through the three samples, at the middle one
    const double w0 = -h2 / (h1 * (h1 + h2)), w1 = (h2 - h1) / (h1 * h2), w2 = h1 / (h2 * (h1 + h2));
    const double v0 = 2.0 / (h1 * (h1 + h2)), v1 = -2.0 / (h1 * h2), v2 = 2.0 / (h2 * (h1 + h2));
    const double dp = __dmul_rn(w0, p0) + __dmul_rn(w1, p1) + __dmul_rn(w2, p2);
    const double dq = __dmul_rn(w0, q0) + __dmul_rn(w1, q1) + __dmul_rn(w2, q2);
    const double ddp = __dmul_rn(v0, p0) + __dmul_rn(v1, p1) + __dmul_rn(v2, p2);
    const double ddq = __dmul_rn(v0, q0) + __dmul_rn(v1, q1) + __dmul_rn(v2, q2);
    const double den = pow(__dmul_rn(dp, dp) + __dmul_rn(dq, dq), 1.5);
    kappa[k] = den > 0.0 ? (__dmul_rn(dp, ddq) - __dmul_rn(ddp, dq)) / den : 0.0;
    if (kappa[k] > kappa[best]) best = k;
  }
  *corner = best;
  if (nr > 0) {
    const double a = log(lam[best - 1]), b = log(lam[best + 1]);
    for (int j = 1; j <= nr; ++j) next[j - 1] = exp(a + (b - a) * (double)j / (double)(nr + 1));
  }
}

// out[k] = in[perm[k]] for k < N (doubles), and the rows of X likewise (length n)
__global__ void k_lc_permute(const int* __restrict__ perm, int N, const double* __restrict__ in,
                             double* __restrict__ out) {
  for (int k = threadIdx.x; k < N; k += blockDim.x) out[k] = in[perm[k]];
}

struct LcBufs {
  double* R = nullptr;     // N_plan x m residuals
  double* Xs = nullptr;    // N_plan x n: rows in sweep order, then permuted
  double* lam = nullptr;   // N_plan (sweep order)
  double* rn = nullptr;
  double* xn = nullptr;
  double* lam_m = nullptr;  // merged, ascending
  double* rn_m = nullptr;
  double* xn_m = nullptr;
  double* kappa = nullptr;
  double* next = nullptr;   // the second sweep's parameters
  int* perm = nullptr;
  int* corner = nullptr;
};
void lc_carve(Arena& a, int64_t m, int64_t n, int Np, LcBufs& L) {
  L.R = a.take<double>((size_t)Np * m);
  L.Xs = a.take<double>((size_t)Np * n);
  L.lam = a.take<double>(Np);
  L.rn = a.take<double>(Np);
  L.xn = a.take<double>(Np);
  L.lam_m = a.take<double>(Np);
  L.rn_m = a.take<double>(Np);
  L.xn_m = a.take<double>(Np);
  L.kappa = a.take<double>(Np);
  L.next = a.take<double>(Np);
  L.perm = a.take<int>(Np);
  L.corner = a.take<int>(4);
}

// rn, xn of the `cnt` solutions X (rows, length n) into rn[off..], xn[off..]:
// r = b - X A^T in float64 (on the tensor cores from the digit planes of A
// when the mixed form made them, else on the float64 pipe).
tk_status lc_norms(const tk_problem* p, const Plan& P, Bufs& B, const LcBufs& L, const double* Xrows, int cnt,
                   int off, cudaStream_t st) {
  if (cnt <= 0) return TK_OK;
  if (P.mixed && P.o.emulate_fp64) {
    TK_TRY(oz_prepare(Xrows, TK_F64, cnt, P.n, P.n, B.Xoz, B.EX, st));
    TK_TRY(oz_residual(B.Aoz, B.EA, P.m, P.n, B.Xoz, B.EX, cnt, p->b, L.R, P.m, B.oz_err, st));
  } else {
    k_bcast<<<rgrid(P.m, cnt), 256, 0, st>>>(p->b, P.m, L.R, cnt);
    k_fill<<<1, 256, 0, st>>>(B.ones, cnt, 1.0);
    TK_LAUNCH_CHECK();
    if (P.dt == TK_F64)
      TK_TRY((gemm<double, double, double>(false, true, cnt, P.m, P.n, Xrows, P.n, (const double*)p->A, P.lda, L.R,
                                           P.m, -1.0, B.ones, L.R, P.m, st)));
    else
      TK_TRY((gemm<double, float, double>(false, true, cnt, P.m, P.n, Xrows, P.n, (const float*)p->A, P.lda, L.R,
                                          P.m, -1.0, B.ones, L.R, P.m, st)));
  }
  k_lc_norms<<<cnt, 256, 0, st>>>(L.R, P.m, Xrows, P.n, L.rn + off, L.xn + off);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

}  // namespace
}  // namespace tk

using namespace tk;

extern "C" {

TK_API tk_status tk_opts_default(tk_opts* o) {
  if (!o) return TK_EINVAL;
  memset(o, 0, sizeof(*o));
  o->sketch = TK_SKETCH_SRHT;
  o->s = 0;
  o->precond = TK_PRECOND_CHOL;
  o->alpha = 2.0;
  o->precision = TK_PREC_FP64;
  o->tol = 1e-14;
  o->maxiter = 500;
  o->max_refine = 8;
  o->inner_tol = 1e-7;
  o->refine_tol = 1e-11;
  o->seed = 1;
  o->schedule = TK_SCHED_BATCHED;
  o->lsqr_tc = 2;
  o->group = 1;
  o->emulate_fp64 = 1;
  return TK_OK;
}

TK_API const char* tk_status_str(tk_status s) {
  switch (s) {
    case TK_OK: return "ok";
    case TK_EINVAL: return "invalid argument";
    case TK_ENOMEM: return "workspace too small";
    case TK_ENOTSPD: return "Cholesky breakdown (C + lambda I not positive definite)";
    case TK_ENOCONV: return "no convergence within the iteration cap";
    case TK_ENUMERIC: return "NaN or Inf in the recurrences";
    case TK_ETIMEOUT: return "device-side wait timed out";
    case TK_ECUDA: return "CUDA error";
  }
  return "unknown status";
}

TK_API const char* tk_last_error(void) { return tk::g_err; }

TK_API tk_status tk_workspace_size(const tk_problem* p, int N, const tk_opts* o, size_t* bytes) {
  if (!bytes) return einval("bytes pointer is NULL");
  Plan P;
  TK_TRY(make_plan(p, N, o, P));
  *bytes = plan_bytes(P);
  return TK_OK;
}

TK_API tk_status tk_solve(const tk_problem* p, const double* lambdas, int N, const tk_opts* o, void* work,
                          size_t work_bytes, void* stream, double* X, tk_info* info) {
  return solve_impl(p, lambdas, N, o, work, work_bytes, (cudaStream_t)stream, X, info);
}

// ---- many problems -------------------------------------------------------
// Two schedules.  Grouped (every problem mixed, overdetermined, batched,
// n <= 4096, N <= 64, SIMT products, opts.group = 1): each problem's sketch
// and preconditioner are built on host lanes (below), then ONE grouped LSQR
// and refinement advances all problems together (tk_group.cu).  Otherwise
// the problems are spread over up to kLanes host threads; each lane owns a
// stream (joined to the caller's stream by events) and a slice of the
// workspace, and solves its problems one after another.
static constexpr int kLanes = 8;

static int batched_lanes(int P) { return std::max(1, std::min(P, kLanes)); }

static const tk_opts* opts_of(const tk_opts* o, int n_opts, int i) { return n_opts == 1 ? o : o + i; }

namespace {
struct BatchLayout {
  bool grouped = false;
  int lanes = 1;
  size_t per = 0;                // lanes: slice per lane
  std::vector<size_t> keep_off;  // grouped: what problem i keeps for the LSQR phase
  std::vector<size_t> keep_len;
  size_t scratch_off = 0, scratch_per = 0;  // grouped: build scratch per lane
  size_t group_off = 0, group_len = 0;
  size_t svd_off = 0, svd_len = 0;  // grouped SVD of the low-rank problems
  size_t total = 0;
};

tk_status batch_layout(const tk_problem* ps, int P, int N, const tk_opts* o, int n_opts, BatchLayout& L) {
  L = BatchLayout{};
  L.lanes = batched_lanes(P);
  if (n_opts == 1 && P > 1 && o->x0) return einval("a warm start x0 belongs to one problem: pass one tk_opts per problem");
  std::vector<Plan> pl(P);
  bool grouped = P >= 2 && N >= 1 && N <= kGroupMaxLambda && (int64_t)P * N <= 65535;  // slot lists index grid.y
  for (int i = 0; i < P; ++i) {
    TK_TRY(make_plan(&ps[i], N, opts_of(o, n_opts, i), pl[i]));
    const Plan& q = pl[i];
    grouped = grouped && q.mixed && !q.under && q.o.schedule == TK_SCHED_BATCHED && !q.lsqr_tc &&
              q.n <= kGroupMaxN && q.o.group != 0 && !q.o.x0;  // warm starts run on the lanes
  }
  L.grouped = grouped;
  if (!grouped) {
    for (int i = 0; i < P; ++i) L.per = std::max(L.per, (plan_bytes(pl[i]) + 255) & ~size_t(255));
    L.total = L.per * (size_t)L.lanes;
    return TK_OK;
  }
  size_t off = 0;
  std::vector<GroupProblem> gp(P);
  L.keep_off.resize(P);
  L.keep_len.resize(P);
  for (int i = 0; i < P; ++i) {
    pl[i].prep_only = true;
    const auto kb = plan_bytes_split(pl[i]);
    L.keep_off[i] = off;
    L.keep_len[i] = (kb.first + 255) & ~size_t(255);
    off += L.keep_len[i];
    L.scratch_per = std::max(L.scratch_per, (kb.second + 255) & ~size_t(255));
    gp[i].m = pl[i].m;
    gp[i].n = pl[i].n;
    gp[i].emulate = pl[i].o.emulate_fp64 ? 1 : 0;  // the digit scratch of the float64 passes
  }
  L.scratch_off = off;
  off += L.scratch_per * (size_t)L.lanes;
  L.group_off = off;
  L.group_len = (group_workspace(gp, N) + 255) & ~size_t(255);
  off += L.group_len;
  std::vector<SvdJob> jobs;
  for (int i = 0; i < P; ++i)
    if (pl[i].lowrank) {
      SvdJob j;
      j.s = pl[i].s;
      j.n = pl[i].c;
      jobs.push_back(j);
    }
  L.svd_off = off;
  L.svd_len = (svd_grouped_workspace(jobs) + 255) & ~size_t(255);
  L.total = off + L.svd_len;
  return TK_OK;
}
}  // namespace

TK_API tk_status tk_workspace_size_batched(const tk_problem* ps, int P, int N, const tk_opts* o, int n_opts,
                                           size_t* bytes) {
  if (!bytes || P < 0 || (P > 0 && (!ps || !o)) || (n_opts != 1 && n_opts != P))
    return einval("bad batched arguments (n_opts must be 1 or P)");
  BatchLayout L;
  TK_TRY(batch_layout(ps, P, N, o, n_opts, L));
  *bytes = L.total;
  return TK_OK;
}

TK_API tk_status tk_solve_batched(const tk_problem* ps, int P, const double* lambdas, int N, const tk_opts* o,
                                  int n_opts, void* work, size_t work_bytes, void* stream, double* const* X,
                                  tk_info* info) {
  if (P < 0 || (P > 0 && (!ps || !lambdas || !X || !o)) || (n_opts != 1 && n_opts != P))
    return einval("bad batched arguments (n_opts must be 1 or P)");
  if (P == 0) return TK_OK;
  BatchLayout Ly;
  TK_TRY(batch_layout(ps, P, N, o, n_opts, Ly));
  const int lanes = Ly.lanes;
  if (!work || work_bytes < Ly.total) {
    set_error_msg("workspace smaller than tk_workspace_size_batched()");
    return TK_ENOMEM;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  int dev = 0;
  TK_CUDA(cudaGetDevice(&dev));
  cudaStream_t ls[kLanes];
  cudaEvent_t ev_in, ev_out[kLanes];
  TK_CUDA(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
  TK_CUDA(cudaEventRecord(ev_in, cs));
  for (int l = 0; l < lanes; ++l) {
    TK_CUDA(cudaStreamCreateWithFlags(&ls[l], cudaStreamNonBlocking));
    TK_CUDA(cudaEventCreateWithFlags(&ev_out[l], cudaEventDisableTiming));
    TK_CUDA(cudaStreamWaitEvent(ls[l], ev_in, 0));
  }
  std::vector<tk_info> own_info(info ? 0 : (size_t)P * N);
  tk_info* infos = info ? info : own_info.data();
  std::vector<GroupProblem> gps(Ly.grouped ? P : 0);
  for (int i = 0; i < (int)gps.size(); ++i) gps[i].inf = infos + (size_t)i * N;
  std::vector<tk_status> st(P, TK_OK);
  std::vector<std::string> err(lanes);
  auto lane_fn = [&](int l) {
    cudaSetDevice(dev);
    for (int i = l; i < P; i += lanes) {
      if (Ly.grouped) {
        st[i] = solve_impl(&ps[i], lambdas + (size_t)i * N, N, opts_of(o, n_opts, i), (char*)work + Ly.keep_off[i],
                           Ly.keep_len[i], ls[l], X[i], nullptr, &gps[i],
                           (char*)work + Ly.scratch_off + Ly.scratch_per * (size_t)l, Ly.scratch_per);
      } else {
        st[i] = solve_impl(&ps[i], lambdas + (size_t)i * N, N, opts_of(o, n_opts, i),
                           (char*)work + Ly.per * (size_t)l, Ly.per, ls[l], X[i], infos + (size_t)i * N);
      }
      if (st[i] == TK_EINVAL || st[i] == TK_ENOMEM || st[i] == TK_ECUDA) {
        err[l] = tk::g_err;
        break;
      }
    }
    cudaEventRecord(ev_out[l], ls[l]);
  };
  std::vector<std::thread> th;
  for (int l = 1; l < lanes; ++l) th.emplace_back(lane_fn, l);
  lane_fn(0);
  for (auto& t : th) t.join();
  tk_status worst = TK_OK;
  bool hard = false;
  for (int l = 0; l < lanes; ++l) {
    cudaStreamWaitEvent(cs, ev_out[l], 0);
    if (!err[l].empty()) set_error_msg(err[l].c_str());
  }
  for (int i = 0; i < P; ++i) {
    if (st[i] == TK_EINVAL || st[i] == TK_ENOMEM || st[i] == TK_ECUDA) {
      worst = st[i];
      hard = true;
    } else if (!hard) {
      worst = worse(worst, st[i]);
    }
  }
  if (Ly.grouped && !hard) {
    // the low-rank problems' SVDs together (one launch per Jacobi round), then
    // their ranks and diagonals
    std::vector<SvdJob> jobs;
    std::vector<int> jp;
    for (int i = 0; i < P; ++i)
      if (gps[i].lowrank) {
        SvdJob j;
        j.Y = gps[i].svd_Y;
        j.s = gps[i].lr_parts.s;
        j.n = gps[i].lr_parts.c;
        j.sigma = gps[i].lr_parts.sig;
        j.V = gps[i].lr_parts.lrV;
        j.scratch = gps[i].svd_scratch;
        j.scratch_bytes = gps[i].svd_bytes;
        jobs.push_back(j);
        jp.push_back(i);
      }
    tk_status g = TK_OK;
    if (!jobs.empty()) {
      const int tok = prof_begin(TK_PHASE_SVD, cs);
      g = jacobi_svd_grouped(jobs, (char*)work + Ly.svd_off, Ly.svd_len, cs);
      double fl = 0.0;
      for (const auto& j : jobs) fl += 3.5 * j.sweeps * (double)j.s * j.s * j.n;
      prof_end(tok, cs, fl, 0.0);
      for (size_t k = 0; k < jp.size() && g == TK_OK; ++k)
        g = lowrank_finish(gps[jp[k]].lr_parts, gps[jp[k]].inf, gps[jp[k]].ok_ids, cs);
    }
    // every problem's preconditioner is built: all of them iterate together
    if (g == TK_OK) g = group_solve_mixed(gps, N, (char*)work + Ly.group_off, Ly.group_len, cs);
    if (g != TK_OK) {
      worst = g;
    } else {
      for (size_t k = 0; k < (size_t)P * N; ++k) worst = worse(worst, infos[k].status);
    }
  }
  const cudaError_t sync = cudaStreamSynchronize(cs);
  for (int l = 0; l < lanes; ++l) {
    cudaStreamDestroy(ls[l]);
    cudaEventDestroy(ev_out[l]);
  }
  cudaEventDestroy(ev_in);
  if (sync != cudaSuccess) {
    tk::set_error(sync, __FILE__, __LINE__);
    return TK_ECUDA;
  }
  return worst;
}

TK_API tk_status tk_autotune(const tk_problem* p, int N, const tk_opts* o, void* work, size_t work_bytes,
                             void* stream) {
  Plan P;
  TK_TRY(make_plan(p, N, o, P));
  if (N == 0) return TK_OK;
  if (!p->A || !p->b) return einval("A and b must be non-NULL");
  if (!work || work_bytes < plan_bytes(P)) {
    set_error_msg("workspace smaller than tk_workspace_size()");
    return TK_ENOMEM;
  }
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  Bufs B;
  carve(P, a, a, B);
  cudaStream_t st = (cudaStream_t)stream;
  const int Nc = P.N_cap;
  // the lambda-row counts a solve meets as lambdas retire: 1, 2, 4, ... and N
  std::vector<int> Ms;
  for (int q = 1; q < Nc; q *= 2) Ms.push_back(q);
  Ms.push_back(Nc);
  if (!P.mixed) {
    if (P.under) return TK_OK;  // the underdetermined products keep the fixed rules
    const double* A64 = (P.dt == TK_F64) ? (const double*)p->A : B.A64;
    const int64_t lda = (P.dt == TK_F64) ? P.lda : P.n;
    Lsqr<double>& e = B.e64;
    for (int M : Ms) {
      // U = T A^T (+ coef U)  and the split-K  G = U A
      TK_TRY((tune_gemm<double, double, double>(false, true, M, P.m, P.n, e.Tt, P.n, A64, lda, e.Ut, P.m, 1.0,
                                                nullptr, nullptr, 0, 1, nullptr, st)));
      TK_TRY((tune_gemm<double, double, double>(false, false, M, P.n, P.m, e.Ut, P.m, A64, lda, nullptr, 0, 1.0,
                                                nullptr, nullptr, 0, e.splits, e.part_g, st)));
    }
  } else {
    k_fill<<<1, 256, 0, st>>>(B.ones, std::max(N, 1), 1.0);
    TK_LAUNCH_CHECK();
    const float* A32 = (P.dt == TK_F32) ? (const float*)p->A : B.A32;
    const int64_t lda32 = (P.dt == TK_F32) ? P.lda : P.n;
    Lsqr<float>& e = B.e32;
    for (int M : Ms) {
      // the float64 residual r = b - X A^T and the split-K A^T r
      if (P.dt == TK_F64) {
        TK_TRY((tune_gemm<double, double, double>(false, true, M, P.m, P.n, B.Xa, P.n, (const double*)p->A, P.lda,
                                                  B.Rres, P.m, -1.0, B.ones, B.Rres, P.m, 1, nullptr, st)));
        TK_TRY((tune_gemm<double, double, double>(false, false, M, P.n, P.m, B.Rres, P.m, (const double*)p->A, P.lda,
                                                  nullptr, 0, 1.0, nullptr, nullptr, 0, B.splits, B.part, st)));
      } else {
        TK_TRY((tune_gemm<double, float, double>(false, true, M, P.m, P.n, B.Xa, P.n, A32, lda32, B.Rres, P.m, -1.0,
                                                 B.ones, B.Rres, P.m, 1, nullptr, st)));
        TK_TRY((tune_gemm<double, float, double>(false, false, M, P.n, P.m, B.Rres, P.m, A32, lda32, nullptr, 0, 1.0,
                                                 nullptr, nullptr, 0, B.splits, B.part, st)));
      }
      // the split count of the float32 A^T U product
      if (!P.lsqr_tc)
        TK_TRY((tune_gemm<float, float, double>(false, false, M, P.n, P.m, e.Ut, P.m, A32, lda32, nullptr, 0, 1.0,
                                                nullptr, nullptr, 0, e.splits, e.part_g, st)));
    }
  }
  TK_CUDA(cudaStreamSynchronize(st));
  return TK_OK;
}

namespace tk {
struct ResidualBufs {
  void *Aoz, *Xoz, *AozC, *colmax, *Roz;
  int *EA, *EX, *EC, *ER, *err;
  double *ones, *part;
  int splits;
};
static void residual_carve(Arena& a, int64_t m, int64_t n, int M, ResidualBufs& w) {
  w.splits = oz_normal_splits(m, n, M);
  w.Aoz = a.take<char>(oz_slices_bytes(m, n));
  w.EA = a.take<int>(m);
  w.Xoz = a.take<char>(oz_slices_bytes(M, n));
  w.EX = a.take<int>(M);
  w.AozC = a.take<char>(oz_slices_bytes(n, m));
  w.EC = a.take<int>(n);
  w.colmax = a.take<char>(oz_colmax_bytes(n));
  w.Roz = a.take<char>(oz_slices_bytes(M, m));
  w.ER = a.take<int>(M);
  w.ones = a.take<double>(std::max(M, 1));
  w.part = a.take<double>((size_t)w.splits * M * n);
  w.err = a.take<int>(4);
}
__global__ void k_residual_sum_splits(const double* __restrict__ part, int splits, int64_t total,
                                      double* __restrict__ G) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < splits; ++z) acc += part[(int64_t)z * total + k];
    G[k] = acc;
  }
}
}  // namespace tk

TK_API size_t tk_residual_workspace(int64_t m, int64_t n, int M) {
  Arena a;
  ResidualBufs w;
  residual_carve(a, m, n, M, w);
  return a.used + 1024;
}

TK_API tk_status tk_residual(const tk_problem* p, const double* X, int M, int64_t ldx, int emulate, double* R,
                             double* G, void* work, size_t work_bytes, void* stream) {
  if (!p || !p->A || !p->b || (M > 0 && (!X || !R))) return einval("A, b, X and R must be non-NULL");
  if (p->m < 1 || p->n < 1 || p->lda < p->n || M < 0 || (M > 0 && ldx < p->n))
    return einval("bad shapes (m, n >= 1, lda >= n, ldx >= n)");
  if (p->dtype != TK_F64 && p->dtype != TK_F32) return einval("unknown dtype");
  if (emulate && p->n > (int64_t(1) << 27)) return einval("emulate: n above 2^27 (the exact int64 level sums)");
  if (M == 0) return TK_OK;
  if (!work || work_bytes < tk_residual_workspace(p->m, p->n, M)) {
    set_error_msg("workspace smaller than tk_residual_workspace()");
    return TK_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  ResidualBufs w;
  residual_carve(a, p->m, p->n, M, w);
  const int64_t m = p->m, n = p->n;
  int herr = 0;
  if (emulate) {
    TK_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    TK_TRY(oz_prepare(p->A, p->dtype, m, n, p->lda, w.Aoz, w.EA, st));
    TK_TRY(oz_prepare(X, TK_F64, M, n, ldx, w.Xoz, w.EX, st));
    TK_TRY(oz_residual(w.Aoz, w.EA, m, n, w.Xoz, w.EX, M, p->b, R, m, w.err, st));
    if (G) {
      TK_TRY(oz_prepare_cols(p->A, p->dtype, m, n, p->lda, w.AozC, w.EC, w.colmax, st));
      TK_TRY(oz_normal(w.AozC, w.EC, m, n, R, m, M, w.Roz, w.ER, w.part, w.splits, w.err, st));
      k_residual_sum_splits<<<(unsigned)std::min<int64_t>(cdiv((int64_t)M * n, 256), 152 * 8), 256, 0, st>>>(
          w.part, w.splits, (int64_t)M * n, G);
      TK_LAUNCH_CHECK();
    }
  } else {
    double* ones = w.ones;
    k_fill<<<1, 256, 0, st>>>(ones, M, 1.0);
    TK_LAUNCH_CHECK();
    // R = 1 * broadcast(b) - X A^T;  G = R A
    if (p->dtype == TK_F64) {
      TK_TRY((gemm<double, double, double>(false, true, M, m, n, X, ldx, (const double*)p->A, p->lda, R, m, -1.0,
                                           ones, p->b, 0, st)));
      if (G) TK_TRY((gemm<double, double, double>(false, false, M, n, m, R, m, (const double*)p->A, p->lda, G, n, 1.0,
                                                  nullptr, nullptr, 0, st)));
    } else {
      TK_TRY((gemm<double, float, double>(false, true, M, m, n, X, ldx, (const float*)p->A, p->lda, R, m, -1.0, ones,
                                          p->b, 0, st)));
      if (G) TK_TRY((gemm<double, float, double>(false, false, M, n, m, R, m, (const float*)p->A, p->lda, G, n, 1.0,
                                                 nullptr, nullptr, 0, st)));
    }
  }
  if (emulate) TK_CUDA(cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    set_error_msg("emulated float64 product: a pipeline wait timed out");
    return TK_ETIMEOUT;
  }
  return TK_OK;
}

TK_API size_t tk_autotune_entries(void) { return tune_size(); }
TK_API void tk_autotune_clear(void) { tune_clear(); }
TK_API size_t tk_autotune_describe(char* buf, size_t len) { return tune_describe(buf, len); }

TK_API size_t tk_sketch_draw_workspace(int64_t mp) { return draw_workspace(mp > 0 ? mp : 1) + 1024; }

TK_API tk_status tk_sketch_draw(uint64_t seed, int64_t mp, int64_t s, int8_t* signs, int64_t* rows, void* work,
                                size_t work_bytes, void* stream) {
  if (mp < 1 || mp > kMaxLong) return einval("mp out of range");
  if (s < 0 || s > mp) return einval("s out of range");
  if (rows && s > 0 && (!work || work_bytes < tk_sketch_draw_workspace(mp))) {
    set_error_msg("workspace smaller than tk_sketch_draw_workspace()");
    return TK_ENOMEM;
  }
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  cudaStream_t st = (cudaStream_t)stream;
  TK_TRY(draw_signs_rows(seed, mp, s, signs, rows, nullptr, a, st));
  TK_CUDA(cudaStreamSynchronize(st));
  return TK_OK;
}

TK_API size_t tk_sketch_draw_sparse_workspace(int64_t L, int64_t s) {
  if (L < 1 || s < 1) return 0;
  return sparse_rows_workspace(L, 1, s) + 1024;
}

TK_API tk_status tk_sketch_draw_sparse(uint64_t seed, int64_t L, int64_t s, int32_t* h, int8_t* sign, int32_t* order,
                                       int32_t* start, void* work, size_t work_bytes, void* stream) {
  if (L < 1 || L > INT32_MAX || s < 1 || s > kSparseMaxS) return einval("need 1 <= L < 2^31 and 1 <= s <= 2^22");
  if (!work || work_bytes < tk_sketch_draw_sparse_workspace(L, s)) {
    set_error_msg("workspace smaller than tk_sketch_draw_sparse_workspace()");
    return TK_ENOMEM;
  }
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  cudaStream_t st = (cudaStream_t)stream;
  TK_TRY(sparse_draw_sorted(seed, L, s, h, sign, order, start, a, st));
  TK_CUDA(cudaStreamSynchronize(st));
  return TK_OK;
}

TK_API tk_status tk_sketch_apply_workspace(const tk_problem* p, const tk_opts* o, size_t* bytes) {
  if (!bytes) return einval("bytes pointer is NULL");
  Plan P;
  TK_TRY(make_plan(p, 1, o, P));
  Arena a;
  if (P.under) {
    a.take<char>((size_t)P.m * P.n * (P.dt == TK_F64 ? 8 : 4));
    a.take<double>((size_t)P.s * P.c);
  }
  a.take<char>(sketch_scratch(P));
  *bytes = a.used + 4096;
  return TK_OK;
}

TK_API tk_status tk_sketch_apply(const tk_problem* p, const tk_opts* o, double* Y, void* work, size_t work_bytes,
                                 void* stream) {
  Plan P;
  TK_TRY(make_plan(p, 1, o, P));
  if (P.mixed && !tc_sketch(P)) return einval("tk_sketch_apply: MIXED selects the tensor-core Gaussian sketch only");
  if (!p->A || !Y) return einval("A and Y must be non-NULL");
  size_t need = 0;
  TK_TRY(tk_sketch_apply_workspace(p, o, &need));
  if (!work || work_bytes < need) {
    set_error_msg("workspace smaller than tk_sketch_apply_workspace()");
    return TK_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  Bufs B;
  if (P.under) {
    B.AT = a.take<char>((size_t)P.m * P.n * (P.dt == TK_F64 ? 8 : 4));
    B.Y = a.take<double>((size_t)P.s * P.c);
  } else {
    B.Y = Y;
  }
  B.scratch_bytes = sketch_scratch(P);
  B.scratch = a.take<char>(B.scratch_bytes);
  if (!a.ok()) return TK_ENOMEM;
  TK_TRY(do_sketch(P, p->A, P.dt, P.lda, B, st));
  if (P.under) TK_TRY(transpose(B.Y, TK_F64, P.s, P.m, P.m, Y, st));  // (s x m) -> (m x s)
  TK_CUDA(cudaStreamSynchronize(st));
  return TK_OK;
}

TK_API tk_status tk_gram(const double* Y, int64_t r, int64_t c, int transpose_first, double* C, void* stream) {
  if (!Y || !C || r < 1 || c < 1) return einval("bad Gram arguments");
  cudaStream_t st = (cudaStream_t)stream;
  if (transpose_first)
    TK_TRY((gemm<double, double, double>(true, false, c, c, r, Y, c, Y, c, C, c, 1.0, nullptr, nullptr, 0, st)));
  else
    TK_TRY((gemm<double, double, double>(false, true, r, r, c, Y, c, Y, c, C, r, 1.0, nullptr, nullptr, 0, st)));
  TK_CUDA(cudaStreamSynchronize(st));
  return TK_OK;
}

TK_API size_t tk_gram_emulated_workspace(int64_t r, int64_t c) {
  if (r < 1 || c < 1) return 0;
  Arena a;
  a.take<char>(oz_gram_workspace(r, c));
  a.take<int>(4);
  return a.used + 512;
}

TK_API tk_status tk_gram_emulated(const double* Y, int64_t r, int64_t c, double* C, void* work, size_t work_bytes,
                                  void* stream) {
  if (!Y || !C || r < 1 || c < 1) return einval("bad Gram arguments");
  if (!work || work_bytes < tk_gram_emulated_workspace(r, c)) {
    set_error_msg("workspace smaller than tk_gram_emulated_workspace()");
    return TK_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  const size_t gb = oz_gram_workspace(r, c);
  void* gw = a.take<char>(gb);
  int* err = a.take<int>(4);
  TK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  TK_TRY(oz_gram(Y, r, c, C, gw, gb, err, st));
  int herr = 0;
  TK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    set_error_msg("emulated float64 Gram matrix: a pipeline wait timed out");
    return TK_ETIMEOUT;
  }
  return TK_OK;
}

TK_API size_t tk_cholesky_workspace(int64_t n, int N) {
  if (n < 1 || N < 1) return 0;
  const int64_t np = cdiv(n, 64) * 64;
  Arena a;
  a.take<double>(N);
  a.take<int>(N);
  a.take<double>((size_t)N * np * np);
  return a.used + 1024;
}

TK_API size_t tk_cholesky_emulated_workspace(int64_t n, int N) {
  if (n < 1 || N < 1) return 0;
  const int64_t np = cdiv(n, 64) * 64;
  return tk_cholesky_workspace(n, N) + oz_chol_workspace(np, N) + 1024;
}

namespace {
tk_status cholesky_common(const double* C, int64_t n, const double* lambdas, int N, double* R, int* breakdown,
                          void* work, size_t work_bytes, void* stream, bool emulate) {
  if (!C || !R || !lambdas || n < 1 || n > kMaxShort || N < 1) return einval("bad Cholesky arguments");
  for (int i = 0; i < N; ++i)
    if (!std::isfinite(lambdas[i])) return einval("lambda must be finite");
  const size_t need = emulate ? tk_cholesky_emulated_workspace(n, N) : tk_cholesky_workspace(n, N);
  if (!work || work_bytes < need) {
    set_error_msg("workspace smaller than the Cholesky workspace query");
    return TK_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t np = cdiv(n, 64) * 64;
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  double* lam = a.take<double>(N);
  int* info = a.take<int>(N);
  double* Rp = a.take<double>((size_t)N * np * np);
  int* err = a.take<int>(4);
  TK_CUDA(cudaMemcpyAsync(lam, lambdas, sizeof(double) * N, cudaMemcpyHostToDevice, st));
  Arena none;
  OzCholPlan plan;
  if (emulate) {
    const size_t ob = oz_chol_workspace(np, N);
    void* ow = a.take<char>(ob);
    if (!a.ok()) return TK_ENOMEM;
    TK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    TK_TRY(oz_chol_begin(Rp, np, np * np, N, np, ow, ob, err, &plan, st));
  }
  TK_TRY(chol_shifted(C, n, lam, N, Rp, np, np * np, info, none, st, emulate ? &plan : nullptr));
  for (int i = 0; i < N; ++i)
    TK_CUDA(cudaMemcpy2DAsync(R + (size_t)i * n * n, sizeof(double) * n, Rp + (size_t)i * np * np,
                              sizeof(double) * np, sizeof(double) * n, n, cudaMemcpyDeviceToDevice, st));
  std::vector<int> h(N);
  int herr = 0;
  TK_CUDA(cudaMemcpyAsync(h.data(), info, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  if (emulate) TK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    set_error_msg("emulated Cholesky update: a pipeline wait timed out");
    return TK_ETIMEOUT;
  }
  tk_status worst = TK_OK;
  for (int i = 0; i < N; ++i) {
    if (breakdown) breakdown[i] = h[i];
    if (h[i]) worst = worse(worst, h[i] < 0 ? TK_ENUMERIC : TK_ENOTSPD);
  }
  return worst;
}
}  // namespace

TK_API tk_status tk_cholesky_shifted(const double* C, int64_t n, const double* lambdas, int N, double* R,
                                     int* breakdown, void* work, size_t work_bytes, void* stream) {
  return cholesky_common(C, n, lambdas, N, R, breakdown, work, work_bytes, stream, false);
}

TK_API tk_status tk_cholesky_shifted_emulated(const double* C, int64_t n, const double* lambdas, int N, double* R,
                                              int* breakdown, void* work, size_t work_bytes, void* stream) {
  return cholesky_common(C, n, lambdas, N, R, breakdown, work, work_bytes, stream, true);
}

TK_API size_t tk_bp2_factor_workspace(int64_t s, int64_t n, int N) {
  if (s < 0 || n < 1 || N < 1) return 0;
  const int64_t np = cdiv(n, 64) * 64;
  Arena a;
  a.take<double>(N);
  a.take<int>(N);
  a.take<double>((size_t)N * np * np);
  return a.used + bp2_workspace(s, n, N) + 1024;
}

TK_API tk_status tk_bp2_factor(const double* Y, int64_t s, int64_t n, const double* lambdas, int N, double* R,
                               int* breakdown, void* work, size_t work_bytes, void* stream) {
  if (!Y || !R || !lambdas || s < 0 || n < 1 || n > kMaxShort || N < 1) return einval("bad BP2 arguments");
  for (int i = 0; i < N; ++i)
    if (!(lambdas[i] > 0.0) || !std::isfinite(lambdas[i])) return einval("every lambda must be a positive finite number");
  if (!work || work_bytes < tk_bp2_factor_workspace(s, n, N)) {
    set_error_msg("workspace smaller than tk_bp2_factor_workspace()");
    return TK_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t np = cdiv(n, 64) * 64;
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  double* lam = a.take<double>(N);
  int* info = a.take<int>(N);
  double* Rp = a.take<double>((size_t)N * np * np);
  const size_t qb = bp2_workspace(s, n, N);
  void* qw = a.take<char>(qb);
  if (!a.ok()) return TK_ENOMEM;
  TK_CUDA(cudaMemcpyAsync(lam, lambdas, sizeof(double) * N, cudaMemcpyHostToDevice, st));
  TK_TRY(bp2_factor(Y, s, n, lam, N, Rp, np, np, np * np, info, qw, qb, st));
  for (int i = 0; i < N; ++i)
    TK_CUDA(cudaMemcpy2DAsync(R + (size_t)i * n * n, sizeof(double) * n, Rp + (size_t)i * np * np,
                              sizeof(double) * np, sizeof(double) * n, n, cudaMemcpyDeviceToDevice, st));
  std::vector<int> h(N);
  TK_CUDA(cudaMemcpyAsync(h.data(), info, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  tk_status worst = TK_OK;
  for (int i = 0; i < N; ++i) {
    if (breakdown) breakdown[i] = h[i];
    if (h[i]) worst = worse(worst, h[i] < 0 ? TK_ENUMERIC : TK_ENOTSPD);
  }
  return worst;
}

TK_API size_t tk_sketch_svd_workspace(int64_t s, int64_t n) { return svd_workspace(s, n) + 1024; }

TK_API tk_status tk_sketch_svd(const double* Y, int64_t s, int64_t n, double* sigma, double* V, int* sweeps,
                               void* work, size_t work_bytes, void* stream) {
  if (!Y || !sigma || !V || s < 1 || n < 1 || s > n) return einval("bad SVD arguments (need 1 <= s <= n)");
  if (!work || work_bytes < tk_sketch_svd_workspace(s, n)) {
    set_error_msg("workspace smaller than tk_sketch_svd_workspace()");
    return TK_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  int sw = 0;
  TK_TRY(jacobi_svd(Y, s, n, sigma, V, &sw, a, st));
  if (sweeps) *sweeps = sw;
  TK_CUDA(cudaStreamSynchronize(st));
  return TK_OK;
}

TK_API size_t tk_lowrank_ranks_workspace(int N) {
  Arena a;
  a.take<double>(N > 0 ? N : 1);
  a.take<double>(N > 0 ? N : 1);
  a.take<int64_t>(N > 0 ? N : 1);
  return a.used + 1024;
}

TK_API tk_status tk_lowrank_ranks(const double* sigma, int64_t s, const double* lambdas, int N, double alpha,
                                  double* sd, int64_t* ranks, void* work, size_t work_bytes, void* stream) {
  if (!sigma || !lambdas || !ranks || s < 1 || N < 1 || !(alpha >= 1.0)) return einval("bad rank arguments");
  if (!work || work_bytes < tk_lowrank_ranks_workspace(N)) {
    set_error_msg("workspace smaller than tk_lowrank_ranks_workspace()");
    return TK_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  double* lam = a.take<double>(N);
  double* sdd = a.take<double>(N);
  int64_t* rk = a.take<int64_t>(N);
  TK_CUDA(cudaMemcpyAsync(lam, lambdas, sizeof(double) * N, cudaMemcpyHostToDevice, st));
  TK_TRY(lowrank_ranks_dev(sigma, s, lam, N, alpha, sdd, rk, st));
  if (sd) TK_CUDA(cudaMemcpyAsync(sd, sdd, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaMemcpyAsync(ranks, rk, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  return TK_OK;
}

// ---- L-curve (Section 4.3) ----------------------------------------------------
namespace {
tk_status lcurve_plan(const tk_problem* p, int N, int N_refine, const tk_opts* o, Plan& P, size_t& plan_b,
                      size_t& total) {
  if (N < 3) return einval("tk_lcurve: at least 3 lambdas are needed for a curvature");
  if (N_refine < 0 || N + N_refine > 4096) return einval("tk_lcurve: N_refine must be >= 0 and N + N_refine <= 4096");
  if (o && o->x0) return einval("tk_lcurve: no warm start (x0) in an L-curve sweep");
  TK_TRY(make_plan(p, N + N_refine, o, P));
  plan_b = (plan_bytes(P) + 255) & ~size_t(255);
  Arena a;
  LcBufs L;
  lc_carve(a, P.m, P.n, N + N_refine, L);
  total = plan_b + a.used + 4096;
  return TK_OK;
}
}  // namespace

TK_API tk_status tk_lcurve_workspace_size(const tk_problem* p, int N, int N_refine, const tk_opts* o,
                                          size_t* bytes) {
  if (!bytes) return einval("bytes pointer is NULL");
  Plan P;
  size_t pb = 0, tot = 0;
  TK_TRY(lcurve_plan(p, N, N_refine, o, P, pb, tot));
  *bytes = tot;
  return TK_OK;
}

TK_API tk_status tk_lcurve(const tk_problem* p, const double* lambdas, int N, int N_refine, const tk_opts* o,
                           void* work, size_t work_bytes, void* stream, double* X, tk_lcurve_point* points,
                           int* corner) {
  Plan P;
  size_t plan_b = 0, total = 0;
  TK_TRY(lcurve_plan(p, N, N_refine, o, P, plan_b, total));
  if (!lambdas || !X || !points || !corner) return einval("tk_lcurve: lambdas, X, points and corner must be non-NULL");
  for (int i = 0; i < N; ++i)
    if (!(lambdas[i] > 0.0) || !std::isfinite(lambdas[i])) return einval("every lambda must be a positive finite number");
  if (!p->A || !p->b) return einval("A and b must be non-NULL");
  if (!work || work_bytes < total) {
    set_error_msg("workspace smaller than tk_lcurve_workspace_size()");
    return TK_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int Np = N + N_refine;
  // the solve's own buffers (the same carve solve_impl makes) and the L-curve's after them
  Arena a;
  a.base = (char*)work;
  a.cap = plan_b;
  Bufs B;
  carve(P, a, a, B);
  Arena la;
  la.base = (char*)work + plan_b;
  la.cap = work_bytes - plan_b;
  LcBufs L;
  lc_carve(la, P.m, P.n, Np, L);
  // first sweep: the given lambdas in ascending order
  std::vector<double> lam(lambdas, lambdas + N);
  std::sort(lam.begin(), lam.end());
  std::vector<tk_info> info(Np);
  SweepCtx sw;
  sw.N_plan = Np;
  tk_status s1 = solve_impl(p, lam.data(), N, o, work, plan_b, st, L.Xs, info.data(), nullptr, nullptr, 0, &sw);
  if (s1 == TK_EINVAL || s1 == TK_ENOMEM || s1 == TK_ECUDA || s1 == TK_ETIMEOUT) return s1;
  TK_CUDA(cudaMemcpyAsync(L.lam, lam.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
  TK_TRY(lc_norms(p, P, B, L, L.Xs, N, 0, st));
  k_lc_curvature<<<1, 32, 0, st>>>(L.lam, L.rn, L.xn, N, L.kappa, L.corner, N_refine, L.next);
  TK_LAUNCH_CHECK();
  std::vector<double> next(std::max(N_refine, 1));
  tk_status s2 = TK_OK;
  if (N_refine > 0) {
    // second sweep between the corner's neighbours, reusing the sketch, the Gram matrix (or the
    // SVD of the sketch) and the copies and digit planes of A
    TK_CUDA(cudaMemcpyAsync(next.data(), L.next, sizeof(double) * N_refine, cudaMemcpyDeviceToHost, st));
    TK_CUDA(cudaStreamSynchronize(st));
    sw.reuse = true;
    s2 = solve_impl(p, next.data(), N_refine, o, work, plan_b, st, L.Xs + (size_t)N * P.n, info.data() + N,
                    nullptr, nullptr, 0, &sw);
    if (s2 == TK_EINVAL || s2 == TK_ENOMEM || s2 == TK_ECUDA || s2 == TK_ETIMEOUT) return s2;
    TK_CUDA(cudaMemcpyAsync(L.lam + N, next.data(), sizeof(double) * N_refine, cudaMemcpyHostToDevice, st));
    TK_TRY(lc_norms(p, P, B, L, L.Xs + (size_t)N * P.n, N_refine, N, st));
  }
  // both sweeps merged in ascending lambda (two sorted lists), curvature and corner of the merged grid
  std::vector<double> all(lam);
  all.insert(all.end(), next.begin(), next.begin() + N_refine);
  std::vector<int> perm(Np);
  for (int i = 0; i < Np; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return all[x] < all[y]; });
  TK_CUDA(cudaMemcpyAsync(L.perm, perm.data(), sizeof(int) * Np, cudaMemcpyHostToDevice, st));
  k_lc_permute<<<1, 256, 0, st>>>(L.perm, Np, L.lam, L.lam_m);
  k_lc_permute<<<1, 256, 0, st>>>(L.perm, Np, L.rn, L.rn_m);
  k_lc_permute<<<1, 256, 0, st>>>(L.perm, Np, L.xn, L.xn_m);
  k_lc_curvature<<<1, 32, 0, st>>>(L.lam_m, L.rn_m, L.xn_m, Np, L.kappa, L.corner, 0, nullptr);
  // X rows in the merged order
  TK_LAUNCH_CHECK();
  k_gather_x<<<rgrid(P.n, Np), 256, 0, st>>>(L.Xs, P.n, L.perm, X);
  TK_LAUNCH_CHECK();
  std::vector<double> hl(Np), hr(Np), hx(Np), hk(Np);
  int hc = -1, herr = 0;
  TK_CUDA(cudaMemcpyAsync(hl.data(), L.lam_m, sizeof(double) * Np, cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaMemcpyAsync(hr.data(), L.rn_m, sizeof(double) * Np, cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaMemcpyAsync(hx.data(), L.xn_m, sizeof(double) * Np, cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaMemcpyAsync(hk.data(), L.kappa, sizeof(double) * Np, cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaMemcpyAsync(&hc, L.corner, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (P.mixed && P.o.emulate_fp64) TK_CUDA(cudaMemcpyAsync(&herr, B.oz_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    set_error_msg("tk_lcurve: an emulated float64 residual pass timed out");
    return TK_ETIMEOUT;
  }
  tk_status worst = TK_OK;
  for (int i = 0; i < Np; ++i) {
    const tk_info& q = info[perm[i]];
    points[i].lambda = hl[i];
    points[i].rnorm = hr[i];
    points[i].xnorm = hx[i];
    points[i].curvature = hk[i];
    points[i].iters = q.iters;
    points[i].status = q.status;
    worst = worse(worst, q.status);
  }
  *corner = hc;
  return worst;
}

// ---- the products of one LSQR step on their own (parity of the fused form) ----------
namespace {
struct StepBufs {
  void *Aoz, *AozC, *colmax, *Wq, *Uq;
  int *EA, *EC, *EW, *EU, *err;
  double* part;
  float* A32;
  int planes;
};
void step_carve(Arena& a, int64_t m, int64_t n, int count, StepBufs& w) {
  w.planes = std::max({oz_normal_splits(m, n, count, OZ_LSQR_DIGITS), 152, lm_small_atu_splits(m, n)});
  w.A32 = a.take<float>((size_t)m * n);
  w.Aoz = a.take<char>(oz_slices_bytes(m, n));
  w.EA = a.take<int>(m);
  w.AozC = a.take<char>(oz_slices_bytes(n, m));
  w.EC = a.take<int>(n);
  w.colmax = a.take<char>(oz_colmax_bytes(n));
  w.Wq = a.take<char>(oz_slices_bytes(count, n, OZ_LSQR_DIGITS));
  w.EW = a.take<int>(count);
  w.Uq = a.take<char>(oz_slices_bytes(count, m, OZ_LSQR_DIGITS));
  w.EU = a.take<int>(count);
  w.part = a.take<double>((size_t)w.planes * count * n);
  w.err = a.take<int>(4);
}
}  // namespace
namespace tk {
__global__ void k_step_to_f32(const double* __restrict__ s, int64_t rows, int64_t cols, int64_t lds,
                              float* __restrict__ d) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < rows * cols; k += (int64_t)gridDim.x * blockDim.x)
    d[k] = (float)s[(k / cols) * lds + k % cols];
}
__global__ void k_step_sum_planes(const double* __restrict__ part, int planes, int64_t total, double* __restrict__ G) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < planes; ++z) acc += part[(int64_t)z * total + k];
    G[k] = acc;
  }
}
}  // namespace tk

TK_API size_t tk_lsqr_step_products_workspace(int64_t m, int64_t n, int count) {
  if (m < 1 || n < 1 || count < 1) return 0;
  Arena a;
  StepBufs w;
  step_carve(a, m, n, count, w);
  return a.used + 1024;
}

TK_API tk_status tk_lsqr_step_products(const tk_problem* p, const float* W, int count, float* U, const double* coef,
                                       double* G, int mode, void* work, size_t work_bytes, void* stream) {
  if (!p || !p->A || !W || !U || !G || count < 1 || count > 32 || p->m < 1 || p->n < 1 || p->lda < p->n)
    return einval("bad step-product arguments (1 <= count <= 32)");
  if (p->dtype != TK_F64 && p->dtype != TK_F32) return einval("unknown dtype");
  if (mode < 0 || mode > 2) return einval("mode must be 0, 1 or 2");
  const bool fused = mode == 1;
  if (fused && !oz_fused_supported(p->m, p->n, count)) return einval("the fused step needs n <= 2048");
  if (mode == 2 && !(count <= 16 && lm_small_aw_supported(p->n, count)))
    return einval("the float32 products need count <= 16 and W within shared memory");
  if (!work || work_bytes < tk_lsqr_step_products_workspace(p->m, p->n, count)) {
    set_error_msg("workspace smaller than tk_lsqr_step_products_workspace()");
    return TK_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  StepBufs w;
  step_carve(a, p->m, p->n, count, w);
  const int64_t m = p->m, n = p->n;
  TK_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  int planes = 0;
  if (mode == 2) {  // the float32 products of the tail (<= 16 lambda) from a float32 copy of A
    const float* A32 = static_cast<const float*>(p->A);
    int64_t lda32 = p->lda;
    if (p->dtype == TK_F64) {
      k_step_to_f32<<<(unsigned)std::min<int64_t>(cdiv(m * n, 256), 152 * 32), 256, 0, st>>>(
          static_cast<const double*>(p->A), m, n, p->lda, w.A32);
      TK_LAUNCH_CHECK();
      A32 = w.A32;
      lda32 = n;
    }
    TK_TRY(lm_small_aw(A32, lda32, m, n, W, n, count, U, m, coef, st));
    planes = std::min(w.planes, lm_small_atu_splits(m, n));
    TK_TRY(lm_small_atu(A32, lda32, m, n, U, m, count, w.part, planes, st));
  } else {
  TK_TRY(oz_prepare(p->A, p->dtype, m, n, p->lda, w.Aoz, w.EA, st));
  if (fused) {
    TK_TRY(oz_lsqr_fused(w.Aoz, w.EA, m, n, W, n, count, w.Wq, w.EW, U, m, coef, w.part, w.planes, &planes, w.err,
                         st));
  } else {
    TK_TRY(oz_prepare_cols(p->A, p->dtype, m, n, p->lda, w.AozC, w.EC, w.colmax, st));
    TK_TRY(oz_lsqr_aw(w.Aoz, w.EA, m, n, W, n, count, w.Wq, w.EW, U, m, coef, w.err, st));
    planes = std::min(w.planes, oz_normal_splits(m, n, count, OZ_LSQR_DIGITS));
    TK_TRY(oz_lsqr_atu(w.AozC, w.EC, m, n, U, m, count, w.Uq, w.EU, w.part, planes, w.err, st));
  }
  }
  const int64_t total = (int64_t)count * n;
  k_step_sum_planes<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), 152 * 8)), 256, 0, st>>>(
      w.part, planes, total, G);
  TK_LAUNCH_CHECK();
  int herr = 0;
  TK_CUDA(cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    set_error_msg("LSQR step products: a pipeline wait timed out");
    return TK_ETIMEOUT;
  }
  return TK_OK;
}

}  // extern "C"
