// Grouped mixed-precision solve of many independent overdetermined problems
// (the batching form of Algorithms 1 and 3 over uneven problems).
//
// Every active lambda of every problem owns a slot; problem p keeps its slots
// 0..nact_p-1 contiguous (a retired slot is refilled by the problem's last
// active one), lambda-major as in the single-problem engine.  One launch per
// phase covers all problems:
//   * the two float32 products with A run over a tile list (problem, column
//     tile[, K split]); a tile multiplies every active lambda of its problem
//     (the lambda-major tile body shared with the single-problem GEMM),
//   * the per-slot kernels (norms, Golub-Kahan scalars, preconditioner apply)
//     run over a slot list (problem, slot),
//   * the float64 refinement passes (r = b - A x and A^T r - lambda x) run
//     over tile lists of the generic GEMM tile body.
// The host reads one small report per step to retire converged slots.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "tk_gemm_tiles.cuh"
#include "tk_group.cuh"
#include "tk_lsqr.cuh"

namespace tk {
namespace {

constexpr int kThreads = 256;
constexpr int64_t kKps = 4096;    // rows of A per K split of the float32 A^T U product
constexpr int64_t kKps64 = 4096;  // rows of A per K split of the float64 A^T r pass
constexpr int kBM64 = 32, kBN64 = 128;

struct GDesc {
  int64_t m, n;
  const float* A32;
  int64_t lda32;
  const void* Af;
  int f64;
  int64_t ldaf;
  const double* b;
  const double* lam;
  double* X;
  int lowrank;
  const float* Mi;
  const float* Mti;
  int64_t np;
  const float* lrV;
  const float* lrS;
  int64_t lr_s;
  double atol;
  int maxiter;
  // slot storage: row k of each N x n (or N x m) block belongs to local slot k
  float *V, *W, *Y, *Vraw, *Tt, *Ub, *Xt, *Ut;
  double* part;  // splits x nact x n  (float32 A^T U partial sums)
  int splits;
  double* coef;
  Scal* sc;
  int* slot_lam;
  // refinement: the round's lambda list and the float64 pass buffers
  const int* ids;
  double *D, *Xa, *G, *Rres, *part64;  // part64: splits64 x cnt x n
  int splits64;
  int sp64;  // planes of part64 written this round (<= splits64)
  double* nrm;  // 3 x N
};

struct GSlot {
  int p, k;
};
struct GTile {
  int p, z, m0, pad;
  int64_t n0;
};
struct GReport {
  int istop, iters;
  double rnorm, arnorm;
};
struct GMove {
  int p, src, dst, pad;
};

enum Field : int { F_V = 0, F_W, F_Y, F_VRAW, F_TT, F_UB, F_XT };

__device__ __forceinline__ float* field(const GDesc& d, int f) {
  switch (f) {
    case F_V: return d.V;
    case F_W: return d.W;
    case F_Y: return d.Y;
    case F_VRAW: return d.Vraw;
    case F_TT: return d.Tt;
    case F_UB: return d.Ub;
    default: return d.Xt;
  }
}

// ---- LSQR, per slot --------------------------------------------------------
// Round start: slot k takes lambda ids[k]; Ut = b (round 0) or 0 and
// Ub = 0 (round 0) or G_k / sqrt(l): the right-hand side [b; 0] or [0; g/sqrt(l)].
__global__ void k_g_init(const GDesc* __restrict__ Dd, const GSlot* __restrict__ sl, int round0) {
  const GSlot q = sl[blockIdx.y];
  const GDesc& d = Dd[q.p];
  const int l = d.ids[q.k];
  const double lv = d.lam[l];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Scal z;
    memset(&z, 0, sizeof(z));
    z.lam_idx = l;
    z.lam = lv;
    z.sqrtl = sqrt(lv);
    d.sc[q.k] = z;
    d.slot_lam[q.k] = l;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float* ut = d.Ut + (int64_t)q.k * d.m;
  for (int64_t i = i0; i < d.m; i += stride) ut[i] = round0 ? (float)d.b[i] : 0.f;
  float* ub = d.Ub + (int64_t)q.k * d.n;
  const double inv = 1.0 / sqrt(lv);
  const double* g = d.G + (int64_t)q.k * d.n;
  for (int64_t j = i0; j < d.n; j += stride) ub[j] = round0 ? 0.f : (float)(g[j] * inv);
}

// beta_1 = ||[Ut; Ub]||; scalars reset.
__global__ void __launch_bounds__(kThreads) k_g_init_beta(const GDesc* __restrict__ Dd, const GSlot* __restrict__ sl) {
  __shared__ double sh[32];
  const GSlot q = sl[blockIdx.x];
  const GDesc& d = Dd[q.p];
  const float* ut = d.Ut + (int64_t)q.k * d.m;
  const float* ub = d.Ub + (int64_t)q.k * d.n;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < d.m; i += blockDim.x) acc = fma((double)ut[i], (double)ut[i], acc);
  for (int64_t j = threadIdx.x; j < d.n; j += blockDim.x) acc = fma((double)ub[j], (double)ub[j], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    const double beta = sqrt(acc);
    Scal z = d.sc[q.k];
    z.beta = beta;
    z.bnorm = beta;
    z.phibar = beta;
    z.anorm2 = 0.0;
    z.iters = 0;
    z.istop = (beta == 0.0) ? 1 : 0;
    z.rnorm = beta;
    z.arnorm = 0.0;
    z.ynorm = 0.0;
    d.sc[q.k] = z;
  }
}

// Tt = (sum_z part_z + sqrt(l) Ub) / beta   (the normalized A^T u part of M^T u)
__global__ void k_g_over_g(const GDesc* __restrict__ Dd, const int* __restrict__ nact, const GSlot* __restrict__ sl) {
  const GSlot q = sl[blockIdx.y];
  const GDesc& d = Dd[q.p];
  const double sq = d.sc[q.k].sqrtl, beta = d.sc[q.k].beta;
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  const int64_t plane = (int64_t)nact[q.p] * d.n;
  const float* ub = d.Ub + (int64_t)q.k * d.n;
  float* tt = d.Tt + (int64_t)q.k * d.n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < d.splits; ++z) acc += d.part[z * plane + (int64_t)q.k * d.n + j];
    acc = fma(sq, (double)ub[j], acc);
    tt[j] = (float)(acc * inv);
  }
}

// Ub = sqrt(l) Tt + coef Ub;  beta = ||[Ut; Ub]||;  anorm2 += alpha^2 + beta^2
__global__ void __launch_bounds__(kThreads) k_g_beta(const GDesc* __restrict__ Dd, const GSlot* __restrict__ sl) {
  __shared__ double sh[32];
  const GSlot q = sl[blockIdx.x];
  const GDesc& d = Dd[q.p];
  const double sq = d.sc[q.k].sqrtl, coef = d.sc[q.k].coef;
  const float* ut = d.Ut + (int64_t)q.k * d.m;
  const float* tt = d.Tt + (int64_t)q.k * d.n;
  float* ub = d.Ub + (int64_t)q.k * d.n;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < d.m; i += blockDim.x) acc = fma((double)ut[i], (double)ut[i], acc);
  for (int64_t j = threadIdx.x; j < d.n; j += blockDim.x) {
    const float v = (float)fma(sq, (double)tt[j], coef * (double)ub[j]);
    ub[j] = v;
    acc = fma((double)v, (double)v, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    const double beta = sqrt(acc);
    Scal z = d.sc[q.k];
    z.anorm2 += z.alpha * z.alpha + beta * beta;
    z.beta = beta;
    d.sc[q.k] = z;
  }
}

// The v-step (shared body with the single-problem engine); the GEMM
// coefficient -alpha/beta and a report for the host are written beside it.
__global__ void __launch_bounds__(kThreads)
    k_g_vstep(const GDesc* __restrict__ Dd, const GSlot* __restrict__ sl, int init, GReport* __restrict__ rep) {
  __shared__ double sh[32];
  const GSlot q = sl[blockIdx.x];
  const GDesc& d = Dd[q.p];
  const int64_t off = (int64_t)q.k * d.n;
  vstep_block<float>(d.Vraw + off, d.V + off, d.W + off, d.Y + off, d.n, d.sc + q.k, d.atol, d.atol, d.maxiter,
                     init, sh);
  if (threadIdx.x == 0) {  // the thread that wrote the scalars
    const Scal z = d.sc[q.k];
    d.coef[q.k] = z.coef;
    GReport r;
    r.istop = z.istop;
    r.iters = z.iters;
    r.rnorm = z.rnorm;
    r.arnorm = z.arnorm;
    rep[blockIdx.x] = r;
  }
}

// ---- preconditioner apply, per slot ----------------------------------------
// Cholesky problems: out = R^-1 in (UPPER) or R^-T in, explicit float32 inverse.
template <bool UPPER>
__global__ void __launch_bounds__(256)
    k_g_trmv(const GDesc* __restrict__ Dd, const GSlot* __restrict__ sl, int fsrc, int fdst) {
  extern __shared__ float4 g_trmv_v4[];  // 16-byte aligned staging
  const GSlot q = sl[blockIdx.y];
  const GDesc& d = Dd[q.p];
  const int64_t i0 = (int64_t)blockIdx.x * tiles::kTrmvRows;
  if (d.lowrank || i0 >= d.n) return;
  const float* Ml = (UPPER ? d.Mi : d.Mti) + (int64_t)d.slot_lam[q.k] * d.np * d.np;
  tiles::trmv_rows<float, UPPER>(d.n, Ml, d.np, field(d, fsrc) + (int64_t)q.k * d.n,
                                 field(d, fdst) + (int64_t)q.k * d.n, i0, g_trmv_v4);
}

// Low-rank problems (Section 3.1): out = l^{-1/2} (x - V diag(S_l) V^T x),
// symmetric, one CTA per slot; x and t = S_l V^T x / sqrt(l) in shared memory.
__global__ void __launch_bounds__(256)
    k_g_lr(const GDesc* __restrict__ Dd, const GSlot* __restrict__ sl, int fsrc, int fdst) {
  extern __shared__ float g_lr_sm[];
  const GSlot q = sl[blockIdx.x];
  const GDesc& d = Dd[q.p];
  if (!d.lowrank) return;
  const int64_t n = d.n, s = d.lr_s;
  const int l = d.slot_lam[q.k];
  const float* x = field(d, fsrc) + (int64_t)q.k * n;
  float* y = field(d, fdst) + (int64_t)q.k * n;
  float* xs = g_lr_sm;
  float* t = g_lr_sm + n;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) xs[j] = x[j];
  __syncthreads();
  const double is = 1.0 / sqrt(d.lam[l]);
  const float* V = d.lrV;
  const float* S = d.lrS + (int64_t)l * s;
  for (int64_t c = threadIdx.x; c < s; c += blockDim.x) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int64_t i = 0;
    for (; i + 3 < n; i += 4) {
      a0 = fmaf(V[i * s + c], xs[i], a0);
      a1 = fmaf(V[(i + 1) * s + c], xs[i + 1], a1);
      a2 = fmaf(V[(i + 2) * s + c], xs[i + 2], a2);
      a3 = fmaf(V[(i + 3) * s + c], xs[i + 3], a3);
    }
    for (; i < n; ++i) a0 = fmaf(V[i * s + c], xs[i], a0);
    const float a = (a0 + a1) + (a2 + a3);
    t[c] = (float)((double)a * (double)S[c] * is);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t i = w; i < n; i += nw) {
    float acc = 0.f;
    for (int64_t c = lane; c < s; c += 32) acc = fmaf(V[i * s + c], t[c], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[i] = (float)(-(double)acc + is * (double)xs[i]);
  }
}

// ---- the two products with A, over tile lists --------------------------------
// TRANSB: Ut = Tt A^T + coef .* Ut (tile = problem, 256 rows of A).
// else:   part_z = Ut A over rows [z kKps, (z+1) kKps) (tile = problem, 256
//         columns, split z).
template <bool TRANSB, int BM, int TM>
__global__ void __launch_bounds__(256)
    k_g_lm(const GDesc* __restrict__ Dd, const int* __restrict__ nact, const GTile* __restrict__ tl) {
  __shared__ __align__(16) tiles::LmSmem<BM> sm;
  const GTile t = tl[blockIdx.x];
  const int M = nact[t.p];
  if (M == 0) return;
  const GDesc& d = Dd[t.p];
  const bool abase = ((uintptr_t)d.A32 % 16 == 0) && (d.lda32 % 4 == 0);
  if (TRANSB) {
    tiles::gemm_lm_tile<true, BM, TM>(sm, abase && (d.n % 4 == 0), M, d.m, d.Tt, d.n, d.A32, d.lda32, d.Ut, d.m,
                                      d.coef, d.Ut, d.m, t.n0, 0, d.n, nullptr);
  } else {
    const int64_t kb = (int64_t)t.z * kKps, ke = std::min<int64_t>(d.m, kb + kKps);
    tiles::gemm_lm_tile<false, BM, TM>(sm, abase && (d.m % 4 == 0), M, d.n, d.Ut, d.m, d.A32, d.lda32, nullptr, 0,
                                       nullptr, nullptr, 0, t.n0, kb, ke, d.part + (int64_t)t.z * M * d.n);
  }
}

// ---- retirement ----------------------------------------------------------------
// D[l] = Xt[k] for the listed (retiring) slots: the correction of lambda l.
__global__ void k_g_scatter(const GDesc* __restrict__ Dd, const GSlot* __restrict__ sl) {
  const GSlot q = sl[blockIdx.y];
  const GDesc& d = Dd[q.p];
  const int l = d.slot_lam[q.k];
  const float* x = d.Xt + (int64_t)q.k * d.n;
  double* o = d.D + (int64_t)l * d.n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x)
    o[j] = (double)x[j];
}

// Refill retired slot dst of problem p with its active slot src (src >= the
// new active count > dst: sources and destinations are disjoint).
__global__ void k_g_move(const GDesc* __restrict__ Dd, const GMove* __restrict__ mv) {
  const GMove q = mv[blockIdx.y];
  const GDesc& d = Dd[q.p];
  const int64_t n = d.n, m = d.m;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t j = i0; j < n; j += stride) {
    d.V[q.dst * n + j] = d.V[q.src * n + j];
    d.W[q.dst * n + j] = d.W[q.src * n + j];
    d.Y[q.dst * n + j] = d.Y[q.src * n + j];
    d.Ub[q.dst * n + j] = d.Ub[q.src * n + j];
  }
  for (int64_t i = i0; i < m; i += stride) d.Ut[q.dst * m + i] = d.Ut[q.src * m + i];
  if (i0 == 0) {
    d.sc[q.dst] = d.sc[q.src];
    d.slot_lam[q.dst] = d.slot_lam[q.src];
    d.coef[q.dst] = d.coef[q.src];
  }
}

// ---- float64 refinement passes ---------------------------------------------------
// Xa[k] = X[ids[k]]
__global__ void k_g_gather_x(const GDesc* __restrict__ Dd, const GSlot* __restrict__ sl) {
  const GSlot q = sl[blockIdx.y];
  const GDesc& d = Dd[q.p];
  const double* x = d.X + (int64_t)d.ids[q.k] * d.n;
  double* o = d.Xa + (int64_t)q.k * d.n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n; j += (int64_t)gridDim.x * blockDim.x)
    o[j] = x[j];
}

// MODE 0: Rres = b - Xa A^T (tile = problem, 32 lambda rows, 128 rows of A);
// MODE 1: part64_z = Rres A over rows [z kKps64, ...) (tile = problem, 32
// lambda rows, 128 columns, split z).  Float64 arithmetic on A as given.
template <typename TB, int MODE>
__global__ void __launch_bounds__(256) k_g_gemm64(const GDesc* __restrict__ Dd, const int* __restrict__ cnt,
                                                  const GTile* __restrict__ tl, const double* __restrict__ ones) {
  __shared__ tiles::GemmSmem<double, TB, kBM64, kBN64, 16> sm;
  const GTile t = tl[blockIdx.x];
  const GDesc& d = Dd[t.p];
  const int M = cnt[t.p];
  const TB* Af = reinterpret_cast<const TB*>(d.Af);
  if (MODE == 0) {
    tiles::gemm_tile<double, TB, double, kBM64, kBN64, 16, 4, 4>(sm, false, true, M, d.m, d.Xa, d.n, Af, d.ldaf,
                                                                 d.Rres, d.m, -1.0, ones, d.b, 0, t.m0, t.n0, 0,
                                                                 d.n, nullptr);
  } else {
    const int64_t kb = (int64_t)t.z * kKps64, ke = std::min<int64_t>(d.m, kb + kKps64);
    tiles::gemm_tile<double, TB, double, kBM64, kBN64, 16, 4, 4>(sm, false, false, M, d.n, d.Rres, d.m, Af, d.ldaf,
                                                                 nullptr, 0, 1.0, nullptr, nullptr, 0, t.m0, t.n0,
                                                                 kb, ke, d.part64 + (int64_t)t.z * M * d.n);
  }
}

// G[k] = sum_z part64_z[k] - lambda Xa[k]  (A^T (b - A x) - lambda x); nrm[3k] = ||G[k]||
__global__ void __launch_bounds__(kThreads)
    k_g_ne_finish(const GDesc* __restrict__ Dd, const int* __restrict__ cnt, const GSlot* __restrict__ sl) {
  __shared__ double sh[32];
  const GSlot q = sl[blockIdx.x];
  const GDesc& d = Dd[q.p];
  const double lv = d.lam[d.ids[q.k]];
  const int64_t plane = (int64_t)cnt[q.p] * d.n;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < d.n; j += blockDim.x) {
    double g = 0.0;
    for (int z = 0; z < d.sp64; ++z) g += d.part64[z * plane + (int64_t)q.k * d.n + j];
    g = fma(-lv, d.Xa[(int64_t)q.k * d.n + j], g);
    d.G[(int64_t)q.k * d.n + j] = g;
    acc = fma(g, g, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) d.nrm[3 * q.k] = sqrt(acc);
}

// X_l += D_l;  nrm[3k+1] = ||D_l||, nrm[3k+2] = ||X_l||
__global__ void __launch_bounds__(kThreads) k_g_refine_update(const GDesc* __restrict__ Dd, const GSlot* __restrict__ sl) {
  __shared__ double sh[32];
  const GSlot q = sl[blockIdx.x];
  const GDesc& d = Dd[q.p];
  const int l = d.ids[q.k];
  double dd = 0.0, xx = 0.0;
  for (int64_t j = threadIdx.x; j < d.n; j += blockDim.x) {
    const double dv = d.D[(int64_t)l * d.n + j];
    const double x = d.X[(int64_t)l * d.n + j] + dv;
    d.X[(int64_t)l * d.n + j] = x;
    dd = fma(dv, dv, dd);
    xx = fma(x, x, xx);
  }
  dd = block_sum(dd, sh);
  xx = block_sum(xx, sh);
  if (threadIdx.x == 0) {
    d.nrm[3 * q.k + 1] = sqrt(dd);
    d.nrm[3 * q.k + 2] = sqrt(xx);
  }
}

__global__ void k_g_fill(double* x, int n, double v) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = v;
}

inline dim3 chunk_grid(int64_t len, int rows) {
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(len, 256), 16)), (unsigned)rows);
}

// ---- host side ---------------------------------------------------------------------
struct Sizes {
  int splits = 1, splits64 = 1;
};

Sizes sizes_of(const GroupProblem& g) {
  Sizes z;
  z.splits = (int)std::max<int64_t>(1, cdiv(g.m, kKps));
  z.splits64 = (int)std::max<int64_t>(1, cdiv(g.m, kKps64));
  return z;
}

struct GState {
  int P = 0, N = 0, BM = 16;
  int64_t maxn = 0;
  std::vector<GDesc> hd;
  GDesc* dd = nullptr;
  int* nact = nullptr;
  int* cnt = nullptr;
  int* ids_all = nullptr;
  double* nrm_all = nullptr;
  double* ones = nullptr;
  GSlot* slots = nullptr;   // live slot list of the running LSQR
  GSlot* rnd = nullptr;     // the round's list (slot k of problem p <-> ids[k])
  GSlot* rslots = nullptr;  // retiring slots
  GMove* moves = nullptr;
  GReport* rep = nullptr;
  GTile* t_aw = nullptr;
  GTile* t_atu = nullptr;
  GTile* t_64 = nullptr;  // per-round float64 tiles (residual, then normal equations)
  int n_aw = 0, n_atu = 0;
  size_t cap64 = 0;
  double fl_aw = 0.0;  // flops of one step (all slots active): for the profiler
  // the emulated float64 passes: digit planes of one problem at a time (the largest fits)
  int64_t oz_m = 0, oz_n = 0;
  size_t oz_rows_bytes = 0, oz_cols_bytes = 0, oz_vec_bytes = 0;
  void *oz_rows = nullptr, *oz_cols = nullptr, *oz_colmax = nullptr, *oz_vec = nullptr;
  int *oz_EA = nullptr, *oz_EC = nullptr, *oz_EV = nullptr, *oz_err = nullptr;
};

void carve_group(const std::vector<GroupProblem>& g, int N, Arena& a, GState& S) {
  const int P = (int)g.size();
  S.P = P;
  S.N = N;
  S.hd.assign(P, GDesc{});
  size_t naw = 0, natu = 0, n64 = 0;
  for (int p = 0; p < P; ++p) {
    const GroupProblem& q = g[p];
    const Sizes z = sizes_of(q);
    GDesc& d = S.hd[p];
    memset(&d, 0, sizeof(d));
    d.m = q.m;
    d.n = q.n;
    d.A32 = q.A32;
    d.lda32 = q.lda32;
    d.Af = q.Af;
    d.f64 = q.f64;
    d.ldaf = q.ldaf;
    d.b = q.b;
    d.lam = q.lam;
    d.X = q.X;
    d.lowrank = q.lowrank;
    d.Mi = q.Mi;
    d.Mti = q.Mti;
    d.np = q.np;
    d.lrV = q.lrV;
    d.lrS = q.lrS;
    d.lr_s = q.lr_s;
    d.atol = q.inner_tol;
    d.maxiter = q.maxiter;
    const size_t vn = (size_t)N * q.n;
    d.V = a.take<float>(vn);
    d.W = a.take<float>(vn);
    d.Y = a.take<float>(vn);
    d.Vraw = a.take<float>(vn);
    d.Tt = a.take<float>(vn);
    d.Ub = a.take<float>(vn);
    d.Xt = a.take<float>(vn);
    d.Ut = a.take<float>((size_t)N * q.m);
    d.splits = z.splits;
    d.part = a.take<double>((size_t)z.splits * vn);
    d.coef = a.take<double>(N);
    d.sc = a.take<Scal>(N);
    d.slot_lam = a.take<int>(N);
    d.D = a.take<double>(vn);
    d.Xa = a.take<double>(vn);
    d.G = a.take<double>(vn);
    d.Rres = a.take<double>((size_t)N * q.m);
    d.splits64 = z.splits64;
    d.sp64 = z.splits64;
    d.part64 = a.take<double>((size_t)z.splits64 * vn);
    if (q.emulate) {
      S.oz_m = std::max(S.oz_m, q.m);
      S.oz_n = std::max(S.oz_n, q.n);
      S.oz_rows_bytes = std::max(S.oz_rows_bytes, oz_slices_bytes(q.m, q.n));
      S.oz_cols_bytes = std::max(S.oz_cols_bytes, oz_slices_bytes(q.n, q.m));
      S.oz_vec_bytes = std::max({S.oz_vec_bytes, oz_slices_bytes(N, q.n), oz_slices_bytes(N, q.m)});
    }
    naw += (size_t)cdiv(q.m, tiles::LM_BN);
    natu += (size_t)cdiv(q.n, tiles::LM_BN) * z.splits;
    n64 += (size_t)cdiv(N, kBM64) * (size_t)std::max(cdiv(q.m, kBN64), cdiv(q.n, kBN64) * z.splits64);
    S.maxn = std::max(S.maxn, q.n);
  }
  S.dd = a.take<GDesc>(std::max(P, 1));
  S.nact = a.take<int>(std::max(P, 1));
  S.cnt = a.take<int>(std::max(P, 1));
  S.ids_all = a.take<int>((size_t)std::max(P, 1) * N);
  S.nrm_all = a.take<double>((size_t)std::max(P, 1) * 3 * N);
  S.ones = a.take<double>(kGroupMaxLambda);
  const size_t ns = (size_t)std::max(P, 1) * N;
  S.slots = a.take<GSlot>(ns);
  S.rnd = a.take<GSlot>(ns);
  S.rslots = a.take<GSlot>(ns);
  S.moves = a.take<GMove>(ns);
  S.rep = a.take<GReport>(ns);
  S.t_aw = a.take<GTile>(std::max<size_t>(naw, 1));
  S.t_atu = a.take<GTile>(std::max<size_t>(natu, 1));
  S.t_64 = a.take<GTile>(std::max<size_t>(n64, 1));
  S.cap64 = n64;
  for (int p = 0; p < P; ++p) {
    S.hd[p].ids = S.ids_all + (size_t)p * N;
    S.hd[p].nrm = S.nrm_all + (size_t)p * 3 * N;
  }
  S.BM = N <= 16 ? 16 : (N <= 32 ? 32 : 64);
  if (S.oz_rows_bytes > 0) {
    // the largest problem's digit planes of A's rows and columns, and of the lambda-side vectors
    // (X: N x n, r: N x m), reused problem by problem
    S.oz_rows = a.take<char>(S.oz_rows_bytes);
    S.oz_cols = a.take<char>(S.oz_cols_bytes);
    S.oz_colmax = a.take<char>(oz_colmax_bytes(S.oz_n));
    S.oz_vec = a.take<char>(S.oz_vec_bytes);
    S.oz_EA = a.take<int>((size_t)S.oz_m);
    S.oz_EC = a.take<int>((size_t)S.oz_n);
    S.oz_EV = a.take<int>((size_t)N);
    S.oz_err = a.take<int>(4);
  }
}

// ---- launch helpers ----------------------------------------------------------------
tk_status launch_lm(const GState& S, bool transb, cudaStream_t st) {
  const GTile* tl = transb ? S.t_aw : S.t_atu;
  const int nt = transb ? S.n_aw : S.n_atu;
  if (nt == 0) return TK_OK;
#define TK_GLM(TRB, BMV, TMV) k_g_lm<TRB, BMV, TMV><<<nt, 256, 0, st>>>(S.dd, S.nact, tl)
  if (S.BM == 16) { if (transb) TK_GLM(true, 16, 2); else TK_GLM(false, 16, 2); }
  else if (S.BM == 32) { if (transb) TK_GLM(true, 32, 4); else TK_GLM(false, 32, 4); }
  else { if (transb) TK_GLM(true, 64, 8); else TK_GLM(false, 64, 8); }
#undef TK_GLM
  TK_LAUNCH_CHECK();
  return TK_OK;
}

// Preconditioner apply over a slot list (both kinds; each kernel skips the other's slots).
tk_status launch_prec(const GState& S, bool transposed, const GSlot* sl, int nsl, int fsrc, int fdst,
                      bool any_chol, bool any_lr, cudaStream_t st) {
  if (nsl == 0) return TK_OK;
  if (any_chol) {
    const dim3 grid((unsigned)cdiv(S.maxn, tiles::kTrmvRows), (unsigned)nsl);
    const size_t smem = tiles::trmv_smem_bytes<float>(S.maxn);
    if (!transposed) k_g_trmv<true><<<grid, 256, smem, st>>>(S.dd, sl, fsrc, fdst);
    else k_g_trmv<false><<<grid, 256, smem, st>>>(S.dd, sl, fsrc, fdst);
    TK_LAUNCH_CHECK();
  }
  if (any_lr) {
    k_g_lr<<<nsl, 256, sizeof(float) * 2 * (size_t)S.maxn, st>>>(S.dd, sl, fsrc, fdst);
    TK_LAUNCH_CHECK();
  }
  return TK_OK;
}

}  // namespace

size_t group_workspace(const std::vector<GroupProblem>& g, int N) {
  Arena a;
  GState S;
  carve_group(g, N, a, S);
  return a.used + 4096;
}

tk_status group_solve_mixed(std::vector<GroupProblem>& g, int N, void* work, size_t bytes, cudaStream_t st) {
  const int P = (int)g.size();
  if (P == 0 || N == 0) return TK_OK;
  if (N > kGroupMaxLambda) {
    set_error_msg("grouped solve: at most 64 lambda per problem");
    return TK_EINVAL;
  }
  Arena a;
  a.base = (char*)work;
  a.cap = bytes;
  GState S;
  carve_group(g, N, a, S);
  if (!a.ok()) {
    set_error_msg("workspace smaller than the grouped solve needs");
    return TK_ENOMEM;
  }
  bool any_chol = false, any_lr = false;
  for (const auto& q : g) {
    if (q.n > kGroupMaxN) {
      set_error_msg("grouped solve: n above 4096");
      return TK_EINVAL;
    }
    (q.lowrank ? any_lr : any_chol) = true;
  }
  TK_CUDA(cudaMemcpyAsync(S.dd, S.hd.data(), sizeof(GDesc) * P, cudaMemcpyHostToDevice, st));
  k_g_fill<<<1, 64, 0, st>>>(S.ones, kGroupMaxLambda, 1.0);
  TK_LAUNCH_CHECK();
  // tile lists of the float32 products over the problems that still have
  // active slots (rebuilt when that set shrinks by a quarter: a retired
  // problem's tiles would only launch CTAs that exit at once)
  std::vector<GTile> t_aw, t_atu;
  int tiled_problems = 0;
  auto build_tiles = [&](const std::vector<int>& live) -> tk_status {
    t_aw.clear();
    t_atu.clear();
    tiled_problems = 0;
    for (int p = 0; p < P; ++p) {
      if (!live[p]) continue;
      ++tiled_problems;
      for (int64_t n0 = 0; n0 < g[p].m; n0 += tiles::LM_BN) t_aw.push_back(GTile{p, 0, 0, 0, n0});
      for (int64_t n0 = 0; n0 < g[p].n; n0 += tiles::LM_BN)
        for (int z = 0; z < S.hd[p].splits; ++z) t_atu.push_back(GTile{p, z, 0, 0, n0});
    }
    S.n_aw = (int)t_aw.size();
    S.n_atu = (int)t_atu.size();
    if (!t_aw.empty())
      TK_CUDA(cudaMemcpyAsync(S.t_aw, t_aw.data(), sizeof(GTile) * t_aw.size(), cudaMemcpyHostToDevice, st));
    if (!t_atu.empty())
      TK_CUDA(cudaMemcpyAsync(S.t_atu, t_atu.data(), sizeof(GTile) * t_atu.size(), cudaMemcpyHostToDevice, st));
    return TK_OK;
  };
  std::vector<std::vector<int>> act(P);
  std::vector<std::vector<double>> prev_dn(P, std::vector<double>(N, INFINITY));
  for (int p = 0; p < P; ++p) act[p] = g[p].ok_ids;
  std::vector<int> hcnt(P), hnact(P);
  std::vector<std::vector<int>> mirror(P);  // host copy of slot -> lambda
  std::vector<int> ids_h((size_t)P * N);
  std::vector<double> nrm_h((size_t)P * 3 * N);
  std::vector<GSlot> rl, sl, retire;
  std::vector<GMove> mv;
  std::vector<GReport> rep((size_t)P * N);
  std::vector<GTile> t64;

  for (int round = 0;; ++round) {
    int total = 0;
    for (int p = 0; p < P; ++p) {
      if (round >= g[p].max_refine) {
        for (int l : act[p]) g[p].inf[l].status = worse(g[p].inf[l].status, TK_ENOCONV);
        act[p].clear();
      }
      hcnt[p] = (int)act[p].size();
      total += hcnt[p];
      std::copy(act[p].begin(), act[p].end(), ids_h.begin() + (size_t)p * N);
    }
    if (total == 0) break;
    rl.clear();
    for (int p = 0; p < P; ++p)
      for (int k = 0; k < hcnt[p]; ++k) rl.push_back(GSlot{p, k});
    const int nrl = (int)rl.size();
    TK_CUDA(cudaMemcpyAsync(S.ids_all, ids_h.data(), sizeof(int) * ids_h.size(), cudaMemcpyHostToDevice, st));
    TK_CUDA(cudaMemcpyAsync(S.cnt, hcnt.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
    TK_CUDA(cudaMemcpyAsync(S.rnd, rl.data(), sizeof(GSlot) * nrl, cudaMemcpyHostToDevice, st));

    if (round > 0) {
      // ---- float64 pass: Rres = b - A x, G = A^T Rres - lambda x, for the listed lambda
      k_g_gather_x<<<chunk_grid(S.maxn, nrl), 256, 0, st>>>(S.dd, S.rnd);
      TK_LAUNCH_CHECK();
      // problems that emulate the float64 products: r = b - Xa A^T and the planes of r A from exact
      // digits on the tensor cores, one problem at a time through the shared digit scratch
      bool any_oz = false;
      for (int p = 0; p < P; ++p) any_oz = any_oz || (hcnt[p] > 0 && g[p].emulate);
      if (any_oz) {
        TK_CUDA(cudaMemsetAsync(S.oz_err, 0, sizeof(int), st));
        for (int mode = 0; mode < 2; ++mode) {
          double fl = 0.0, by = 0.0, ib = 0.0;
          const int tok = prof_begin(mode == 0 ? TK_PHASE_RES64 : TK_PHASE_NE64, st);
          for (int p = 0; p < P; ++p) {
            if (hcnt[p] == 0 || !g[p].emulate) continue;
            const GDesc& d = S.hd[p];
            const tk_dtype dt = g[p].f64 ? TK_F64 : TK_F32;
            const int M = hcnt[p];
            if (mode == 0) {
              TK_TRY(oz_prepare(g[p].Af, dt, g[p].m, g[p].n, g[p].ldaf, S.oz_rows, S.oz_EA, st));
              TK_TRY(oz_prepare(d.Xa, TK_F64, M, g[p].n, g[p].n, S.oz_vec, S.oz_EV, st));
              TK_TRY(oz_residual(S.oz_rows, S.oz_EA, g[p].m, g[p].n, S.oz_vec, S.oz_EV, M, g[p].b, d.Rres, g[p].m,
                                 S.oz_err, st));
            } else {
              const int sp = std::min(d.splits64, oz_normal_splits(g[p].m, g[p].n, M));
              TK_TRY(oz_prepare_cols(g[p].Af, dt, g[p].m, g[p].n, g[p].ldaf, S.oz_cols, S.oz_EC, S.oz_colmax, st));
              TK_TRY(oz_normal(S.oz_cols, S.oz_EC, g[p].m, g[p].n, d.Rres, g[p].m, M, S.oz_vec, S.oz_EV, d.part64, sp,
                               S.oz_err, st));
              S.hd[p].sp64 = sp;
            }
            const double es = g[p].f64 ? 8.0 : 4.0;
            fl += 2.0 * M * g[p].m * g[p].n;
            by += es * g[p].m * g[p].n + 16.0 * M * g[p].m;
            ib += (2.0 * es + 32.0) * g[p].m * g[p].n + 16.0 * M * g[p].m;  // A read twice, 8 planes out and in
          }
          prof_end(tok, st, fl, by, ib);
        }
        TK_CUDA(cudaMemcpyAsync(S.dd, S.hd.data(), sizeof(GDesc) * P, cudaMemcpyHostToDevice, st));
      }
      for (int mode = 0; mode < 2; ++mode) {
        for (int f = 0; f < 2; ++f) {  // float64 and float32 inputs launch separately
          t64.clear();
          double fl = 0.0, by = 0.0;
          for (int p = 0; p < P; ++p) {
            if (hcnt[p] == 0 || g[p].f64 != (f == 0) || g[p].emulate) continue;
            for (int m0 = 0; m0 < hcnt[p]; m0 += kBM64) {
              if (mode == 0) {
                for (int64_t n0 = 0; n0 < g[p].m; n0 += kBN64) t64.push_back(GTile{p, 0, m0, 0, n0});
              } else {
                for (int64_t n0 = 0; n0 < g[p].n; n0 += kBN64)
                  for (int z = 0; z < S.hd[p].splits64; ++z) t64.push_back(GTile{p, z, m0, 0, n0});
              }
            }
            fl += 2.0 * hcnt[p] * g[p].m * g[p].n;
            by += (g[p].f64 ? 8.0 : 4.0) * g[p].m * g[p].n + 16.0 * hcnt[p] * g[p].m;
          }
          if (t64.empty()) continue;
          if (t64.size() > S.cap64) {
            set_error_msg("grouped solve: float64 tile list overflow");
            return TK_EINVAL;
          }
          TK_CUDA(cudaMemcpyAsync(S.t_64, t64.data(), sizeof(GTile) * t64.size(), cudaMemcpyHostToDevice, st));
          const int tok = prof_begin(mode == 0 ? TK_PHASE_RES64 : TK_PHASE_NE64, st);
          const unsigned nt = (unsigned)t64.size();
          if (f == 0) {
            if (mode == 0) k_g_gemm64<double, 0><<<nt, 256, 0, st>>>(S.dd, S.cnt, S.t_64, S.ones);
            else k_g_gemm64<double, 1><<<nt, 256, 0, st>>>(S.dd, S.cnt, S.t_64, S.ones);
          } else {
            if (mode == 0) k_g_gemm64<float, 0><<<nt, 256, 0, st>>>(S.dd, S.cnt, S.t_64, S.ones);
            else k_g_gemm64<float, 1><<<nt, 256, 0, st>>>(S.dd, S.cnt, S.t_64, S.ones);
          }
          TK_LAUNCH_CHECK();
          prof_end(tok, st, fl, by);
          TK_CUDA(cudaStreamSynchronize(st));  // t64 is refilled
        }
      }
      k_g_ne_finish<<<nrl, kThreads, 0, st>>>(S.dd, S.cnt, S.rnd);
      TK_LAUNCH_CHECK();
      if (any_oz) {
        int herr = 0;
        TK_CUDA(cudaMemcpyAsync(&herr, S.oz_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        TK_CUDA(cudaStreamSynchronize(st));
        if (herr) {
          set_error_msg("grouped solve: a pipeline wait of the emulated float64 passes timed out");
          return TK_ETIMEOUT;
        }
      }
    }

    // ---- float32 LSQR on [b; 0] (round 0) or [0; g / sqrt(l)]: all problems together
    for (int p = 0; p < P; ++p) {
      hnact[p] = hcnt[p];
      mirror[p].assign(act[p].begin(), act[p].end());
    }
    TK_CUDA(cudaMemcpyAsync(S.nact, hnact.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
    {
      std::vector<int> live(P);
      for (int p = 0; p < P; ++p) live[p] = hnact[p] > 0;
      TK_TRY(build_tiles(live));
    }
    sl = rl;
    int nsl = nrl;
    k_g_init<<<chunk_grid(std::max<int64_t>(S.maxn, 1 << 14), nsl), 256, 0, st>>>(S.dd, S.rnd, round == 0);
    TK_LAUNCH_CHECK();
    k_g_init_beta<<<nsl, kThreads, 0, st>>>(S.dd, S.rnd);
    TK_LAUNCH_CHECK();
    auto prec_flops = [&]() {
      double f = 0.0;
      for (int p = 0; p < P; ++p)
        f += g[p].lowrank ? 4.0 * hnact[p] * g[p].n * g[p].lr_s : (double)hnact[p] * g[p].n * g[p].n;
      return f;
    };
    // (flops, algorithmic bytes: A once in its own dtype, implementation bytes: the float32 A read)
    struct FB {
      double first, second, impl;
    };
    auto step_flops = [&]() {
      FB r{0.0, 0.0, 0.0};
      for (int p = 0; p < P; ++p) {
        if (hnact[p] == 0) continue;  // retired problems are not in the tile lists
        const double mn = (double)g[p].m * g[p].n, vec = 4.0 * hnact[p] * (double)(g[p].n + 2 * g[p].m);
        r.first += 2.0 * hnact[p] * mn;
        r.second += (g[p].f64 ? 8.0 : 4.0) * mn + vec;
        r.impl += 4.0 * mn + vec;
      }
      return r;
    };
    {
      auto fb = step_flops();
      const int tok = prof_begin(TK_PHASE_ATU, st);
      TK_TRY(launch_lm(S, false, st));
      prof_end(tok, st, fb.first, fb.second, fb.impl);
    }
    k_g_over_g<<<chunk_grid(S.maxn, nsl), 256, 0, st>>>(S.dd, S.nact, S.rnd);
    TK_LAUNCH_CHECK();
    {
      const int tok = prof_begin(TK_PHASE_PRECOND, st);
      TK_TRY(launch_prec(S, true, S.rnd, nsl, F_TT, F_VRAW, any_chol, any_lr, st));
      prof_end(tok, st, prec_flops(), 0.0);
    }
    k_g_vstep<<<nsl, kThreads, 0, st>>>(S.dd, S.rnd, 1, S.rep);
    TK_LAUNCH_CHECK();
    // the live slot list is S.slots from here on
    TK_CUDA(cudaMemcpyAsync(S.slots, sl.data(), sizeof(GSlot) * nsl, cudaMemcpyHostToDevice, st));
    for (;;) {
      // ------------------------------------------------------- retire finished slots
      TK_CUDA(cudaMemcpyAsync(rep.data(), S.rep, sizeof(GReport) * nsl, cudaMemcpyDeviceToHost, st));
      TK_CUDA(cudaStreamSynchronize(st));
      retire.clear();
      for (int j = 0; j < nsl; ++j) {
        if (rep[j].istop == 0) continue;
        const GSlot q = sl[j];
        retire.push_back(q);
        const int l = mirror[q.p][q.k];
        tk_info& in = g[q.p].inf[l];
        in.iters += rep[j].iters;
        in.istop = rep[j].istop;
        in.rnorm = rep[j].rnorm;
        in.arnorm = rep[j].arnorm;
        if (rep[j].istop == 5) in.status = worse(in.status, TK_ENUMERIC);
      }
      if (!retire.empty()) {
        const int nr = (int)retire.size();
        TK_CUDA(cudaMemcpyAsync(S.rslots, retire.data(), sizeof(GSlot) * nr, cudaMemcpyHostToDevice, st));
        // x = R^-1 y of the retiring slots, written as the lambda's correction
        TK_TRY(launch_prec(S, false, S.rslots, nr, F_Y, F_XT, any_chol, any_lr, st));
        k_g_scatter<<<chunk_grid(S.maxn, nr), 256, 0, st>>>(S.dd, S.rslots);
        TK_LAUNCH_CHECK();
        // per problem: survivors beyond the new end move into holes below it
        std::vector<std::vector<char>> dead(P);
        for (const GSlot& q : retire) {
          if (dead[q.p].empty()) dead[q.p].assign(hnact[q.p], 0);
          dead[q.p][q.k] = 1;
        }
        mv.clear();
        for (int p = 0; p < P; ++p) {
          if (dead[p].empty()) continue;
          int nr_p = 0;
          for (char c : dead[p]) nr_p += c;
          const int nnew = hnact[p] - nr_p;
          std::vector<int> holes, srcs;
          for (int k = 0; k < nnew; ++k)
            if (dead[p][k]) holes.push_back(k);
          for (int k = nnew; k < hnact[p]; ++k)
            if (!dead[p][k]) srcs.push_back(k);
          for (size_t i = 0; i < holes.size(); ++i) {
            mv.push_back(GMove{p, srcs[i], holes[i], 0});
            mirror[p][holes[i]] = mirror[p][srcs[i]];
          }
          hnact[p] = nnew;
          mirror[p].resize(nnew);
        }
        if (!mv.empty()) {
          TK_CUDA(cudaMemcpyAsync(S.moves, mv.data(), sizeof(GMove) * mv.size(), cudaMemcpyHostToDevice, st));
          k_g_move<<<chunk_grid(1 << 14, (int)mv.size()), 256, 0, st>>>(S.dd, S.moves);
          TK_LAUNCH_CHECK();
        }
        sl.clear();
        for (int p = 0; p < P; ++p)
          for (int k = 0; k < hnact[p]; ++k) sl.push_back(GSlot{p, k});
        nsl = (int)sl.size();
        TK_CUDA(cudaMemcpyAsync(S.nact, hnact.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
        if (nsl > 0) TK_CUDA(cudaMemcpyAsync(S.slots, sl.data(), sizeof(GSlot) * nsl, cudaMemcpyHostToDevice, st));
        {
          std::vector<int> live(P);
          int nlive = 0;
          for (int p = 0; p < P; ++p) nlive += (live[p] = hnact[p] > 0);
          if (nlive > 0 && 4 * nlive <= 3 * tiled_problems) TK_TRY(build_tiles(live));
        }
        TK_CUDA(cudaStreamSynchronize(st));  // host lists are reused
      }
      if (nsl == 0) break;
      // ------------------------------------------------------------ one step
      auto fb = step_flops();
      int tok = prof_begin(TK_PHASE_PRECOND, st);
      TK_TRY(launch_prec(S, false, S.slots, nsl, F_V, F_TT, any_chol, any_lr, st));  // T = R^-1 v
      prof_end(tok, st, prec_flops(), 0.0);
      tok = prof_begin(TK_PHASE_AW, st);
      TK_TRY(launch_lm(S, true, st));  // Ut = T A^T - (alpha/beta) Ut
      prof_end(tok, st, fb.first, fb.second, fb.impl);
      k_g_beta<<<nsl, kThreads, 0, st>>>(S.dd, S.slots);
      TK_LAUNCH_CHECK();
      tok = prof_begin(TK_PHASE_ATU, st);
      TK_TRY(launch_lm(S, false, st));  // part = Ut A
      prof_end(tok, st, fb.first, fb.second, fb.impl);
      k_g_over_g<<<chunk_grid(S.maxn, nsl), 256, 0, st>>>(S.dd, S.nact, S.slots);
      TK_LAUNCH_CHECK();
      tok = prof_begin(TK_PHASE_PRECOND, st);
      TK_TRY(launch_prec(S, true, S.slots, nsl, F_TT, F_VRAW, any_chol, any_lr, st));  // R^-T g
      prof_end(tok, st, prec_flops(), 0.0);
      k_g_vstep<<<nsl, kThreads, 0, st>>>(S.dd, S.slots, 0, S.rep);
      TK_LAUNCH_CHECK();
    }

    // ---- x <- x + d and the stopping decisions
    k_g_refine_update<<<nrl, kThreads, 0, st>>>(S.dd, S.rnd);
    TK_LAUNCH_CHECK();
    TK_CUDA(cudaMemcpyAsync(nrm_h.data(), S.nrm_all, sizeof(double) * nrm_h.size(), cudaMemcpyDeviceToHost, st));
    TK_CUDA(cudaStreamSynchronize(st));
    for (int p = 0; p < P; ++p) {
      std::vector<int> next;
      const double* hn = nrm_h.data() + (size_t)p * 3 * N;
      for (int q = 0; q < hcnt[p]; ++q) {
        const int l = act[p][q];
        tk_info& qi = g[p].inf[l];
        qi.refine_steps += 1;
        if (round > 0) qi.ne_norm = hn[3 * q];
        const double dn = hn[3 * q + 1], xn = hn[3 * q + 2];
        const bool done = refine_done(round, dn, prev_dn[p][l], xn, g[p].refine_tol);
        prev_dn[p][l] = dn;
        if (!done) next.push_back(l);
      }
      act[p].swap(next);
    }
  }
  return TK_OK;
}

}  // namespace tk
