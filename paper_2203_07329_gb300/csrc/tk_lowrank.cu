// Low-rank preconditioner of Section 3.1 / Algorithm 3.
//
//  * [~, Sigma, V] = svd(Y, 'econ') (step 4) by one-sided Jacobi on the rows
//    of Y (the columns of Y^T), so no Gram matrix is ever formed.  Rows are
//    paired by the round-robin (circle) schedule: each launch rotates s/2
//    disjoint pairs, s-1 launches make a sweep; sweeps repeat until no pair
//    is rotated.
//  * sd_i = sum_j 1/(1 + lambda_i/sigma_j^2) (Section 3.1.2) and the ranks
//    s_i = min(s, ceil(alpha ceil(sd_i))) (step 5), in float64 with the sum
//    taken in ascending j and no contraction, so equal sigma give equal ranks
//    on any IEEE machine.
//  * S_i = diag(1 - sqrt(1/(1 + sigma_j^2/lambda_i))) (step 7) and the apply
//    R_i^-1 x = lambda_i^{-1/2} (x - V_i S_i V_i^T x) (eq. for R^-1, step 8).
#include <algorithm>
#include <numeric>
#include <vector>

#include "tk_lsqr.cuh"

namespace tk {
namespace {

constexpr int kJacThreads = 256;

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// Pair k of round `round` of the circle schedule over sp (even) players
// (player sp-1 is a dummy when s is odd): rows p < q of W are rotated so that
// they become orthogonal, unless already orthogonal to tol.  One warp per
// pair; the squared row norms a = nrm2[p], b = nrm2[q] are carried from the
// start of the sweep and updated by the rotation (a' = a - t g, b' = b + t g),
// so only g = w_p . w_q is computed per pair.
__device__ __forceinline__ void jacobi_pair_warp(double* __restrict__ W, double* __restrict__ nrm2, int64_t s,
                                                 int64_t n, int64_t sp, int64_t round, int64_t k, double tol,
                                                 double* __restrict__ off_max, int* __restrict__ rotated) {
  const int lane = threadIdx.x & 31;
  int64_t p, q;
  if (k == 0) {
    p = sp - 1;
    q = round;
  } else {
    p = (round + k) % (sp - 1);
    q = (round - k + (sp - 1)) % (sp - 1);
  }
  if (p > q) {
    int64_t t = p;
    p = q;
    q = t;
  }
  if (q >= s) return;  // pair with the dummy
  double* wp = W + p * n;
  double* wq = W + q * n;
  double g = 0.0;
  for (int64_t i = lane; i < n; i += 32) g = fma(wp[i], wq[i], g);
  g = warp_sum(g);
  const double a = nrm2[p], b = nrm2[q];
  if (a == 0.0 || b == 0.0) return;
  const double rel = fabs(g) / sqrt(a * b);
  if (!(rel > tol)) return;
  const double zeta = (b - a) / (2.0 * g);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t);
  const double sn = c * t;
  for (int64_t i = lane; i < n; i += 32) {
    const double x = wp[i], y = wq[i];
    wp[i] = c * x - sn * y;
    wq[i] = sn * x + c * y;
  }
  if (lane == 0) {
    nrm2[p] = a - t * g;
    nrm2[q] = b + t * g;
    atomic_max_pos(off_max, rel);
    atomicAdd(rotated, 1);
  }
}

constexpr int kPairsPerCta = kJacThreads / 32;

// One round for one matrix: sp/2 disjoint pairs, one warp each.
__global__ void __launch_bounds__(kJacThreads)
    k_jacobi_round(double* __restrict__ W, double* __restrict__ nrm2, int64_t s, int64_t n, int64_t sp, int64_t round,
                   double tol, double* __restrict__ off_max, int* __restrict__ rotated) {
  const int64_t k = (int64_t)blockIdx.x * kPairsPerCta + (threadIdx.x >> 5);
  if (k < sp / 2) jacobi_pair_warp(W, nrm2, s, n, sp, round, k, tol, off_max, rotated);
}

// Squared row norms at the start of a sweep (one warp per row).
__global__ void __launch_bounds__(kJacThreads)
    k_row_norms2(const double* __restrict__ W, int64_t s, int64_t n, double* __restrict__ nrm2) {
  const int64_t r = (int64_t)blockIdx.x * kPairsPerCta + (threadIdx.x >> 5);
  if (r >= s) return;
  const int lane = threadIdx.x & 31;
  double a = 0.0;
  for (int64_t i = lane; i < n; i += 32) a = fma(W[r * n + i], W[r * n + i], a);
  a = warp_sum(a);
  if (lane == 0) nrm2[r] = a;
}

// One round for many matrices (grouped batch): CTA = (matrix, 8 pairs).
struct SvdDesc {
  double* W;
  double* nrm2;
  int64_t s, n, sp;
  double* off_max;
  int* rotated;
  int done;
};
struct SvdTile {
  int job, k0;
};
__global__ void __launch_bounds__(kJacThreads)
    k_jacobi_round_grouped(const SvdDesc* __restrict__ D, const SvdTile* __restrict__ tl, int64_t round, double tol) {
  const SvdTile t = tl[blockIdx.x];
  const SvdDesc& d = D[t.job];
  const int64_t k = t.k0 + (threadIdx.x >> 5);
  if (d.done || round >= d.sp - 1 || k >= d.sp / 2) return;
  jacobi_pair_warp(d.W, d.nrm2, d.s, d.n, d.sp, round, k, tol, d.off_max, d.rotated);
}

// Squared row norms of every matrix still rotating (CTA = (matrix, 8 rows)).
__global__ void __launch_bounds__(kJacThreads)
    k_row_norms2_grouped(const SvdDesc* __restrict__ D, const SvdTile* __restrict__ tl) {
  const SvdTile t = tl[blockIdx.x];
  const SvdDesc& d = D[t.job];
  const int64_t r = t.k0 + (threadIdx.x >> 5);
  if (d.done || r >= d.s) return;
  const int lane = threadIdx.x & 31;
  double a = 0.0;
  for (int64_t i = lane; i < d.n; i += 32) a = fma(d.W[r * d.n + i], d.W[r * d.n + i], a);
  a = warp_sum(a);
  if (lane == 0) d.nrm2[r] = a;
}

__global__ void k_svd_reset(SvdDesc* __restrict__ D, int J) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < J && !D[j].done) {
    *D[j].rotated = 0;
    *D[j].off_max = 0.0;
  }
}

__global__ void k_row_norms(const double* __restrict__ W, int64_t n, double* __restrict__ nrm) {
  __shared__ double sh[32];
  const int64_t p = blockIdx.x;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a = fma(W[p * n + i], W[p * n + i], a);
  a = block_sum(a, sh);
  if (threadIdx.x == 0) nrm[p] = sqrt(a);
}

// V[k*s + j] = W[perm[j]][k] / sigma_j ; sigma[j] = nrm[perm[j]]
__global__ void k_write_v(const double* __restrict__ W, const double* __restrict__ nrm, const int* __restrict__ perm,
                          int64_t s, int64_t n, double* __restrict__ V, double* __restrict__ sigma) {
  const int64_t j = blockIdx.y;
  const int p = perm[j];
  const double sg = nrm[p];
  const double inv = sg > 0.0 ? 1.0 / sg : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) sigma[j] = sg;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    V[k * s + j] = W[(int64_t)p * n + k] * inv;
}

// sd_i and s_i for each lambda (one thread per lambda; sum in ascending j).
__global__ void k_ranks(const double* __restrict__ sigma, int64_t s, const double* __restrict__ lam, int N,
                        double alpha, double* __restrict__ sd_out, int64_t* __restrict__ rank_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double l = lam[i];
  double acc = 0.0;
  for (int64_t j = 0; j < s; ++j) {
    double sg = sigma[j];
    if (sg > 0.0) acc = __dadd_rn(acc, __ddiv_rn(1.0, __dadd_rn(1.0, __ddiv_rn(l, __dmul_rn(sg, sg)))));
  }
  double t = ceil(__dmul_rn(alpha, ceil(acc)));
  int64_t r = (t > (double)s) ? s : (t < 1.0 ? 1 : (int64_t)t);
  if (sd_out) sd_out[i] = acc;
  rank_out[i] = r;
}

// S[l][j] = 1 - sqrt(1/(1 + sigma_j^2/lambda_l)) for j < rank_l, else 0.
template <typename T>
__global__ void k_lr_diag(const double* __restrict__ sigma, int64_t s, const double* __restrict__ lam,
                          const int64_t* __restrict__ rank, T* __restrict__ S) {
  const int l = blockIdx.y;
  const double lv = lam[l];
  const int64_t r = rank[l];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < s; j += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (j < r) v = 1.0 - sqrt(1.0 / (1.0 + sigma[j] * sigma[j] / lv));
    S[(int64_t)l * s + j] = (T)v;
  }
}

// tmp[k][j] *= S[l_k][j] / sqrt(lambda_l);  invs[k] = 1/sqrt(lambda_l)
template <typename T>
__global__ void k_lr_scale(T* __restrict__ tmp, int64_t s, const T* __restrict__ S, const int* __restrict__ lam_idx,
                           const double* __restrict__ lam, double* __restrict__ invs) {
  const int k = blockIdx.y;
  const int l = lam_idx[k];
  const double is = 1.0 / sqrt(lam[l]);
  if (blockIdx.x == 0 && threadIdx.x == 0) invs[k] = is;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < s; j += (int64_t)gridDim.x * blockDim.x)
    tmp[(int64_t)k * s + j] = (T)((double)tmp[(int64_t)k * s + j] * (double)S[(int64_t)l * s + j] * is);
}

}  // namespace

size_t svd_workspace(int64_t s, int64_t n) {
  Arena a;
  a.take<double>((size_t)s * n);
  a.take<double>((size_t)s);
  a.take<int>((size_t)s);
  a.take<double>(1);
  a.take<int>(1);
  a.take<double>((size_t)s);  // squared row norms carried through a sweep
  return a.used + 512;
}

// The sorted singular values and right singular vectors from the rotated
// rows: sigma_j = ||W_perm[j]||, V[:, j] = W_perm[j] / sigma_j.
static tk_status svd_finish(const double* W, int64_t s, int64_t n, double* nrm, int* perm, double* sigma, double* V,
                            cudaStream_t st) {
  k_row_norms<<<(unsigned)s, 256, 0, st>>>(W, n, nrm);
  TK_LAUNCH_CHECK();
  std::vector<double> h(s);
  TK_CUDA(cudaMemcpyAsync(h.data(), nrm, sizeof(double) * s, cudaMemcpyDeviceToHost, st));
  TK_CUDA(cudaStreamSynchronize(st));
  std::vector<int> order(s);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h[a] > h[b]; });
  TK_CUDA(cudaMemcpyAsync(perm, order.data(), sizeof(int) * s, cudaMemcpyHostToDevice, st));
  dim3 g((unsigned)std::min<int64_t>(cdiv(n, 256), 64), (unsigned)s);
  k_write_v<<<g, 256, 0, st>>>(W, nrm, perm, s, n, V, sigma);
  TK_LAUNCH_CHECK();
  TK_CUDA(cudaStreamSynchronize(st));  // `order` is a host temporary
  return TK_OK;
}

tk_status jacobi_svd(const double* Y, int64_t s, int64_t n, double* sigma, double* V, int* sweeps_host, Arena& ar,
                     cudaStream_t st) {
  double* W = ar.take<double>((size_t)s * n);
  double* nrm = ar.take<double>((size_t)s);
  int* perm = ar.take<int>((size_t)s);
  double* off_max = ar.take<double>(1);
  int* rotated = ar.take<int>(1);
  double* nrm2 = ar.take<double>((size_t)s);
  if (!ar.ok()) return TK_ENOMEM;
  if (s == 0) return TK_OK;
  TK_CUDA(cudaMemcpyAsync(W, Y, sizeof(double) * (size_t)s * n, cudaMemcpyDeviceToDevice, st));
  const int64_t sp = (s % 2 == 0) ? s : s + 1;
  const double tol = 1e-15;
  int sweep = 0;
  const int max_sweeps = 80;
  for (; sweep < max_sweeps && s > 1; ++sweep) {
    TK_CUDA(cudaMemsetAsync(rotated, 0, sizeof(int), st));
    TK_CUDA(cudaMemsetAsync(off_max, 0, sizeof(double), st));
    k_row_norms2<<<(unsigned)cdiv(s, kPairsPerCta), kJacThreads, 0, st>>>(W, s, n, nrm2);
    TK_LAUNCH_CHECK();
    for (int64_t r = 0; r < sp - 1; ++r) {
      k_jacobi_round<<<(unsigned)cdiv(sp / 2, kPairsPerCta), kJacThreads, 0, st>>>(W, nrm2, s, n, sp, r, tol,
                                                                                    off_max, rotated);
      TK_LAUNCH_CHECK();
    }
    int hrot = 0;
    TK_CUDA(cudaMemcpyAsync(&hrot, rotated, sizeof(int), cudaMemcpyDeviceToHost, st));
    TK_CUDA(cudaStreamSynchronize(st));
    if (hrot == 0) break;
  }
  if (sweeps_host) *sweeps_host = sweep + 1;
  return svd_finish(W, s, n, nrm, perm, sigma, V, st);
}

tk_status jacobi_svd_grouped(std::vector<SvdJob>& jobs, void* work, size_t work_bytes, cudaStream_t st) {
  const int J = (int)jobs.size();
  if (J == 0) return TK_OK;
  std::vector<SvdDesc> hd(J);
  std::vector<SvdTile> tiles;
  Arena a;
  a.base = (char*)work;
  a.cap = work_bytes;
  SvdDesc* dd = a.take<SvdDesc>(J);
  double* offs = a.take<double>(J);
  int* rots = a.take<int>(J);
  size_t ntiles = 0;
  for (const auto& j : jobs) ntiles += (size_t)cdiv(std::max<int64_t>(((j.s % 2 == 0) ? j.s : j.s + 1) / 2, j.s),
                                                    kPairsPerCta);
  SvdTile* dt = a.take<SvdTile>(std::max<size_t>(ntiles, 1));
  if (!a.ok()) {
    set_error_msg("grouped SVD: workspace too small");
    return TK_ENOMEM;
  }
  int64_t max_rounds = 0;
  for (int j = 0; j < J; ++j) {
    SvdJob& q = jobs[j];
    Arena sa;
    sa.base = (char*)q.scratch;
    sa.cap = q.scratch_bytes;
    q.W = sa.take<double>((size_t)q.s * q.n);
    q.nrm = sa.take<double>((size_t)q.s);
    q.perm = sa.take<int>((size_t)q.s);
    sa.take<double>(1);
    sa.take<int>(1);
    double* nrm2 = sa.take<double>((size_t)q.s);
    if (!sa.ok()) return TK_ENOMEM;
    if (q.s > 0) TK_CUDA(cudaMemcpyAsync(q.W, q.Y, sizeof(double) * (size_t)q.s * q.n, cudaMemcpyDeviceToDevice, st));
    const int64_t sp = (q.s % 2 == 0) ? q.s : q.s + 1;
    hd[j] = SvdDesc{q.W, nrm2, q.s, q.n, sp, offs + j, rots + j, q.s <= 1 ? 1 : 0};
    for (int64_t k = 0; k < std::max<int64_t>(sp / 2, q.s); k += kPairsPerCta) tiles.push_back(SvdTile{j, (int)k});
    if (q.s > 1) max_rounds = std::max(max_rounds, sp - 1);
    q.sweeps = 0;
  }
  TK_CUDA(cudaMemcpyAsync(dd, hd.data(), sizeof(SvdDesc) * J, cudaMemcpyHostToDevice, st));
  TK_CUDA(cudaMemcpyAsync(dt, tiles.data(), sizeof(SvdTile) * tiles.size(), cudaMemcpyHostToDevice, st));
  const double tol = 1e-15;  // the single-matrix SVD's threshold
  const int max_sweeps = 80;
  std::vector<int> hrot(J);
  for (int sweep = 0; sweep < max_sweeps && max_rounds > 0; ++sweep) {
    k_svd_reset<<<cdiv(J, 128), 128, 0, st>>>(dd, J);
    TK_LAUNCH_CHECK();
    k_row_norms2_grouped<<<(unsigned)tiles.size(), kJacThreads, 0, st>>>(dd, dt);
    TK_LAUNCH_CHECK();
    for (int64_t r = 0; r < max_rounds; ++r) {
      k_jacobi_round_grouped<<<(unsigned)tiles.size(), kJacThreads, 0, st>>>(dd, dt, r, tol);
      TK_LAUNCH_CHECK();
    }
    TK_CUDA(cudaMemcpyAsync(hrot.data(), rots, sizeof(int) * J, cudaMemcpyDeviceToHost, st));
    TK_CUDA(cudaStreamSynchronize(st));
    max_rounds = 0;
    for (int j = 0; j < J; ++j) {
      if (hd[j].done) continue;
      jobs[j].sweeps = sweep + 1;
      if (hrot[j] == 0) hd[j].done = 1;
      else max_rounds = std::max(max_rounds, hd[j].sp - 1);
    }
    if (max_rounds == 0) break;
    TK_CUDA(cudaMemcpyAsync(dd, hd.data(), sizeof(SvdDesc) * J, cudaMemcpyHostToDevice, st));
  }
  for (auto& q : jobs)
    if (q.s > 0) TK_TRY(svd_finish(q.W, q.s, q.n, q.nrm, q.perm, q.sigma, q.V, st));
  TK_CUDA(cudaStreamSynchronize(st));  // hd, tiles are host temporaries
  return TK_OK;
}

size_t svd_grouped_workspace(const std::vector<SvdJob>& jobs) {
  Arena a;
  size_t ntiles = 0;
  for (const auto& j : jobs) ntiles += (size_t)cdiv(std::max<int64_t>(((j.s % 2 == 0) ? j.s : j.s + 1) / 2, j.s),
                                                    kPairsPerCta);
  a.take<SvdDesc>(std::max<size_t>(jobs.size(), 1));
  a.take<double>(std::max<size_t>(jobs.size(), 1));
  a.take<int>(std::max<size_t>(jobs.size(), 1));
  a.take<SvdTile>(std::max<size_t>(ntiles, 1));
  return a.used + 1024;
}

tk_status lowrank_ranks_dev(const double* sigma, int64_t s, const double* lam_dev, int N, double alpha,
                            double* sd_dev, int64_t* rank_dev, cudaStream_t st) {
  if (N <= 0) return TK_OK;
  k_ranks<<<cdiv(N, 128), 128, 0, st>>>(sigma, s, lam_dev, N, alpha, sd_dev, rank_dev);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

template <typename T>
tk_status lowrank_diag_dev(const double* sigma, int64_t s, const double* lam_dev, const int64_t* rank_dev, int N,
                           T* S, cudaStream_t st) {
  if (N <= 0 || s <= 0) return TK_OK;
  dim3 g((unsigned)std::min<int64_t>(cdiv(s, 256), 64), (unsigned)N);
  k_lr_diag<T><<<g, 256, 0, st>>>(sigma, s, lam_dev, rank_dev, S);
  TK_LAUNCH_CHECK();
  return TK_OK;
}
template tk_status lowrank_diag_dev<double>(const double*, int64_t, const double*, const int64_t*, int, double*,
                                            cudaStream_t);
template tk_status lowrank_diag_dev<float>(const double*, int64_t, const double*, const int64_t*, int, float*,
                                           cudaStream_t);

template <typename T>
tk_status lr_apply(int count, int64_t n, int64_t s, const T* V, const T* S, const int* lam_idx,
                   const double* lam_dev, const T* in, T* out, T* tmp, double* invs, cudaStream_t st) {
  if (count <= 0) return TK_OK;
  // tmp = in V  (count x s)
  TK_TRY((gemm<T, T, T>(false, false, count, s, n, in, n, V, s, tmp, s, 1.0, nullptr, nullptr, 0, st)));
  dim3 g((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(s, 256), 64)), (unsigned)count);
  k_lr_scale<T><<<g, 256, 0, st>>>(tmp, s, S, lam_idx, lam_dev, invs);
  TK_LAUNCH_CHECK();
  // out = -tmp V^T + invs * in
  TK_TRY((gemm<T, T, T>(false, true, count, n, s, tmp, s, V, s, out, n, -1.0, invs, in, n, st)));
  return TK_OK;
}
template tk_status lr_apply<double>(int, int64_t, int64_t, const double*, const double*, const int*, const double*,
                                    const double*, double*, double*, double*, cudaStream_t);
template tk_status lr_apply<float>(int, int64_t, int64_t, const float*, const float*, const int*, const double*,
                                   const float*, float*, float*, double*, cudaStream_t);

}  // namespace tk
