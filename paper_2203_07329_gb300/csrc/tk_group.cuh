// Grouped solve of many independent overdetermined problems in the mixed
// form (internal).  After each problem's sketch and preconditioner are built,
// all problems advance together: every phase of an LSQR step (preconditioner
// apply, the product with A, the norms, the product with A^T, the v-step) and
// of a refinement pass (r = b - A x, A^T r - lambda x) is ONE launch over a
// tile or slot list that covers every problem, so the number of launches per
// step does not grow with the number of problems.
#pragma once

#include <vector>

#include "tk_internal.cuh"

namespace tk {

// The low-rank preconditioner's parts after the sketch (device pointers):
// the SVD fills sig and lrV; the ranks, S and the float32 copies follow.
struct LowRankParts {
  int64_t s = 0, c = 0;
  int N = 0;
  double alpha = 2.0;
  const double* lam = nullptr;
  double* sig = nullptr;
  double* sd = nullptr;
  int64_t* ranks = nullptr;
  double* lrV = nullptr;  // c x s
  double* lrS = nullptr;  // N x s
  float* lrV32 = nullptr;
  float* lrS32 = nullptr;
};

// One prepared problem (device pointers; the caller keeps them alive).
struct GroupProblem {
  int64_t m = 0, n = 0;
  const float* A32 = nullptr;  // float32 A for the LSQR products
  int64_t lda32 = 0;
  const void* Af = nullptr;  // A as given (float64 or float32), for the float64 passes
  int f64 = 0;
  int64_t ldaf = 0;
  const double* b = nullptr;
  const double* lam = nullptr;  // N lambdas (device)
  double* X = nullptr;          // N x n, zero on entry
  int lowrank = 0;
  const float* Mi = nullptr;  // Cholesky: R^-1, R^-T (N x np x np, float32)
  const float* Mti = nullptr;
  int64_t np = 0;
  const float* lrV = nullptr;  // low rank: V (n x lr_s), S (N x lr_s)
  const float* lrS = nullptr;
  int64_t lr_s = 0;
  double inner_tol = 1e-7;
  int maxiter = 500;
  int max_refine = 8;
  double refine_tol = 1e-11;
  int emulate = 0;  // the float64 refinement passes from exact digits on the tensor cores
  std::vector<int> ok_ids;  // lambdas that have a preconditioner
  tk_info* inf = nullptr;   // host, N entries
  // low rank, before the grouped SVD: the sketch Y (s x n) and its scratch
  LowRankParts lr_parts;
  const double* svd_Y = nullptr;
  void* svd_scratch = nullptr;
  size_t svd_bytes = 0;
};

// Largest n handled by the grouped engine (the vector of a slot is staged in
// shared memory by the preconditioner kernels).
constexpr int64_t kGroupMaxN = 4096;
constexpr int kGroupMaxLambda = 64;

size_t group_workspace(const std::vector<GroupProblem>& g, int N);
tk_status group_solve_mixed(std::vector<GroupProblem>& g, int N, void* work, size_t bytes, cudaStream_t st);

}  // namespace tk
