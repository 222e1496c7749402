// Handle calls of the C ABI: a stream plus a library-owned workspace that
// grows to the largest size a solve on the handle has needed (tk_create,
// tk_destroy, tk_handle_solve, tk_handle_solve_batched).  They sequence
// nothing themselves: each solve forwards to tk_solve / tk_solve_batched with
// the handle's stream and workspace.
#include <mutex>

#include "tk_internal.cuh"

struct tk_handle {
  cudaStream_t stream = nullptr;
  int device = 0;
  void* work = nullptr;
  size_t bytes = 0;
  std::mutex mu;  // one solve at a time per handle (the workspace is shared)
};

namespace tk {
namespace {
// Make the workspace at least `need` bytes: the only allocation on this path,
// done when a larger problem than any before arrives (the stream is drained
// first, since a solve in flight may still use the old buffer).
tk_status grow(tk_handle* h, size_t need) {
  if (need <= h->bytes) return TK_OK;
  TK_CUDA(cudaStreamSynchronize(h->stream));
  if (h->work) TK_CUDA(cudaFree(h->work));
  h->work = nullptr;
  h->bytes = 0;
  const size_t rounded = (need + (size_t(1) << 20) - 1) & ~((size_t(1) << 20) - 1);
  const cudaError_t e = cudaMalloc(&h->work, rounded);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    set_error_msg("tk_handle: cudaMalloc of the workspace failed (device memory exhausted?)");
    return TK_ENOMEM;
  }
  h->bytes = rounded;
  return TK_OK;
}
}  // namespace
}  // namespace tk

using namespace tk;

extern "C" {

TK_API tk_status tk_create(tk_handle** out, void* stream) {
  if (!out) {
    set_error_msg("tk_create: handle pointer is NULL");
    return TK_EINVAL;
  }
  *out = nullptr;
  tk_handle* h = new tk_handle;
  h->stream = (cudaStream_t)stream;
  const cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    set_error(e, __FILE__, __LINE__);
    return TK_ECUDA;
  }
  *out = h;
  return TK_OK;
}

TK_API tk_status tk_destroy(tk_handle* h) {
  if (!h) return TK_OK;
  tk_status st = TK_OK;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && h->work) e = cudaFree(h->work);
    if (e != cudaSuccess) {
      set_error(e, __FILE__, __LINE__);
      st = TK_ECUDA;
    }
    cudaSetDevice(cur);
  }
  delete h;
  return st;
}

TK_API size_t tk_handle_workspace_bytes(const tk_handle* h) { return h ? h->bytes : 0; }

TK_API tk_status tk_handle_solve(tk_handle* h, const tk_problem* p, const double* lambdas, int N, const tk_opts* o,
                                 double* X, tk_info* info) {
  if (!h) {
    set_error_msg("tk_handle_solve: handle is NULL");
    return TK_EINVAL;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  TK_CUDA(cudaSetDevice(h->device));
  size_t need = 0;
  TK_TRY(tk_workspace_size(p, N, o, &need));
  TK_TRY(grow(h, need));
  return tk_solve(p, lambdas, N, o, h->work, h->bytes, h->stream, X, info);
}

TK_API tk_status tk_handle_solve_batched(tk_handle* h, const tk_problem* ps, int P, const double* lambdas, int N,
                                         const tk_opts* o, int n_opts, double* const* X, tk_info* info) {
  if (!h) {
    set_error_msg("tk_handle_solve_batched: handle is NULL");
    return TK_EINVAL;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  TK_CUDA(cudaSetDevice(h->device));
  size_t need = 0;
  TK_TRY(tk_workspace_size_batched(ps, P, N, o, n_opts, &need));
  TK_TRY(grow(h, need));
  return tk_solve_batched(ps, P, lambdas, N, o, n_opts, h->work, h->bytes, h->stream, X, info);
}

}  // extern "C"
