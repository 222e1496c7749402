// Integer draws of the SRHT embedding (Section 2.1.1): the random signs of D
// and the random row subset of S.
//
// The subset is "the s smallest (key, row) pairs" of 64-bit Philox keys.  On
// the GPU that is a radix select of the s-th smallest key (eight 8-bit
// digit passes) followed by an order-preserving compaction, so the selected
// rows come out ascending with no sort.
#include <mutex>

#include "tk_internal.cuh"

namespace tk {

// Scratch of tk_sketch_draw_static: the 64-bit sampling keys plus the two
// words of the radix select, for at most TK_DRAW_STATIC_MAX_MP rows.  Every
// device that loads the library holds this array (8 MiB + 16 B) until exit.
static __device__ __align__(256) uint64_t g_draw_scratch[TK_DRAW_STATIC_MAX_MP + 2];

namespace {

__global__ void k_signs_keys(uint64_t seed, int64_t mp, int8_t* __restrict__ signs, uint64_t* __restrict__ keys) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mp; i += stride) {
    if (signs) {
      uint4 w = philox((uint64_t)i, STREAM_SIGNS, seed);
      signs[i] = (w.x & 1u) ? (int8_t)-1 : (int8_t)1;
    }
    if (keys) {
      uint4 w = philox((uint64_t)i, STREAM_KEYS, seed);
      keys[i] = ((uint64_t)w.x << 32) | (uint64_t)w.y;
    }
  }
}

constexpr int kSelThreads = 1024;

// One CTA.  Finds T = the s-th smallest key and how many keys equal to T
// belong to the subset (the lowest-index ones, which realizes the (key, row)
// tie-break).  sel[0] = T, sel[1] = number of T-keys taken.  1 <= s <= mp.
__global__ void __launch_bounds__(kSelThreads) k_radix_select(const uint64_t* __restrict__ keys, int64_t mp,
                                                              int64_t s, uint64_t* __restrict__ sel) {
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long s_prefix, s_mask;
  __shared__ long long s_rank;
  if (threadIdx.x == 0) {
    s_prefix = 0ull;
    s_mask = 0ull;
    s_rank = (long long)s;
  }
  for (int digit = 7; digit >= 0; --digit) {
    for (int v = threadIdx.x; v < 256; v += blockDim.x) hist[v] = 0u;
    __syncthreads();
    const unsigned long long prefix = s_prefix, mask = s_mask;
    const int shift = 8 * digit;
    for (int64_t i = threadIdx.x; i < mp; i += blockDim.x) {
      unsigned long long k = keys[i];
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255ull], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long cum = 0, rank = s_rank;
      for (int v = 0; v < 256; ++v) {
        long long h = hist[v];
        if (cum + h >= rank) {
          s_prefix = prefix | ((unsigned long long)v << shift);
          s_mask = mask | (255ull << shift);
          s_rank = rank - cum;
          break;
        }
        cum += h;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sel[0] = s_prefix;
    sel[1] = (uint64_t)s_rank;
  }
}

// Exclusive scan over a 1024-thread block; returns the prefix, writes the total.
__device__ int block_exclusive_scan(int v, int* sh_warp, int* total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int t = sh_warp[lane];
    int u = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, u, o);
      if (lane >= o) u += y;
    }
    sh_warp[lane] = u - t;  // exclusive prefix of warp totals
    if (lane == 31) sh_warp[32] = u;
  }
  __syncthreads();
  int r = sh_warp[wid] + x - v;
  *total = sh_warp[32];
  __syncthreads();
  return r;
}

// One CTA: rows[] = selected indices ascending; rowmap[i] = position or -1.
__global__ void __launch_bounds__(kSelThreads) k_compact(const uint64_t* __restrict__ keys, int64_t mp, int64_t s,
                                                         const uint64_t* __restrict__ sel, int64_t* __restrict__ rows,
                                                         int32_t* __restrict__ rowmap) {
  __shared__ int sh[33];
  const uint64_t T = sel[0];
  const long long take = (long long)sel[1];
  long long run_sel = 0, run_eq = 0;
  for (int64_t c = 0; c < mp; c += blockDim.x) {
    int64_t i = c + threadIdx.x;
    bool in = i < mp;
    uint64_t k = in ? keys[i] : 0ull;
    int lt = (in && k < T) ? 1 : 0;
    int eq = (in && k == T) ? 1 : 0;
    int eq_tot;
    int eq_pos = block_exclusive_scan(eq, sh, &eq_tot);
    int take_it = lt | ((eq && (run_eq + eq_pos) < take) ? 1 : 0);
    int sel_tot;
    int pos = block_exclusive_scan(take_it, sh, &sel_tot);
    if (in) {
      long long p = run_sel + pos;
      bool keep = take_it && p < s;  // exactly s are selected; the bound only guards the writes
      if (keep && rows) rows[p] = i;
      if (rowmap) rowmap[i] = keep ? (int32_t)p : -1;
    }
    run_eq += eq_tot;
    run_sel += sel_tot;
  }
}

}  // namespace

size_t draw_workspace(int64_t mp) {
  Arena a;
  a.take<uint64_t>((size_t)mp);
  a.take<uint64_t>(2);
  return a.used + 256;
}

tk_status draw_signs_rows(uint64_t seed, int64_t mp, int64_t s, int8_t* signs, int64_t* rows, int32_t* rowmap,
                          Arena& ar, cudaStream_t st) {
  bool need_rows = (rows || rowmap) && s > 0;
  uint64_t* keys = need_rows ? ar.take<uint64_t>((size_t)mp) : nullptr;
  uint64_t* sel = need_rows ? ar.take<uint64_t>(2) : nullptr;
  if (!ar.ok()) return TK_ENOMEM;
  if (mp <= 0) return TK_OK;
  int blocks = (int)std::min<int64_t>(cdiv(mp, 256), 152 * 16);
  if (signs || need_rows) {
    k_signs_keys<<<blocks, 256, 0, st>>>(seed, mp, signs, keys);
    TK_LAUNCH_CHECK();
  }
  if (need_rows) {
    k_radix_select<<<1, kSelThreads, 0, st>>>(keys, mp, s, sel);
    TK_LAUNCH_CHECK();
    k_compact<<<1, kSelThreads, 0, st>>>(keys, mp, s, sel, rows, rowmap);
    TK_LAUNCH_CHECK();
  } else if (rowmap) {
    TK_CUDA(cudaMemsetAsync(rowmap, 0xff, sizeof(int32_t) * (size_t)mp, st));  // s == 0: nothing sampled
  }
  return TK_OK;
}

// Device address of g_draw_scratch on the current device, looked up once per
// device (host code only sees a host-side stand-in under that name).
static tk_status static_scratch(uint64_t** out) {
  static std::mutex mu;
  static uint64_t* addr[64] = {nullptr};
  int dev = 0;
  TK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error_msg("tk_sketch_draw_static: device index out of range");
    return TK_EINVAL;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    TK_CUDA(cudaGetSymbolAddress(&p, g_draw_scratch));
    addr[dev] = static_cast<uint64_t*>(p);
  }
  *out = addr[dev];
  return TK_OK;
}

}  // namespace tk

extern "C" TK_API tk_status tk_sketch_draw_static(uint64_t seed, int64_t mp, int64_t s, int8_t* signs, int64_t* rows,
                                                  void* stream) {
  using namespace tk;
  if (mp < 1 || mp > TK_DRAW_STATIC_MAX_MP) {
    set_error_msg("tk_sketch_draw_static: mp must be in [1, TK_DRAW_STATIC_MAX_MP]; use tk_sketch_draw with a "
                  "caller workspace for longer draws");
    return TK_EINVAL;
  }
  if (s < 0 || s > mp) {
    set_error_msg("tk_sketch_draw_static: s out of range");
    return TK_EINVAL;
  }
  uint64_t* scratch = nullptr;
  TK_TRY(static_scratch(&scratch));
  // Same kernels as tk_sketch_draw; the keys and select words live in the static
  // array.  Every word read is written earlier in the same call (keys[0, mp) by
  // the draw kernel, the select words by the radix select), so the contents a
  // previous call left behind are never read and nothing needs clearing.
  Arena a;
  a.base = reinterpret_cast<char*>(scratch);
  a.cap = sizeof(uint64_t) * (size_t)(TK_DRAW_STATIC_MAX_MP + 2);
  cudaStream_t st = (cudaStream_t)stream;
  TK_TRY(draw_signs_rows(seed, mp, s, signs, rows, nullptr, a, st));
  TK_CUDA(cudaStreamSynchronize(st));
  return TK_OK;
}
