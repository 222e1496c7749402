// Sparse embedding (Section 2.1.1: "one nonzero element in each column"; the
// sparse subspace embedding of Theorem 3.5).  Column i of X (s x L) holds
// sign_i in row h_i, drawn from Philox stream 4 at index i:
//   h_i = floor(w0 s / 2^32),  sign_i = -1 if the low bit of w1 is set, else +1.
// Y = X A (A is L x cols, the long axis first) sums sign_i A[i] into row h_i.
//
// No atomics on the data: the rows are sorted by bucket with a stable radix
// sort (so each bucket lists its rows in ascending order), then one thread per
// (bucket, column) adds its rows in that order in float64 -- the same order of
// operations as the definition written out, so the float64 result does not
// depend on the schedule.  The sort moves 4-byte indices only; A is read
// once, each row as whole contiguous column blocks.
#include <algorithm>

#include "tk_internal.cuh"

namespace tk {
namespace {

constexpr int kRadixBits = 11;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kMaxTiles = 256;

__global__ void k_sparse_draw(uint64_t seed, int64_t L, int64_t s, int32_t* __restrict__ h,
                              int8_t* __restrict__ sign, int32_t* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox((uint64_t)i, STREAM_SPARSE, seed);
    h[i] = (int32_t)(((uint64_t)w.x * (uint64_t)s) >> 32);
    sign[i] = (w.y & 1u) ? (int8_t)-1 : (int8_t)1;
    idx[i] = (int32_t)i;
  }
}

// Per tile of `per` items: the histogram of the digit (key >> shift) & (R-1),
// stored digit-major (hist[d * tiles + tile]) so that one exclusive scan of
// the whole array gives every (digit, tile) its first output position.
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const int32_t* __restrict__ key, int64_t L, int64_t per,
                                                             int shift, int tiles, int32_t* __restrict__ hist) {
  __shared__ int32_t cnt[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) cnt[d] = 0;
  __syncthreads();
  const int64_t b = (int64_t)blockIdx.x * per, e = b + per < L ? b + per : L;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) atomicAdd(&cnt[(key[i] >> shift) & (kRadix - 1)], 1);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * tiles + blockIdx.x] = cnt[d];
}

// Exclusive scan of n ints in place, one CTA (n <= kRadix * kMaxTiles).
__global__ void __launch_bounds__(1024) k_scan_excl(int32_t* __restrict__ x, int64_t n) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t b = t * per, e = b + per < n ? b + per : n;
  int32_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += x[i];
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int32_t run = 0;
    for (int k = 0; k < (int)blockDim.x; ++k) {
      const int32_t v = part[k];
      part[k] = run;
      run += v;
    }
  }
  __syncthreads();
  int32_t run = part[t];
  for (int64_t i = b; i < e; ++i) {
    const int32_t v = x[i];
    x[i] = run;
    run += v;
  }
}

// Stable scatter of one radix pass: the tile's items go out in order, chunk by
// chunk of 256 and warp by warp inside a chunk; a warp ranks equal digits with
// __match_any_sync, and the per-digit running positions sit in shared memory.
__global__ void __launch_bounds__(kSortThreads)
    k_radix_scatter(const int32_t* __restrict__ key, const int32_t* __restrict__ val, int64_t L, int64_t per,
                    int shift, int tiles, const int32_t* __restrict__ offs, int32_t* __restrict__ key_out,
                    int32_t* __restrict__ val_out) {
  __shared__ int32_t pos[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) pos[d] = offs[(int64_t)d * tiles + blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * per, e = b + per < L ? b + per : L;
  for (int64_t c0 = b; c0 < e; c0 += blockDim.x) {
    const int64_t i = c0 + threadIdx.x;
    const bool valid = i < e;
    const int32_t k = valid ? key[i] : 0;
    const int d = (k >> shift) & (kRadix - 1);
    for (int w = 0; w < kSortWarps; ++w) {
      if (warp == w) {
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        if (valid) {
          const unsigned same = __match_any_sync(act, d);
          const int rank = __popc(same & ((1u << lane) - 1u));
          const int p = pos[d] + rank;
          key_out[p] = k;
          val_out[p] = val[i];
          __syncwarp(act);
          if (rank == 0) pos[d] += __popc(same);
        }
      }
      __syncthreads();
    }
  }
}

// start[k] = first position of bucket k in the sorted keys (k = 0..s; start[s] = L).
__global__ void k_bucket_starts(const int32_t* __restrict__ hs, int64_t L, int64_t s, int32_t* __restrict__ start) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= s; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = L;  // first index with hs >= k
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (hs[mid] < k) lo = mid + 1;
      else hi = mid;
    }
    start[k] = (int32_t)lo;
  }
}

// Y[k][c] = sum over the rows r of bucket k, in ascending order, of sign_r A[r][c]
// (float64).  Grid: (buckets, column blocks); a thread owns one column.
template <typename T>
__global__ void __launch_bounds__(256) k_sparse_apply(const T* __restrict__ A, int64_t ld, int64_t cols,
                                                      const int32_t* __restrict__ order,
                                                      const int32_t* __restrict__ start,
                                                      const int8_t* __restrict__ sign, double* __restrict__ Y) {
  const int64_t k = blockIdx.x;
  const int64_t c = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const int32_t b = start[k], e = start[k + 1];
  double acc = 0.0;
  // the rows in ascending order (the order of the definition).  Loading 8 rows' indices first and
  // then 8 independent rows was measured 3.4x slower (2.61 ms against 0.76 ms on 65536 x 2048,
  // s = 32768: about two rows per bucket)
  for (int32_t p = b; p < e; ++p) {
    const int32_t r = order[p];
    const double v = (double)A[(int64_t)r * ld + c];
    acc = acc + (sign[r] < 0 ? -v : v);
  }
  Y[k * cols + c] = acc;
}

int64_t sort_tile(int64_t L) {
  return std::max<int64_t>(4096, cdiv(L, kMaxTiles));
}

struct SparseBufs {
  int32_t *h, *idx, *h2, *idx2, *hist, *start;
  int8_t* sign;
};
void sparse_carve(Arena& a, int64_t L, int64_t s, SparseBufs& B) {
  const int tiles = (int)cdiv(L, sort_tile(L));
  B.h = a.take<int32_t>((size_t)L);
  B.idx = a.take<int32_t>((size_t)L);
  B.h2 = a.take<int32_t>((size_t)L);
  B.idx2 = a.take<int32_t>((size_t)L);
  B.hist = a.take<int32_t>((size_t)kRadix * tiles);
  B.start = a.take<int32_t>((size_t)s + 1);
  B.sign = a.take<int8_t>((size_t)L);
}

// Draws, then a stable LSD radix sort of the row indices by bucket (one pass of
// 11 bits per 11 bits of s - 1).  On return the sorted order is in B.idx
// (keys in B.h) and start[0..s] bounds each bucket.
tk_status sparse_sort(uint64_t seed, int64_t L, int64_t s, SparseBufs& B, cudaStream_t st) {
  const int64_t per = sort_tile(L);
  const int tiles = (int)cdiv(L, per);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(L, 256), 152 * 8));
  k_sparse_draw<<<grid, 256, 0, st>>>(seed, L, s, B.h, B.sign, B.idx);
  TK_LAUNCH_CHECK();
  int bits = 0;
  while ((int64_t(1) << bits) < s) ++bits;
  for (int shift = 0; shift < bits; shift += kRadixBits) {
    k_radix_hist<<<tiles, kSortThreads, 0, st>>>(B.h, L, per, shift, tiles, B.hist);
    k_scan_excl<<<1, 1024, 0, st>>>(B.hist, (int64_t)kRadix * tiles);
    k_radix_scatter<<<tiles, kSortThreads, 0, st>>>(B.h, B.idx, L, per, shift, tiles, B.hist, B.h2, B.idx2);
    TK_LAUNCH_CHECK();
    std::swap(B.h, B.h2);
    std::swap(B.idx, B.idx2);
  }
  k_bucket_starts<<<(unsigned)cdiv(s + 1, 256), 256, 0, st>>>(B.h, L, s, B.start);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

}  // namespace

size_t sparse_rows_workspace(int64_t L, int64_t cols, int64_t s) {
  (void)cols;
  Arena a;
  SparseBufs B;
  sparse_carve(a, L, s, B);
  return a.used + 1024;
}

tk_status sparse_rows(const void* A, tk_dtype dt, int64_t L, int64_t cols, int64_t ld, uint64_t seed, int64_t s,
                      double* Y, Arena& ar, cudaStream_t st) {
  if (s < 1 || s > kSparseMaxS || L > INT32_MAX) {
    set_error_msg("sparse embedding: need 1 <= s <= 2^22 and a long dimension below 2^31");
    return TK_EINVAL;
  }
  SparseBufs B;
  sparse_carve(ar, L, s, B);
  if (!ar.ok()) return TK_ENOMEM;
  if (cols == 0) return TK_OK;
  TK_TRY(sparse_sort(seed, L, s, B, st));
  if (cdiv(cols, 256) > 65535) {
    set_error_msg("sparse embedding: too many columns");
    return TK_EINVAL;
  }
  const dim3 grid((unsigned)s, (unsigned)cdiv(cols, 256));
  if (dt == TK_F64)
    k_sparse_apply<double><<<grid, 256, 0, st>>>((const double*)A, ld, cols, B.idx, B.start, B.sign, Y);
  else
    k_sparse_apply<float><<<grid, 256, 0, st>>>((const float*)A, ld, cols, B.idx, B.start, B.sign, Y);
  TK_LAUNCH_CHECK();
  return TK_OK;
}

tk_status sparse_draw_sorted(uint64_t seed, int64_t L, int64_t s, int32_t* h, int8_t* sign, int32_t* order,
                             int32_t* start, Arena& ar, cudaStream_t st) {
  if (s < 1 || s > kSparseMaxS || L < 1 || L > INT32_MAX) {
    set_error_msg("sparse embedding: need 1 <= s <= 2^22 and 1 <= L < 2^31");
    return TK_EINVAL;
  }
  SparseBufs B;
  sparse_carve(ar, L, s, B);
  if (!ar.ok()) return TK_ENOMEM;
  TK_TRY(sparse_sort(seed, L, s, B, st));
  // the draws in row order: h was permuted by the sort, so draw them again for the caller
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(L, 256), 152 * 8));
  if (h) {
    k_sparse_draw<<<grid, 256, 0, st>>>(seed, L, s, h, sign ? sign : B.sign, B.idx2);
    TK_LAUNCH_CHECK();
  } else if (sign) {
    TK_CUDA(cudaMemcpyAsync(sign, B.sign, (size_t)L, cudaMemcpyDeviceToDevice, st));
  }
  if (order) TK_CUDA(cudaMemcpyAsync(order, B.idx, sizeof(int32_t) * (size_t)L, cudaMemcpyDeviceToDevice, st));
  if (start) TK_CUDA(cudaMemcpyAsync(start, B.start, sizeof(int32_t) * (size_t)(s + 1), cudaMemcpyDeviceToDevice, st));
  return TK_OK;
}

}  // namespace tk
