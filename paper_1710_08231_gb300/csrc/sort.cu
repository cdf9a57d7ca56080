// sort.cu -- device-wide stable LSD radix sort of (uint64 key, uint64 value) pairs.
//
// Each pass handles 8 key bits with three kernels: per-tile digit histograms (digit-major), an
// exclusive scan of the histograms, and a stable scatter in which every tile ranks its items per
// digit in order (warp match + per-warp counts). Used where many independent rows must be sorted at
// once (the contraction of very large clusters).
#include <algorithm>

#include "sort.cuh"

namespace gp {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int64_t kSortTile = (int64_t)kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const unsigned long long *keys, int64_t n, int shift,
                                                             int64_t ntiles, int64_t *hist) {
  __shared__ unsigned h[256];
  for (int t = threadIdx.x; t < 256; t += kSortThreads) h[t] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int k = 0; k < kSortItems; k++) {
    const int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += kSortThreads) hist[(int64_t)t * ntiles + blockIdx.x] = h[t];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const unsigned long long *kin,
                                                                const unsigned long long *vin,
                                                                unsigned long long *kout, unsigned long long *vout,
                                                                int64_t n, int shift, int64_t ntiles,
                                                                const int64_t *offs) {
  __shared__ int64_t base[256];
  __shared__ unsigned wcnt[kSortThreads / 32][256];
  const int wid = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < 256; t += kSortThreads) base[t] = offs[(int64_t)t * ntiles + blockIdx.x];
  __syncthreads();
  const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
  for (int k = 0; k < kSortItems; k++) {
    const int64_t i = tbase + (int64_t)k * kSortThreads + threadIdx.x;
    const bool valid = i < n;
    const unsigned long long key = valid ? kin[i] : 0;
    const unsigned long long val = valid ? vin[i] : 0;
    const int dg = valid ? (int)((key >> shift) & 255) : 256;
    for (int t = threadIdx.x; t < (kSortThreads / 32) * 256; t += kSortThreads) wcnt[t >> 8][t & 255] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(kFull, dg);
    const int rank = __popc(peers & lanemask_lt());
    if (valid && rank == 0) wcnt[wid][dg] = __popc(peers);
    __syncthreads();
    if (valid) {
      int64_t pos = base[dg] + rank;
      for (int w = 0; w < wid; w++) pos += wcnt[w][dg];
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    if (threadIdx.x < 256) {
      unsigned s = 0;
      for (int w = 0; w < kSortThreads / 32; w++) s += wcnt[w][threadIdx.x];
      base[threadIdx.x] += s;
    }
    __syncthreads();
  }
}

}  // namespace

int radix_sort_pairs(unsigned long long *keys, unsigned long long *vals, unsigned long long *keys_tmp,
                     unsigned long long *vals_tmp, int64_t n, int bits, bool *result_in_tmp, Workspace &ws) {
  cudaStream_t s = ws.stream();
  *result_in_tmp = false;
  if (n <= 1 || bits <= 0) return GP_OK;
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  int64_t *hist, *offs;
  GP_TRY(ws.get(&hist, (size_t)(256 * ntiles)));
  GP_TRY(ws.get(&offs, (size_t)(256 * ntiles + 1)));
  unsigned long long *ks = keys, *vs = vals, *kd = keys_tmp, *vd = vals_tmp;
  for (int shift = 0; shift < bits; shift += 8) {
    (::gp::count_launch(), k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ks, n, shift, ntiles, hist));
    GP_TRY(scan_excl_i64(hist, offs, 256 * ntiles, offs + 256 * ntiles, ws));
    (::gp::count_launch(), k_radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ks, vs, kd, vd, n, shift, ntiles, offs));
    GP_LAUNCH_CHECK();
    std::swap(ks, kd);
    std::swap(vs, vd);
    *result_in_tmp = !*result_in_tmp;
  }
  return GP_OK;
}

}  // namespace gp
