// sort.cu -- device-wide stable LSD radix sort of (uint64 key, uint64 value) pairs.
//
// Each pass handles 8 key bits with three kernels: per-tile digit histograms (digit-major), an
// exclusive scan of the histograms, and a stable scatter in which every tile ranks its items per
// digit in order (warp match + per-warp counts), stages them in shared memory in digit order and
// writes each digit's run contiguously. Used where many independent rows must be sorted at
// once (the contraction of very large clusters).
#include <algorithm>

#include "sort.cuh"

namespace gp {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
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

// Stable scatter of one pass. Warp w of a tile owns its items [w, w + 1) * 32 kSortItems (the tile's
// order is warp, then round, then lane). The warps count their digits first; the counts become each
// warp's starting positions inside the tile's digit runs; the warps then place their items in order
// in shared memory, and the tile leaves run by run: consecutive threads write consecutive addresses.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const unsigned long long *kin,
                                                                const unsigned long long *vin,
                                                                unsigned long long *kout, unsigned long long *vout,
                                                                int64_t n, int shift, int64_t ntiles,
                                                                const int64_t *offs) {
  extern __shared__ unsigned long long s_items[];  // kSortTile keys, then kSortTile values
  constexpr int kW = kSortThreads / 32;
  static_assert(kSortThreads == 256, "one thread per digit");
  __shared__ unsigned wpos[kW][256];
  __shared__ unsigned loc[256];
  __shared__ int64_t gbase[256];
  __shared__ unsigned wsum[kW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
  const int64_t wbase = tbase + (int64_t)wid * (32 * kSortItems);
  for (int d = lane; d < 256; d += 32) wpos[wid][d] = 0;
  __syncwarp();
  for (int k = 0; k < kSortItems; k++) {
    const int64_t i = wbase + k * 32 + lane;
    const int dg = i < n ? (int)((kin[i] >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(kFull, dg);
    if (dg < 256 && lane == __ffs(peers) - 1) wpos[wid][dg] += (unsigned)__popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int d = threadIdx.x;
    unsigned tot = 0;
    for (int w = 0; w < kW; w++) tot += wpos[w][d];
    unsigned x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    unsigned run = x - tot;
    for (int w = 0; w < wid; w++) run += wsum[w];
    loc[d] = run;
    for (int w = 0; w < kW; w++) {
      const unsigned c = wpos[w][d];
      wpos[w][d] = run;
      run += c;
    }
    gbase[d] = offs[(int64_t)d * ntiles + blockIdx.x];
  }
  __syncthreads();
  for (int k = 0; k < kSortItems; k++) {
    const int64_t i = wbase + k * 32 + lane;
    const bool valid = i < n;
    const unsigned long long key = valid ? kin[i] : 0, val = valid ? vin[i] : 0;
    const int dg = valid ? (int)((key >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(kFull, dg);
    const unsigned rank = (unsigned)__popc(peers & lanemask_lt());
    if (valid) {
      const unsigned p = wpos[wid][dg] + rank;
      s_items[p] = key;
      s_items[kSortTile + p] = val;
    }
    __syncwarp();
    if (valid && rank == 0) wpos[wid][dg] += (unsigned)__popc(peers);
    __syncwarp();
  }
  __syncthreads();
  const int tn = (int)min((int64_t)kSortTile, n - tbase);
  for (int p = threadIdx.x; p < tn; p += kSortThreads) {
    const unsigned long long key = s_items[p];
    const int dg = (int)((key >> shift) & 255);
    const int64_t out = gbase[dg] + (int64_t)(p - (int)loc[dg]);
    kout[out] = key;
    vout[out] = s_items[kSortTile + p];
  }
}

}  // namespace

int radix_sort_pairs(unsigned long long *keys, unsigned long long *vals, unsigned long long *keys_tmp,
                     unsigned long long *vals_tmp, int64_t n, int bits, bool *result_in_tmp, Workspace &ws) {
  cudaStream_t s = ws.stream();
  *result_in_tmp = false;
  if (n <= 1 || bits <= 0) return GP_OK;
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  constexpr int kScatterSmem = (int)(2 * kSortTile * sizeof(unsigned long long));
  static bool smem_set = false;
  if (!smem_set) {
    GP_CUDA(cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, kScatterSmem));
    smem_set = true;
  }
  int64_t *hist, *offs;
  GP_TRY(ws.get(&hist, (size_t)(256 * ntiles)));
  GP_TRY(ws.get(&offs, (size_t)(256 * ntiles + 1)));
  unsigned long long *ks = keys, *vs = vals, *kd = keys_tmp, *vd = vals_tmp;
  for (int shift = 0; shift < bits; shift += 8) {
    (::gp::count_launch(), k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ks, n, shift, ntiles, hist));
    GP_TRY(scan_excl_i64(hist, offs, 256 * ntiles, offs + 256 * ntiles, ws));
    (::gp::count_launch(), k_radix_scatter<<<(unsigned)ntiles, kSortThreads, kScatterSmem, s>>>(ks, vs, kd, vd, n, shift, ntiles, offs));
    GP_LAUNCH_CHECK();
    std::swap(ks, kd);
    std::swap(vs, vd);
    *result_in_tmp = !*result_in_tmp;
  }
  return GP_OK;
}

}  // namespace gp
