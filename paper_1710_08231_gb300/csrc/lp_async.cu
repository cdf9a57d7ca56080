// lp_async.cu -- the paper's asynchronous label propagation (Section IV-A), a comparator for the
// deterministic Jacobi rounds of lp.cu.
//
// Section III-A's label propagation visits the queued vertices in increasing order of degree and moves
// each at once (in place) to the eligible cluster of strongest connection; Section IV-A parallelises it
// by cutting the degree-sorted order into packets that threads take one after another, with label
// updates visible at once and the cluster sizes updated by compare-and-swap so that U is never
// exceeded. Here a warp takes packets of 32 consecutive vertices of the (degree, id) order from a
// global counter and processes their queued vertices one after another: it sums the connection to
// every neighbouring label in its own shared-memory table (labels and cluster weights read as they are
// at that moment), picks the best eligible label (own label on ties, then larger H(seed, v, L), then
// smaller L), and reserves the target cluster's weight with a compare-and-swap loop that gives up once
// the bound would be exceeded. Results depend on the interleaving of the warps (non-deterministic);
// with a single warp the processing order is the sequential order and the result equals the oracle's.
// Each vertex may have at most 256 distinct neighbouring labels (its table holds 512 slots): any graph
// whose degrees are at most 256, or any run over at most 256 labels (refinement with k <= 256).
#include <algorithm>
#include <cstring>
#include <vector>

#include "gp_internal.cuh"
#include "lp_async.cuh"
#include "sort.cuh"

namespace gp {
namespace {

constexpr int kAsyncWarps = 8;
constexpr int kAsyncThreads = kAsyncWarps * 32;
constexpr int kAsyncCap = 512;  // table slots per warp
constexpr int kPacket = 32;

struct AsyncArgs {
  DGraph g;
  const int32_t *order;
  int32_t *labels;
  long long *lw;
  int64_t U;
  uint64_t smix;
  const uint8_t *act;  // NULL: every vertex is queued (round 0)
  uint8_t *act_next;
  unsigned long long *packet;  // next packet
  unsigned long long *stats;   // visits, entries, moves
};

template <int EW>
__global__ void __launch_bounds__(kAsyncThreads) k_lp_async(AsyncArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long *vals = reinterpret_cast<unsigned long long *>(smem) + wid * kAsyncCap;
  int *keys = reinterpret_cast<int *>(smem + kAsyncWarps * kAsyncCap * 8) + wid * kAsyncCap;
  for (int t = lane; t < kAsyncCap; t += 32) {
    keys[t] = -1;
    vals[t] = 0;
  }
  __syncwarp();
  const int64_t n = A.g.n;
  unsigned long long visits = 0, entries = 0, moves = 0;
  while (true) {
    unsigned long long p = 0;
    if (lane == 0) p = atomicAdd(A.packet, 1ull);
    p = __shfl_sync(kFull, p, 0);
    const int64_t lo = (int64_t)p * kPacket;
    if (lo >= n) break;
    const int64_t hi = min(n, lo + kPacket);
    for (int64_t i = lo; i < hi; i++) {
      const int v = A.order[i];
      if (A.act && !A.act[v]) continue;
      const int64_t rb = A.g.row_begin(v), re = A.g.row_begin(v + 1);
      const int64_t d = re - rb;
      visits += 1;
      entries += (unsigned long long)d;
      if (d == 0) continue;
      int cap = 64;
      while (cap < 2 * d && cap < kAsyncCap) cap <<= 1;
      const unsigned mask = (unsigned)cap - 1;
      const int L0 = *(volatile int32_t *)&A.labels[v];
      long long c0 = 0;
      for (int64_t e0 = rb; e0 < re; e0 += 32) {
        const int64_t e = e0 + lane;
        const bool in = e < re;
        const int L = in ? *(volatile int32_t *)&A.labels[__ldg(A.g.adj + e)] : -1;
        const long long w = in ? load_ew<EW>(A.g.ew, e) : 0;
        if (in && L == L0) c0 += w;
        const bool on = in && L != L0;
        const unsigned peers = __match_any_sync(kFull, on ? L : -1);
        if (on) {
          long long sum = 0;
          for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, w, __ffs(m) - 1);
          if (lane == __ffs(peers) - 1) {
            unsigned sl = mix32((unsigned)L) & mask;
            while (true) {
              const int k = atomicCAS(&keys[sl], -1, L);
              if (k == -1 || k == L) {
                atomicAdd(&vals[sl], (unsigned long long)sum);
                break;
              }
              sl = (sl + 1) & mask;
            }
          }
        }
      }
      c0 = warp_sum64(c0);
      __syncwarp();
      const long long cv = A.g.vweight(v);
      const uint64_t hv = mix64(A.smix ^ (uint64_t)(uint32_t)v);
      long long bc = 0;
      uint64_t bh = 0;
      int bL = -1;
      for (int s = lane; s < cap; s += 32) {
        const int L = keys[s];
        if (L < 0) continue;
        const long long c = (long long)vals[s];
        keys[s] = -1;
        vals[s] = 0;
        if (c <= c0 || *(volatile long long *)&A.lw[L] + cv > A.U) continue;
        const uint64_t h = mix64(hv ^ (uint64_t)(uint32_t)L);
        if (bL < 0 || c > bc || (c == bc && (h > bh || (h == bh && L < bL)))) {
          bc = c;
          bh = h;
          bL = L;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long c2 = __shfl_xor_sync(kFull, bc, o);
        const uint64_t h2 = __shfl_xor_sync(kFull, bh, o);
        const int L2 = __shfl_xor_sync(kFull, bL, o);
        if (L2 >= 0 && (bL < 0 || c2 > bc || (c2 == bc && (h2 > bh || (h2 == bh && L2 < bL))))) {
          bc = c2;
          bh = h2;
          bL = L2;
        }
      }
      __syncwarp();
      if (bL < 0) continue;
      // reserve the target's weight (compare-and-swap; gives up when U would be exceeded)
      int ok = 0;
      if (lane == 0) {
        unsigned long long old = *(volatile unsigned long long *)&A.lw[bL];
        while ((long long)old + cv <= A.U) {
          const unsigned long long prev =
              atomicCAS(reinterpret_cast<unsigned long long *>(&A.lw[bL]), old, old + (unsigned long long)cv);
          if (prev == old) {
            ok = 1;
            break;
          }
          old = prev;
        }
        if (ok) {
          atomicAdd(reinterpret_cast<unsigned long long *>(&A.lw[L0]), (unsigned long long)(-cv));
          A.labels[v] = bL;
          __threadfence();
        }
      }
      ok = __shfl_sync(kFull, ok, 0);
      if (!ok) continue;
      moves += 1;
      for (int64_t e = rb + lane; e < re; e += 32) A.act_next[__ldg(A.g.adj + e)] = 1;
      __syncwarp();
    }
  }
  if (lane == 0) {
    if (visits) atomicAdd(&A.stats[0], visits);
    if (entries) atomicAdd(&A.stats[1], entries);
    if (moves) atomicAdd(&A.stats[2], moves);
  }
}

__global__ void k_order_keys(DGraph g, unsigned long long *keys, unsigned long long *vals) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    keys[v] = ((unsigned long long)(g.row_begin(v + 1) - g.row_begin(v)) << 32) | (unsigned long long)v;
    vals[v] = (unsigned long long)v;
  }
}

__global__ void k_to_i32(const unsigned long long *a, int64_t n, int32_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)a[i];
}

__global__ void k_max_degree(DGraph g, unsigned long long *mx) {
  unsigned long long m = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)(g.row_begin(v + 1) - g.row_begin(v)));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, m);
}

int grid_of(int64_t items) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, (int64_t)num_sms() * 8));
}

}  // namespace

int run_lp_async(const DGraph &g, int32_t *labels, int64_t *lw, int64_t nl, int64_t U, int rounds, uint64_t seed,
                 bool single_warp, gp_lp_stats *stats, cudaStream_t s) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (g.n == 0 || rounds <= 0) return GP_OK;
  Workspace ws(s);
  const int64_t n = g.n;
  unsigned long long *keys, *vals, *keys2, *vals2, *mx, *ctr;
  int32_t *order;
  uint8_t *act[2];
  GP_TRY(ws.get(&keys, (size_t)n));
  GP_TRY(ws.get(&vals, (size_t)n));
  GP_TRY(ws.get(&keys2, (size_t)n));
  GP_TRY(ws.get(&vals2, (size_t)n));
  GP_TRY(ws.get(&order, (size_t)n));
  GP_TRY(ws.get(&act[0], (size_t)n));
  GP_TRY(ws.get(&act[1], (size_t)n));
  GP_TRY(ws.zeros(&mx, 1));
  // per round: packet counter and three statistics
  GP_TRY(ws.zeros(&ctr, (size_t)4 * rounds));
  (count_launch(), k_max_degree<<<grid_of(n), 256, 0, s>>>(g, mx));
  unsigned long long hmx = 0;
  GP_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  if (hmx > kAsyncCap / 2 && nl > kAsyncCap / 2) {
    set_error("asynchronous label propagation: a vertex may have more than 256 distinct neighbouring labels");
    return GP_ERR_UNSUPPORTED;
  }
  (count_launch(), k_order_keys<<<grid_of(n), 256, 0, s>>>(g, keys, vals));
  GP_LAUNCH_CHECK();
  bool in_tmp = false;
  int bits = 32;
  while (bits < 64 && ((hmx >> (bits - 32)) != 0)) bits++;  // degree bits above the 32 id bits
  GP_TRY(radix_sort_pairs(keys, vals, keys2, vals2, n, (bits + 7) / 8 * 8, &in_tmp, ws));
  (count_launch(), k_to_i32<<<grid_of(n), 256, 0, s>>>(in_tmp ? vals2 : vals, n, order));
  GP_LAUNCH_CHECK();
  const size_t smem = (size_t)kAsyncWarps * kAsyncCap * 12;
  const int ew = g.ew_mode();
  static bool attr[3] = {false, false, false};
  if (!attr[ew]) {
    if (ew == 0) GP_CUDA(cudaFuncSetAttribute(k_lp_async<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (ew == 1) GP_CUDA(cudaFuncSetAttribute(k_lp_async<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (ew == 2) GP_CUDA(cudaFuncSetAttribute(k_lp_async<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr[ew] = true;
  }
  const int grid = single_warp ? 1 : num_sms() * 4;
  const int threads = single_warp ? 32 : kAsyncThreads;
  gp_lp_stats st = {0, 0, 0, 0, 0};
  for (int r = 0; r < rounds; r++) {
    AsyncArgs A;
    A.g = g;
    A.order = order;
    A.labels = labels;
    A.lw = reinterpret_cast<long long *>(lw);
    A.U = U;
    A.smix = mix64(seed);
    A.act = r == 0 ? nullptr : act[r & 1];
    A.act_next = act[(r + 1) & 1];
    A.packet = ctr + 4 * r;
    A.stats = ctr + 4 * r + 1;
    GP_CUDA(cudaMemsetAsync(A.act_next, 0, (size_t)n, s));
    {
      ProfScope ps("lp_async", s);
      if (ew == 0) (count_launch(), k_lp_async<0><<<grid, threads, smem, s>>>(A));
      else if (ew == 1) (count_launch(), k_lp_async<1><<<grid, threads, smem, s>>>(A));
      else (count_launch(), k_lp_async<2><<<grid, threads, smem, s>>>(A));
      GP_LAUNCH_CHECK();
    }
    unsigned long long h[3];
    GP_CUDA(cudaMemcpyAsync(h, ctr + 4 * r + 1, sizeof(h), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    st.rounds = r + 1;
    st.visits += (int64_t)h[0];
    st.edges += (int64_t)h[1];
    st.moves += (int64_t)h[2];
    st.movers += (int64_t)h[2];
    if (h[2] == 0) break;
  }
  prof_add_counts("lp_async", st.visits, st.edges, 0);
  if (stats) *stats = st;
  return GP_OK;
}

}  // namespace gp
