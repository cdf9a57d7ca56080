// lp.cu -- size-constrained label propagation on the GPU.
//
// Method: Section III-A ("Clustering") and Section IV-A ("Parallel Size-Constraint Label
// Propagation") of "High-Quality Shared-Memory Graph Partitioning"; as refinement with U = Lmax in
// Section III-C / IV-C. A vertex moves to the eligible cluster of strongest connection; a cluster
// is eligible when it stays within U after the move; neighbours of moved vertices are visited in
// the next iteration.
//
// GPU design (what replaces the paper's degree sort, TBB work packets and CAS on cluster sizes):
//   * each round has two Jacobi sub-rounds split by the hash bit H(seed, r, v) >> 63; all decisions
//     of a sub-round read the labels and label weights of its start, which makes the result
//     independent of scheduling;
//   * active vertices are classified into degree bins (group of 4/8/16/32 lanes, one warp with a
//     shared-memory hash table, one CTA with a shared-memory hash table, several CTAs with a
//     global-memory hash table); the bins only schedule work, the chosen label is the same;
//   * connection sums are exact integers and the choice is a total order (connection, score sum,
//     H(seed, v, L), -L), so the aggregation order never matters;
//   * moves to one target are admitted by a deterministic rule instead of CAS: all proposals to
//     the target are ordered by (gain desc, score sum desc, id asc) and the longest prefix whose
//     weight fits under U is taken. When the total proposed weight fits, no ordering is needed;
//     otherwise the contested proposals are sorted (one CTA in shared memory for small sets, a
//     cooperative LSD radix sort for large ones) and admitted by a segmented prefix sum.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>

#include "lp.cuh"

namespace gp {

namespace {

constexpr int kBins = 7;  // G4, G8, G16, G32, WARP, CTA, HUB
constexpr int kBinZero = 7;  // degree-0 visits (statistics only)
constexpr int kWarpCap = 512;   // slots of a warp table (d <= 256)
constexpr int kCtaCap = 4096;   // slots of a CTA table (d <= 2048)
constexpr int kCtaThreads = 256;
constexpr int kWarpsPerBlock = 8;
constexpr int kHubChunk = 4096;  // CSR entries per hub work item
constexpr int kContestSmall = 4096;
constexpr int kSmallLabels = 2048;  // label spaces this small are aggregated in shared memory

struct LpCounters {
  unsigned int bin_count[8];
  unsigned int n_movers;
  unsigned int n_contested;
  unsigned int stop;
  int err;
  unsigned int hub_chunks;
  unsigned int bar_count, bar_gen;
  unsigned int pad;
  unsigned long long moves_round;
  unsigned long long moves, rounds, movers;
  unsigned long long bin_visits[8], bin_edges[8];
  unsigned long long max_gain, max_q;
};

struct LpArgs {
  DGraph g;
  int64_t nl;
  int64_t U;
  uint64_t smix;  // mix64(seed)
  int32_t *labels;
  int64_t *lw;
  const uint8_t *act;
  uint8_t *act_next;
  int round, sub;
  int deg_warp, deg_cta;
  const int32_t *q;
  int32_t *bin[kBins];
  int32_t *mv_v;
  int32_t *mv_t;
  int64_t *mv_gain;
  int64_t *mv_q;
  uint8_t *mv_adm;
  int64_t *demand;
  uint32_t *ct, *ct2;
  // hub tables
  const int32_t *hub_of;   // vertex -> hub index, -1 otherwise
  const int64_t *hub_base; // hub index -> first slot
  int32_t *hub_keys;
  unsigned long long *hub_vals;
  unsigned int *hub_qv;
  long long *hub_c0;       // per active hub (bin position): connection to the own label
  unsigned int *hub_prefix;  // per active hub: exclusive prefix of work chunks
  // cooperative sort scratch
  unsigned int *hist;   // nblocks * 256
  unsigned long long *hoff;  // nblocks * 256
  LpCounters *ctr;
};

__device__ __forceinline__ int bin_of(int64_t d, int deg_warp, int deg_cta) {
  if (d <= 4) return 0;
  if (d <= 8) return 1;
  if (d <= 16) return 2;
  if (d <= 32) return 3;
  if (d <= deg_warp) return 4;
  if (d <= deg_cta) return 5;
  return 6;
}

__device__ __forceinline__ unsigned warp_append(unsigned int *counter, bool pred) {
  unsigned m = __ballot_sync(kFull, pred);
  if (!m) return 0;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  return base + __popc(m & lanemask_lt());
}

// ------------------------------------------------------------------------------------ candidates
struct Best {
  long long conn;
  long long qs;
  unsigned long long h;
  int L;  // -1: none
};

__device__ __forceinline__ bool better(const Best &a, const Best &b) {
  if (a.L < 0) return false;
  if (b.L < 0) return true;
  if (a.conn != b.conn) return a.conn > b.conn;
  if (a.qs != b.qs) return a.qs > b.qs;
  if (a.h != b.h) return a.h > b.h;
  return a.L < b.L;
}

template <bool LQ>
__device__ __forceinline__ Best shfl_best(const Best &b, int o, int width) {
  Best r;
  r.conn = __shfl_xor_sync(kFull, b.conn, o, width);
  r.qs = LQ ? __shfl_xor_sync(kFull, b.qs, o, width) : 0;
  r.h = __shfl_xor_sync(kFull, b.h, o, width);
  r.L = __shfl_xor_sync(kFull, b.L, o, width);
  return r;
}

template <bool LQ, int W>
__device__ __forceinline__ Best group_best(Best b) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    Best x = shfl_best<LQ>(b, o, W);
    if (better(x, b)) b = x;
  }
  return b;
}

// Candidate L of vertex v (connection conn, score sum qs) against own-label connection c0.
__device__ __forceinline__ Best make_cand(const LpArgs &a, int v, int L, int L0, long long conn,
                                          long long qs, long long c0, long long cv) {
  Best b;
  b.L = -1;
  b.conn = 0;
  b.qs = 0;
  b.h = 0;
  if (L < 0 || L == L0 || conn <= c0) return b;  // own label wins ties
  if (a.lw[L] + cv > a.U) return b;               // not eligible
  b.L = L;
  b.conn = conn;
  b.qs = qs;
  b.h = mix64(mix64(a.smix ^ (uint64_t)(uint32_t)v) ^ (uint64_t)(uint32_t)L);
  return b;
}

__device__ __forceinline__ void write_mover(const LpArgs &a, unsigned idx, int v, const Best &b,
                                            long long c0) {
  a.mv_v[idx] = v;
  a.mv_t[idx] = b.L;
  a.mv_gain[idx] = b.conn - c0;
  a.mv_q[idx] = b.qs;
  a.mv_adm[idx] = 0;
}

// ------------------------------------------------------------------------------------ kernels
__global__ void k_degree_classes(DGraph g, int deg_warp, int deg_cta, LpCounters *ctr) {
  __shared__ unsigned int cnt[8];
  if (threadIdx.x < 8) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = g.row_begin(v + 1) - g.row_begin(v);
    if (d > 0) atomicAdd(&cnt[bin_of(d, deg_warp, deg_cta)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 8 && cnt[threadIdx.x]) atomicAdd(&ctr->bin_count[threadIdx.x], cnt[threadIdx.x]);
}

__global__ void k_sub_reset(LpCounters *ctr) {
  if (ctr->stop) return;
  if (threadIdx.x < 8) ctr->bin_count[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    ctr->n_movers = 0;
    ctr->n_contested = 0;
    ctr->hub_chunks = 0;
    ctr->max_gain = 0;
    ctr->max_q = 0;
  }
}

__global__ void k_round_end(LpCounters *ctr) {
  if (threadIdx.x != 0 || ctr->stop) return;
  ctr->rounds += 1;
  ctr->moves += ctr->moves_round;
  if (ctr->moves_round == 0) ctr->stop = 1;
  ctr->moves_round = 0;
}

__global__ void k_classify(LpArgs a, uint64_t rmix) {
  if (a.ctr->stop) return;
  __shared__ unsigned long long s_vis[8], s_edg[8];
  if (threadIdx.x < 8) {
    s_vis[threadIdx.x] = 0;
    s_edg[threadIdx.x] = 0;
  }
  __syncthreads();
  const int64_t n = a.g.n;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    int b = -1;
    int64_t d = 0;
    if (v < n) {
      bool act = (a.round == 0 || a.act[v]) && (int)(mix64(rmix ^ (uint64_t)v) >> 63) == a.sub;
      if (act) {
        d = a.g.row_begin(v + 1) - a.g.row_begin(v);
        b = d == 0 ? kBinZero : bin_of(d, a.deg_warp, a.deg_cta);
        atomicAdd(&s_vis[b], 1ull);
        atomicAdd(&s_edg[b], (unsigned long long)d);
      }
    }
#pragma unroll
    for (int bb = 0; bb < kBins; bb++) {
      unsigned pos = warp_append(&a.ctr->bin_count[bb], b == bb);
      if (b == bb) a.bin[bb][pos] = (int32_t)v;
    }
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    if (s_vis[threadIdx.x]) atomicAdd(&a.ctr->bin_visits[threadIdx.x], s_vis[threadIdx.x]);
    if (s_edg[threadIdx.x]) atomicAdd(&a.ctr->bin_edges[threadIdx.x], s_edg[threadIdx.x]);
  }
}

// Groups of G lanes, one vertex per group, d <= G: every lane holds one neighbour and computes the
// connection of its neighbour's label by comparing with all other lanes of the group.
template <int G, int EW, bool LQ>
__global__ void __launch_bounds__(256) k_choose_group(LpArgs a, int bin) {
  if (a.ctr->stop) return;
  const unsigned cnt = a.ctr->bin_count[bin];
  const int32_t *list = a.bin[bin];
  constexpr unsigned kGpw = 32 / G;
  const int lane = threadIdx.x & (G - 1);
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned sub = (threadIdx.x & 31) / G;
  for (unsigned base = gw * kGpw; base < cnt; base += nw * kGpw) {
    const unsigned i = base + sub;
    const bool valid = i < cnt;
    const int v = valid ? list[i] : 0;
    int64_t beg = 0, d = 0;
    if (valid) {
      beg = a.g.row_begin(v);
      d = a.g.row_begin(v + 1) - beg;
    }
    const bool has = lane < d;
    int Lu = -1;
    long long w = 0;
    int qq = 0;
    if (has) {
      const int u = __ldg(a.g.adj + beg + lane);
      Lu = a.labels[u];
      w = load_ew<EW>(a.g.ew, beg + lane);
      if (LQ) qq = __ldg(a.q + beg + lane);
    }
    const int L0 = valid ? a.labels[v] : -2;
    long long c0 = (has && Lu == L0) ? w : 0;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) c0 += __shfl_xor_sync(kFull, c0, o, G);
    long long conn = 0, qs = 0;
    bool first = true;
#pragma unroll
    for (int j = 0; j < G; j++) {
      const int Lj = __shfl_sync(kFull, Lu, j, G);
      long long wj;
      if constexpr (EW == 0) wj = 1;
      else wj = __shfl_sync(kFull, w, j, G);
      int qj = 0;
      if constexpr (LQ) qj = __shfl_sync(kFull, qq, j, G);
      if (Lj == Lu) {
        conn += wj;
        qs += qj;
        if (j < lane) first = false;
      }
    }
    Best b;
    b.L = -1;
    b.conn = b.qs = 0;
    b.h = 0;
    if (has && first) b = make_cand(a, v, Lu, L0, conn, qs, c0, valid ? a.g.vweight(v) : 0);
    b = group_best<LQ, G>(b);
    const bool mover = valid && lane == 0 && b.L >= 0;
    const unsigned idx = warp_append(&a.ctr->n_movers, mover);
    if (mover) write_mover(a, idx, v, b, c0);
  }
}

__device__ __forceinline__ unsigned slot_hash(int L) { return (unsigned)L * 0x9E3779B1u; }

// One warp per vertex, 32 < d <= deg_warp <= 256, open-addressing table in shared memory.
template <int EW, bool LQ>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_choose_warp(LpArgs a) {
  if (a.ctr->stop) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long *vals = reinterpret_cast<unsigned long long *>(smem) + wid * kWarpCap;
  int *keys = reinterpret_cast<int *>(smem + kWarpsPerBlock * kWarpCap * 8) + wid * kWarpCap;
  unsigned int *qv = reinterpret_cast<unsigned int *>(smem + kWarpsPerBlock * kWarpCap * 12) + wid * kWarpCap;
  for (int s = lane; s < kWarpCap; s += 32) {
    keys[s] = -1;
    vals[s] = 0;
    if (LQ) qv[s] = 0;
  }
  __syncwarp();
  const unsigned cnt = a.ctr->bin_count[4];
  const int32_t *list = a.bin[4];
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned i = gw; i < cnt; i += nw) {
    const int v = list[i];
    const int64_t beg = a.g.row_begin(v), end = a.g.row_begin(v + 1);
    const int d = (int)(end - beg);
    int cap = 64;
    while (cap < 2 * d) cap <<= 1;
    const unsigned mask = (unsigned)cap - 1;
    const int L0 = a.labels[v];
    long long c0 = 0;
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int L = a.labels[__ldg(a.g.adj + e)];
      const long long w = load_ew<EW>(a.g.ew, e);
      if (L == L0) {
        c0 += w;
        continue;
      }
      unsigned s = slot_hash(L) & mask;
      while (true) {
        const int k = atomicCAS(&keys[s], -1, L);
        if (k == -1 || k == L) {
          atomicAdd(&vals[s], (unsigned long long)w);
          if (LQ) atomicAdd(&qv[s], (unsigned)__ldg(a.q + e));
          break;
        }
        s = (s + 1) & mask;
      }
    }
    c0 = warp_sum64(c0);
    __syncwarp();
    const long long cv = a.g.vweight(v);
    Best b;
    b.L = -1;
    b.conn = b.qs = 0;
    b.h = 0;
    for (int s = lane; s < cap; s += 32) {
      const int L = keys[s];
      if (L >= 0) {
        Best x = make_cand(a, v, L, L0, (long long)vals[s], LQ ? (long long)qv[s] : 0, c0, cv);
        if (better(x, b)) b = x;
        keys[s] = -1;
        vals[s] = 0;
        if (LQ) qv[s] = 0;
      }
    }
    __syncwarp();
    b = group_best<LQ, 32>(b);
    const bool mover = lane == 0 && b.L >= 0;
    const unsigned idx = warp_append(&a.ctr->n_movers, mover);
    if (mover) write_mover(a, idx, v, b, c0);
  }
}

template <bool LQ>
__device__ __forceinline__ Best block_best(Best b, Best *sh) {
  b = group_best<LQ, 32>(b);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[wid] = b;
  __syncthreads();
  if (wid == 0) {
    Best x;
    x.L = -1;
    x.conn = x.qs = 0;
    x.h = 0;
    if (lane < (int)(blockDim.x >> 5)) x = sh[lane];
    x = group_best<LQ, 32>(x);
    if (lane == 0) sh[0] = x;
  }
  __syncthreads();
  Best r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ long long block_sum(long long x, long long *sh) {
  x = warp_sum64(x);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long y = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
    y = warp_sum64(y);
    if (lane == 0) sh[0] = y;
  }
  __syncthreads();
  long long r = sh[0];
  __syncthreads();
  return r;
}

// One CTA per vertex, deg_warp < d <= deg_cta <= 2048, table in shared memory.
template <int EW, bool LQ>
__global__ void __launch_bounds__(kCtaThreads) k_choose_cta(LpArgs a) {
  if (a.ctr->stop) return;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long *vals = reinterpret_cast<unsigned long long *>(smem);
  int *keys = reinterpret_cast<int *>(smem + kCtaCap * 8);
  unsigned int *qv = reinterpret_cast<unsigned int *>(smem + kCtaCap * 12);
  __shared__ Best sh_best[32];
  __shared__ long long sh_sum[32];
  for (int s = threadIdx.x; s < kCtaCap; s += blockDim.x) {
    keys[s] = -1;
    vals[s] = 0;
    if (LQ) qv[s] = 0;
  }
  __syncthreads();
  const unsigned cnt = a.ctr->bin_count[5];
  const int32_t *list = a.bin[5];
  for (unsigned i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int v = list[i];
    const int64_t beg = a.g.row_begin(v), end = a.g.row_begin(v + 1);
    const int d = (int)(end - beg);
    int cap = 64;
    while (cap < 2 * d) cap <<= 1;
    const unsigned mask = (unsigned)cap - 1;
    const int L0 = a.labels[v];
    long long c0 = 0;
    for (int64_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
      const int L = a.labels[__ldg(a.g.adj + e)];
      const long long w = load_ew<EW>(a.g.ew, e);
      if (L == L0) {
        c0 += w;
        continue;
      }
      unsigned s = slot_hash(L) & mask;
      while (true) {
        const int k = atomicCAS(&keys[s], -1, L);
        if (k == -1 || k == L) {
          atomicAdd(&vals[s], (unsigned long long)w);
          if (LQ) atomicAdd(&qv[s], (unsigned)__ldg(a.q + e));
          break;
        }
        s = (s + 1) & mask;
      }
    }
    c0 = block_sum(c0, sh_sum);  // contains __syncthreads: table complete
    const long long cv = a.g.vweight(v);
    Best b;
    b.L = -1;
    b.conn = b.qs = 0;
    b.h = 0;
    for (int s = threadIdx.x; s < cap; s += blockDim.x) {
      const int L = keys[s];
      if (L >= 0) {
        Best x = make_cand(a, v, L, L0, (long long)vals[s], LQ ? (long long)qv[s] : 0, c0, cv);
        if (better(x, b)) b = x;
        keys[s] = -1;
        vals[s] = 0;
        if (LQ) qv[s] = 0;
      }
    }
    b = block_best<LQ>(b, sh_best);
    if (threadIdx.x == 0 && b.L >= 0) {
      const unsigned idx = atomicAdd(&a.ctr->n_movers, 1u);
      write_mover(a, idx, v, b, c0);
    }
  }
}

// Hubs (d > deg_cta): chunks of kHubChunk entries accumulate into the hub's global table.
__global__ void k_hub_prefix(LpArgs a) {
  if (a.ctr->stop) return;
  __shared__ long long tmp[32];
  __shared__ long long carry_s, tot_s;
  const unsigned cnt = a.ctr->bin_count[6];
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (unsigned base = 0; base < cnt; base += blockDim.x) {
    const unsigned i = base + threadIdx.x;
    long long c = 0;
    if (i < cnt) {
      const int v = a.bin[6][i];
      const int64_t d = a.g.row_begin(v + 1) - a.g.row_begin(v);
      c = (d + kHubChunk - 1) / kHubChunk;
      a.hub_c0[i] = 0;
    }
    const long long ex = block_excl_scan64(c, tmp, &tot_s);
    if (i < cnt) a.hub_prefix[i] = (unsigned)(carry_s + ex);
    __syncthreads();
    if (threadIdx.x == 0) carry_s += tot_s;
    __syncthreads();
  }
  if (threadIdx.x == 0) a.ctr->hub_chunks = (unsigned)carry_s;
}

template <int EW, bool LQ>
__global__ void __launch_bounds__(256) k_hub_accum(LpArgs a) {
  if (a.ctr->stop) return;
  __shared__ long long sh_sum[32];
  const unsigned cnt = a.ctr->bin_count[6];
  const unsigned chunks = a.ctr->hub_chunks;
  for (unsigned c = blockIdx.x; c < chunks; c += gridDim.x) {
    // hub i with hub_prefix[i] <= c < hub_prefix[i+1]
    unsigned lo = 0, hi = cnt;
    while (hi - lo > 1) {
      const unsigned mid = (lo + hi) >> 1;
      if (a.hub_prefix[mid] <= c) lo = mid;
      else hi = mid;
    }
    const unsigned i = lo;
    const int v = a.bin[6][i];
    const int64_t rb = a.g.row_begin(v), re = a.g.row_begin(v + 1);
    const int64_t beg = rb + (int64_t)(c - a.hub_prefix[i]) * kHubChunk;
    const int64_t end = min(re, beg + kHubChunk);
    const int h = a.hub_of[v];
    const int64_t tb = a.hub_base[h];
    const int64_t d = re - rb;
    int64_t cap = 64;
    while (cap < 2 * d) cap <<= 1;
    const uint64_t mask = (uint64_t)cap - 1;
    const int L0 = a.labels[v];
    long long c0 = 0;
    for (int64_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
      const int L = a.labels[__ldg(a.g.adj + e)];
      const long long w = load_ew<EW>(a.g.ew, e);
      if (L == L0) {
        c0 += w;
        continue;
      }
      uint64_t s = ((uint64_t)slot_hash(L) * 0x100000001ull) & mask;
      while (true) {
        const int k = atomicCAS(&a.hub_keys[tb + s], -1, L);
        if (k == -1 || k == L) {
          atomicAdd(&a.hub_vals[tb + s], (unsigned long long)w);
          if (LQ) atomicAdd(&a.hub_qv[tb + s], (unsigned)__ldg(a.q + e));
          break;
        }
        s = (s + 1) & mask;
      }
    }
    c0 = block_sum(c0, sh_sum);
    if (threadIdx.x == 0 && c0) atomicAdd((unsigned long long *)&a.hub_c0[i], (unsigned long long)c0);
  }
}

template <bool LQ>
__global__ void __launch_bounds__(256) k_hub_choose(LpArgs a) {
  if (a.ctr->stop) return;
  __shared__ Best sh_best[32];
  const unsigned cnt = a.ctr->bin_count[6];
  for (unsigned i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int v = a.bin[6][i];
    const int64_t d = a.g.row_begin(v + 1) - a.g.row_begin(v);
    int64_t cap = 64;
    while (cap < 2 * d) cap <<= 1;
    const int h = a.hub_of[v];
    const int64_t tb = a.hub_base[h];
    const int L0 = a.labels[v];
    const long long c0 = a.hub_c0[i];
    const long long cv = a.g.vweight(v);
    Best b;
    b.L = -1;
    b.conn = b.qs = 0;
    b.h = 0;
    for (int64_t s = threadIdx.x; s < cap; s += blockDim.x) {
      const int L = a.hub_keys[tb + s];
      if (L >= 0) {
        Best x = make_cand(a, v, L, L0, (long long)a.hub_vals[tb + s], LQ ? (long long)a.hub_qv[tb + s] : 0, c0, cv);
        if (better(x, b)) b = x;
        a.hub_keys[tb + s] = -1;
        a.hub_vals[tb + s] = 0;
        if (LQ) a.hub_qv[tb + s] = 0;
      }
    }
    b = block_best<LQ>(b, sh_best);
    if (threadIdx.x == 0 && b.L >= 0) {
      const unsigned idx = atomicAdd(&a.ctr->n_movers, 1u);
      write_mover(a, idx, v, b, c0);
    }
  }
}

// ------------------------------------------------------------------------------------ admission
__global__ void k_demand(LpArgs a) {
  if (a.ctr->stop) return;
  __shared__ unsigned long long sdem[kSmallLabels];
  const bool small = a.nl <= kSmallLabels;
  if (small) {
    for (int k = threadIdx.x; k < a.nl; k += blockDim.x) sdem[k] = 0;
    __syncthreads();
  }
  const unsigned nm = a.ctr->n_movers;
  if (threadIdx.x == 0 && blockIdx.x == 0) a.ctr->movers += nm;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += gridDim.x * blockDim.x) {
    const int T = a.mv_t[i];
    const unsigned long long c = (unsigned long long)a.g.vweight(a.mv_v[i]);
    if (small) atomicAdd(&sdem[T], c);
    else atomicAdd(reinterpret_cast<unsigned long long *>(&a.demand[T]), c);
  }
  if (small) {
    __syncthreads();
    for (int k = threadIdx.x; k < a.nl; k += blockDim.x)
      if (sdem[k]) atomicAdd(reinterpret_cast<unsigned long long *>(&a.demand[k]), sdem[k]);
  }
}

template <bool LQ>
__global__ void k_admit(LpArgs a) {
  if (a.ctr->stop) return;
  const unsigned nm = a.ctr->n_movers;
  unsigned long long mg = 0, mq = 0;
  for (unsigned base = blockIdx.x * blockDim.x; base < nm; base += gridDim.x * blockDim.x) {
    const unsigned i = base + threadIdx.x;
    bool contested = false;
    if (i < nm) {
      const int T = a.mv_t[i];
      if (a.lw[T] + a.demand[T] <= a.U) {
        a.mv_adm[i] = 1;
      } else {
        contested = true;
        mg = max(mg, (unsigned long long)a.mv_gain[i]);
        if (LQ) mq = max(mq, (unsigned long long)a.mv_q[i]);
      }
    }
    const unsigned pos = warp_append(&a.ctr->n_contested, contested);
    if (contested) a.ct[pos] = i;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mg = max(mg, __shfl_xor_sync(kFull, mg, o));
    mq = max(mq, __shfl_xor_sync(kFull, mq, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (mg) atomicMax(&a.ctr->max_gain, mg);
    if (LQ && mq) atomicMax(&a.ctr->max_q, mq);
  }
}

// Ordering of contested movers: target asc, gain desc, score sum desc, id asc.
__device__ __forceinline__ bool mover_less(const LpArgs &a, unsigned x, unsigned y) {
  const int tx = a.mv_t[x], ty = a.mv_t[y];
  if (tx != ty) return tx < ty;
  const long long gx = a.mv_gain[x], gy = a.mv_gain[y];
  if (gx != gy) return gx > gy;
  const long long qx = a.mv_q[x], qy = a.mv_q[y];
  if (qx != qy) return qx > qy;
  return a.mv_v[x] < a.mv_v[y];
}

// Segmented inclusive prefix sums of c(v) over the sorted contested list, then admission.
// Processes positions [lo, hi) of `order` with a block-wide carry (one block at a time).
__device__ void admit_sorted_block(const LpArgs &a, const unsigned *order, unsigned lo, unsigned hi,
                                   long long carry_in, int carry_target, long long *tmp,
                                   long long *carry_out, int *carry_target_out) {
  // carry (carry_in, carry_target): running sum of the open segment that ends at position lo-1.
  __shared__ long long s_carry;
  __shared__ int s_ct;
  if (threadIdx.x == 0) {
    s_carry = carry_in;
    s_ct = carry_target;
  }
  __syncthreads();
  for (unsigned base = lo; base < hi; base += blockDim.x) {
    const unsigned p = base + threadIdx.x;
    const bool valid = p < hi;
    unsigned idx = valid ? order[p] : 0;
    const int T = valid ? a.mv_t[idx] : -1;
    const int Tprev = (valid && p > lo) ? a.mv_t[order[p - 1]] : (valid ? s_ct : -1);
    const bool head = valid && T != Tprev;
    long long c = valid ? a.g.vweight(a.mv_v[idx]) : 0;
    // segmented inclusive scan: pairs (flag, value)
    int f = head ? 1 : 0;
    long long x = c;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kFull, x, o);
      const int fy = __shfl_up_sync(kFull, f, o);
      if (lane >= o) {
        if (!f) x += y;
        f |= fy;
      }
    }
    __shared__ long long wsum[32];
    __shared__ int wflag[32];
    if (lane == 31) {
      wsum[wid] = x;
      wflag[wid] = f;
    }
    __syncthreads();
    if (wid == 0) {
      long long s = lane < nw ? wsum[lane] : 0;
      int fl = lane < nw ? wflag[lane] : 0;
      // exclusive scan of (flag, sum) over warps, seeded by the block carry
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, s, o);
        const int fy = __shfl_up_sync(kFull, fl, o);
        if (lane >= o) {
          if (!fl) s += y;
          fl |= fy;
        }
      }
      // s, fl: inclusive over warps 0..lane; convert to exclusive with the block carry
      long long ps = __shfl_up_sync(kFull, s, 1);
      int pf = __shfl_up_sync(kFull, fl, 1);
      if (lane == 0) {
        ps = 0;
        pf = 0;
      }
      long long ex = pf ? ps : ps + s_carry;
      if (lane < nw) wsum[lane] = ex;
    }
    __syncthreads();
    // prefix for this element: if no head at or before it within its warp, add warp exclusive
    const long long incl = f ? x : x + wsum[wid];
    if (valid) {
      if (a.lw[T] + incl <= a.U) a.mv_adm[idx] = 1;
    }
    __syncthreads();
    // new carry: the last valid element of this tile
    const unsigned last = min(hi, base + blockDim.x) - 1;
    if (p == last) {
      s_carry = incl;
      s_ct = T;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (carry_out) *carry_out = s_carry;
    if (carry_target_out) *carry_target_out = s_ct;
  }
  (void)tmp;
}

// Small contested sets: one CTA sorts the indices in shared memory (bitonic) and admits.
__global__ void __launch_bounds__(1024) k_contest_small(LpArgs a) {
  if (a.ctr->stop) return;
  const unsigned cnt = a.ctr->n_contested;
  if (cnt == 0 || cnt > kContestSmall) return;
  __shared__ unsigned key[kContestSmall];
  unsigned P = 1;
  while (P < cnt) P <<= 1;
  for (unsigned i = threadIdx.x; i < P; i += blockDim.x) key[i] = i < cnt ? a.ct[i] : 0xffffffffu;
  __syncthreads();
  for (unsigned k = 2; k <= P; k <<= 1) {
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      for (unsigned t = threadIdx.x; t < P / 2; t += blockDim.x) {
        const unsigned i = 2 * j * (t / j) + (t % j);
        const unsigned l = i + j;
        const bool up = (i & k) == 0;
        const unsigned x = key[i], y = key[l];
        bool swap;
        if (x == 0xffffffffu) swap = (y != 0xffffffffu) == up;
        else if (y == 0xffffffffu) swap = !up;
        else swap = mover_less(a, y, x) == up;
        if (swap) {
          key[i] = y;
          key[l] = x;
        }
      }
      __syncthreads();
    }
  }
  __shared__ long long tmp[32];
  admit_sorted_block(a, key, 0, cnt, 0, -1, tmp, nullptr, nullptr);
}

// Large contested sets: cooperative stable LSD radix sort of the mover indices by
// (target, gain desc, score sum desc, id) -- least significant key first -- then segmented admission.
__device__ __forceinline__ unsigned long long field_key(const LpArgs &a, unsigned idx, int field,
                                                        unsigned long long maxg, unsigned long long maxq) {
  switch (field) {
    case 0: return (unsigned long long)(unsigned)a.mv_v[idx];
    case 1: return maxq - (unsigned long long)a.mv_q[idx];
    case 2: return maxg - (unsigned long long)a.mv_gain[idx];
    default: return (unsigned long long)(unsigned)a.mv_t[idx];
  }
}

__device__ __forceinline__ int bits_for(unsigned long long x) { return x ? 64 - __clzll(x) : 0; }

template <bool LQ>
__global__ void __launch_bounds__(256) k_contest_large(LpArgs a, GridBarrier bar) {
  if (a.ctr->stop) return;
  const unsigned cnt = a.ctr->n_contested;
  if (cnt <= kContestSmall) return;
  const unsigned nb = gridDim.x, b = blockIdx.x;
  const unsigned long long maxg = a.ctr->max_gain, maxq = a.ctr->max_q;
  const int nbits[4] = {bits_for((unsigned long long)(a.g.n > 0 ? a.g.n - 1 : 0)), LQ ? bits_for(maxq) : 0,
                        bits_for(maxg), bits_for((unsigned long long)(a.nl > 0 ? a.nl - 1 : 0))};
  const unsigned chunk = (cnt + nb - 1) / nb;
  const unsigned lo = min(cnt, b * chunk), hi = min(cnt, lo + chunk);
  __shared__ unsigned hist[256];
  __shared__ unsigned long long base[256];
  __shared__ unsigned wcnt[8][256];
  unsigned *src = a.ct, *dst = a.ct2;
  for (int field = 0; field < 4; field++) {
    for (int shift = 0; shift < nbits[field]; shift += 8) {
      // 1. block histogram of its slice
      for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0;
      __syncthreads();
      for (unsigned p = lo + threadIdx.x; p < hi; p += blockDim.x)
        atomicAdd(&hist[(field_key(a, src[p], field, maxg, maxq) >> shift) & 255], 1u);
      __syncthreads();
      for (int t = threadIdx.x; t < 256; t += blockDim.x) a.hist[(size_t)b * 256 + t] = hist[t];
      if (!grid_sync(bar)) return;
      // 2. per digit: exclusive prefix over blocks; digit totals
      for (unsigned t = b * blockDim.x + threadIdx.x; t < 256; t += nb * blockDim.x) {
        unsigned long long run = 0;
        for (unsigned bb = 0; bb < nb; bb++) {
          const unsigned h = a.hist[(size_t)bb * 256 + t];
          a.hoff[(size_t)bb * 256 + t] = run;
          run += h;
        }
        a.hoff[(size_t)nb * 256 + t] = run;  // digit total
      }
      if (!grid_sync(bar)) return;
      // 3. block base per digit = exclusive scan of totals + block prefix
      if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int t = 0; t < 256; t++) {
          base[t] = acc + a.hoff[(size_t)b * 256 + t];
          acc += a.hoff[(size_t)nb * 256 + t];
        }
      }
      __syncthreads();
      // 4. stable scatter of the slice
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      for (unsigned t0 = lo; t0 < hi; t0 += blockDim.x) {
        const unsigned p = t0 + threadIdx.x;
        const bool valid = p < hi;
        const unsigned x = valid ? src[p] : 0;
        const int dg = valid ? (int)((field_key(a, x, field, maxg, maxq) >> shift) & 255) : 256;
        for (int k = threadIdx.x; k < 8 * 256; k += blockDim.x) wcnt[k >> 8][k & 255] = 0;
        __syncthreads();
        const unsigned peers = __match_any_sync(kFull, dg);
        const int rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[wid][dg] = __popc(peers);
        __syncthreads();
        if (valid) {
          unsigned pre = 0;
          for (int w = 0; w < wid; w++) pre += wcnt[w][dg];
          dst[base[dg] + pre + rank] = x;
        }
        __syncthreads();
        if (threadIdx.x < 256) {
          unsigned s = 0;
          for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += wcnt[w][threadIdx.x];
          base[threadIdx.x] += s;
        }
        __syncthreads();
        (void)lane;
      }
      if (!grid_sync(bar)) return;
      unsigned *t = src;
      src = dst;
      dst = t;
    }
  }
  // Segmented admission over the sorted order `src`: blocks take consecutive slices; each block
  // needs the running sum of the segment open at its slice start. Pass 1: per-block (head seen,
  // sum of trailing segment part); pass 2: carries resolved sequentially by one thread.
  __shared__ long long tmp[32];
  {
    long long tail = 0;
    int has_head = 0;
    int last_t = -1;
    if (lo < hi) {
      last_t = a.mv_t[src[hi - 1]];
      // sum of c over the maximal suffix of the slice whose target equals last_t, and whether the
      // slice contains a segment head (target change) in it
      long long part = 0;
      int headseen = 0;
      for (unsigned p = lo + threadIdx.x; p < hi; p += blockDim.x) {
        const unsigned idx = src[p];
        if (a.mv_t[idx] == last_t) part += a.g.vweight(a.mv_v[idx]);
        else headseen = 1;
      }
      tail = block_sum(part, tmp);
      has_head = __syncthreads_or(headseen);
    } else {
      __syncthreads_or(0);
    }
    if (threadIdx.x == 0) {
      a.hoff[(size_t)b * 4 + 0] = (unsigned long long)tail;
      a.hoff[(size_t)b * 4 + 1] = (unsigned long long)has_head;
      a.hoff[(size_t)b * 4 + 2] = (unsigned long long)(long long)last_t;
      a.hoff[(size_t)b * 4 + 3] = (unsigned long long)(hi > lo ? 1 : 0);
    }
    if (!grid_sync(bar)) return;
    if (b == 0 && threadIdx.x == 0) {
      // carry into block bb = running sum of the segment open at its start
      long long run = 0;
      long long run_t = -1;
      for (unsigned bb = 0; bb < nb; bb++) {
        a.hoff[(size_t)nb * 4 + bb * 2 + 0] = (unsigned long long)run;
        a.hoff[(size_t)nb * 4 + bb * 2 + 1] = (unsigned long long)run_t;
        if (!a.hoff[(size_t)bb * 4 + 3]) continue;
        const long long t = (long long)a.hoff[(size_t)bb * 4 + 0];
        const long long lt = (long long)a.hoff[(size_t)bb * 4 + 2];
        const int hh = (int)a.hoff[(size_t)bb * 4 + 1];
        if (!hh && lt == run_t) run += t;
        else run = t;
        run_t = lt;
      }
    }
    if (!grid_sync(bar)) return;
  }
  const long long carry = (long long)a.hoff[(size_t)nb * 4 + b * 2 + 0];
  const int carry_t = (int)(long long)a.hoff[(size_t)nb * 4 + b * 2 + 1];
  if (lo < hi) admit_sorted_block(a, src, lo, hi, carry, carry_t, tmp, nullptr, nullptr);
}

// ------------------------------------------------------------------------------------ apply
__global__ void k_apply(LpArgs a) {
  if (a.ctr->stop) return;
  __shared__ long long sdel[kSmallLabels];
  __shared__ unsigned long long s_moves;
  const bool small = a.nl <= kSmallLabels;
  if (small)
    for (int k = threadIdx.x; k < a.nl; k += blockDim.x) sdel[k] = 0;
  if (threadIdx.x == 0) s_moves = 0;
  __syncthreads();
  const unsigned nm = a.ctr->n_movers;
  const int lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned i = gw; i < nm; i += nw) {
    const int T = a.mv_t[i];
    const bool adm = a.mv_adm[i];
    if (lane == 0) a.demand[T] = 0;
    if (!adm) continue;
    const int v = a.mv_v[i];
    if (lane == 0) {
      const long long c = a.g.vweight(v);
      const int L0 = a.labels[v];
      a.labels[v] = T;
      if (small) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&sdel[T]), (unsigned long long)c);
        atomicAdd(reinterpret_cast<unsigned long long *>(&sdel[L0]), (unsigned long long)(-c));
      } else {
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.lw[T]), (unsigned long long)c);
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.lw[L0]), (unsigned long long)(-c));
      }
      atomicAdd(&s_moves, 1ull);
    }
    const int64_t beg = a.g.row_begin(v), end = a.g.row_begin(v + 1);
    for (int64_t e = beg + lane; e < end; e += 32) a.act_next[__ldg(a.g.adj + e)] = 1;
  }
  __syncthreads();
  if (small)
    for (int k = threadIdx.x; k < a.nl; k += blockDim.x)
      if (sdel[k]) atomicAdd(reinterpret_cast<unsigned long long *>(&a.lw[k]), (unsigned long long)sdel[k]);
  if (threadIdx.x == 0 && s_moves) atomicAdd(&a.ctr->moves_round, s_moves);
}

// ------------------------------------------------------------------------------------ hub setup
__global__ void k_hub_mark(DGraph g, int deg_cta, int32_t *hub_of, int64_t *hub_cap, unsigned *count) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = g.row_begin(v + 1) - g.row_begin(v);
    if (d > deg_cta) {
      const unsigned h = atomicAdd(count, 1u);
      hub_of[v] = (int32_t)h;
      int64_t cap = 64;
      while (cap < 2 * d) cap <<= 1;
      hub_cap[h] = cap;
    } else {
      hub_of[v] = -1;
    }
  }
}

__global__ void k_block_weights(DGraph g, const int32_t *part, int64_t k, int64_t *bw, int *bad) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int b = part[v];
    if (b < 0 || b >= k) {
      if (bad) atomicExch(bad, 1);
      continue;
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(&bw[b]), (unsigned long long)g.vweight(v));
  }
}

template <class K>
int max_blocks(K kernel, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) per_sm = 1;
  return std::max(1, per_sm) * num_sms();
}

template <int EW, bool LQ>
struct LpKernels {
  static int launch_sub(const LpArgs &a, const int64_t cap[kBins], int warp_grid_cap, cudaStream_t s,
                        GridBarrier bar, int coop_grid) {
    const int nsm = num_sms();
    auto grid_for = [&](int64_t items, int per_block, int limit) {
      int64_t g = (items + per_block - 1) / per_block;
      return (int)std::max<int64_t>(1, std::min<int64_t>(g, limit));
    };
    if (cap[0]) {
      ProfScope ps("lp_choose_g4", s);
      (::gp::count_launch(), k_choose_group<4, EW, LQ><<<grid_for(cap[0], 64, nsm * 16), 256, 0, s>>>(a, 0));
    }
    if (cap[1]) {
      ProfScope ps("lp_choose_g8", s);
      (::gp::count_launch(), k_choose_group<8, EW, LQ><<<grid_for(cap[1], 32, nsm * 16), 256, 0, s>>>(a, 1));
    }
    if (cap[2]) {
      ProfScope ps("lp_choose_g16", s);
      (::gp::count_launch(), k_choose_group<16, EW, LQ><<<grid_for(cap[2], 16, nsm * 16), 256, 0, s>>>(a, 2));
    }
    if (cap[3]) {
      ProfScope ps("lp_choose_g32", s);
      (::gp::count_launch(), k_choose_group<32, EW, LQ><<<grid_for(cap[3], 8, nsm * 16), 256, 0, s>>>(a, 3));
    }
    if (cap[4]) {
      ProfScope ps("lp_choose_warp", s);
      {
        const size_t sm = kWarpsPerBlock * kWarpCap * 16;
        (::gp::count_launch(), k_choose_warp<EW, LQ><<<grid_for(cap[4], kWarpsPerBlock, warp_grid_cap), kWarpsPerBlock * 32, sm, s>>>(a));
      }
    }
    if (cap[5]) {
      ProfScope ps("lp_choose_cta", s);
      (::gp::count_launch(), k_choose_cta<EW, LQ><<<grid_for(cap[5], 1, nsm * 3), kCtaThreads, kCtaCap * 16, s>>>(a));
    }
    if (cap[6]) {
      ProfScope ps("lp_choose_hub", s);
      (::gp::count_launch(), k_hub_prefix<<<1, 1024, 0, s>>>(a));
      (::gp::count_launch(), k_hub_accum<EW, LQ><<<nsm * 4, 256, 0, s>>>(a));
      (::gp::count_launch(), k_hub_choose<LQ><<<grid_for(cap[6], 1, nsm * 4), 256, 0, s>>>(a));
    }
    GP_LAUNCH_CHECK();
    const int64_t mv_cap = a.g.n;
    const int ag = grid_for(mv_cap, 256, nsm * 8);
    (::gp::count_launch(), k_demand<<<ag, 256, 0, s>>>(a));
    (::gp::count_launch(), k_admit<LQ><<<ag, 256, 0, s>>>(a));
    (::gp::count_launch(), k_contest_small<<<1, 1024, 0, s>>>(a));
    {
      LpArgs aa = a;
      void *params[] = {(void *)&aa, (void *)&bar};
      count_launch();
      GP_CUDA(cudaLaunchCooperativeKernel((void *)k_contest_large<LQ>, coop_grid, 256, params, 0, s));
    }
    (::gp::count_launch(), k_apply<<<grid_for(mv_cap, 8, nsm * 8), 256, 0, s>>>(a));
    GP_LAUNCH_CHECK();
    return GP_OK;
  }
};

bool g_attr_done[3][2] = {{false, false}, {false, false}, {false, false}};

template <int EW, bool LQ>
int set_attrs() {
  if (g_attr_done[EW][LQ]) return GP_OK;
  GP_CUDA(cudaFuncSetAttribute(k_choose_warp<EW, LQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kWarpsPerBlock * kWarpCap * 16));
  GP_CUDA(cudaFuncSetAttribute(k_choose_cta<EW, LQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCtaCap * 16));
  g_attr_done[EW][LQ] = true;
  return GP_OK;
}

template <int EW, bool LQ>
int run_rounds(LpArgs a, const int64_t cap[kBins], int rounds, uint64_t seed, uint8_t *act_buf[2],
               cudaStream_t s, GridBarrier bar, int coop_grid) {
  GP_TRY(set_attrs<EW, LQ>());
  const int nsm = num_sms();
  const int warp_grid_cap = max_blocks(k_choose_warp<EW, LQ>, kWarpsPerBlock * 32, kWarpsPerBlock * kWarpCap * 16);
  const int cls_grid = (int)std::max<int64_t>(1, std::min<int64_t>((a.g.n + 255) / 256, nsm * 8));
  for (int r = 0; r < rounds; r++) {
    a.round = r;
    a.act = act_buf[r & 1];
    a.act_next = act_buf[(r + 1) & 1];
    GP_CUDA(cudaMemsetAsync(a.act_next, 0, (size_t)a.g.n, s));
    const uint64_t rmix = mix64(a.smix ^ (uint64_t)r);
    for (int sub = 0; sub < 2; sub++) {
      a.sub = sub;
      (::gp::count_launch(), k_sub_reset<<<1, 32, 0, s>>>(a.ctr));
      (::gp::count_launch(), k_classify<<<cls_grid, 256, 0, s>>>(a, rmix));
      GP_TRY((LpKernels<EW, LQ>::launch_sub(a, cap, warp_grid_cap, s, bar, coop_grid)));
    }
    (::gp::count_launch(), k_round_end<<<1, 32, 0, s>>>(a.ctr));
    GP_LAUNCH_CHECK();
  }
  return GP_OK;
}

}  // namespace

LpConfig lp_config_from(const gp_params *p) {
  LpConfig c;
  if (p) {
    if (p->deg_warp > 0) c.deg_warp = std::max(32, std::min(256, (int)p->deg_warp));
    if (p->deg_cta > 0) c.deg_cta = std::max(c.deg_warp, std::min(2048, (int)p->deg_cta));
  }
  if (c.deg_cta < c.deg_warp) c.deg_cta = c.deg_warp;
  return c;
}

int block_weights(const DGraph &g, const int32_t *part, int64_t k, int64_t *bw, int *bad_dev, cudaStream_t s) {
  GP_CUDA(cudaMemsetAsync(bw, 0, sizeof(int64_t) * (size_t)std::max<int64_t>(k, 1), s));
  if (g.n == 0) return GP_OK;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((g.n + 255) / 256, num_sms() * 8));
  (::gp::count_launch(), k_block_weights<<<grid, 256, 0, s>>>(g, part, k, bw, bad_dev));
  GP_LAUNCH_CHECK();
  return GP_OK;
}

int run_lp(const DGraph &g, const int32_t *q, int32_t *labels, int64_t *lw, int64_t nl, int64_t U, int rounds,
           uint64_t seed, gp_lp_stats *stats, cudaStream_t s, const LpConfig &cfg) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (g.n == 0 || rounds <= 0) return GP_OK;
  if (g.n >= (int64_t)1 << 31 || nl >= (int64_t)1 << 31) {
    set_error("label propagation supports n < 2^31");
    return GP_ERR_UNSUPPORTED;
  }
  Workspace ws(s);
  LpCounters *ctr;
  GP_TRY(ws.zeros(&ctr, 1));
  const int nsm = num_sms();
  const int grid_n = (int)std::max<int64_t>(1, std::min<int64_t>((g.n + 255) / 256, nsm * 8));
  (::gp::count_launch(), k_degree_classes<<<grid_n, 256, 0, s>>>(g, cfg.deg_warp, cfg.deg_cta, ctr));
  GP_LAUNCH_CHECK();
  LpCounters h;
  GP_CUDA(cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  int64_t cap[kBins];
  for (int b = 0; b < kBins; b++) cap[b] = h.bin_count[b];
  GP_CUDA(cudaMemsetAsync(ctr, 0, sizeof(LpCounters), s));

  LpArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = g;
  a.nl = nl;
  a.U = U;
  a.smix = mix64(seed);
  a.labels = labels;
  a.lw = lw;
  a.q = q;
  a.deg_warp = cfg.deg_warp;
  a.deg_cta = cfg.deg_cta;
  a.ctr = ctr;
  for (int b = 0; b < kBins; b++) GP_TRY(ws.get(&a.bin[b], (size_t)std::max<int64_t>(cap[b], 1)));
  const size_t n = (size_t)g.n;
  GP_TRY(ws.get(&a.mv_v, n));
  GP_TRY(ws.get(&a.mv_t, n));
  GP_TRY(ws.get(&a.mv_gain, n));
  GP_TRY(ws.get(&a.mv_q, n));
  GP_TRY(ws.get(&a.mv_adm, n));
  GP_TRY(ws.zeros(&a.demand, (size_t)nl));
  GP_TRY(ws.get(&a.ct, n));
  GP_TRY(ws.get(&a.ct2, n));
  uint8_t *act_buf[2];
  GP_TRY(ws.get(&act_buf[0], n));
  GP_TRY(ws.get(&act_buf[1], n));
  GP_CUDA(cudaMemsetAsync(act_buf[0], 0, n, s));
  if (cap[6]) {
    int32_t *hub_of;
    int64_t *hub_cap;
    unsigned *hcount;
    GP_TRY(ws.get(&hub_of, n));
    GP_TRY(ws.get(&hub_cap, (size_t)cap[6] + 1));
    GP_TRY(ws.zeros(&hcount, 1));
    (::gp::count_launch(), k_hub_mark<<<grid_n, 256, 0, s>>>(g, cfg.deg_cta, hub_of, hub_cap, hcount));
    GP_LAUNCH_CHECK();
    int64_t *hub_base, *total;
    GP_TRY(ws.get(&hub_base, (size_t)cap[6] + 1));
    GP_TRY(ws.get(&total, 1));
    GP_TRY(scan_excl_i64(hub_cap, hub_base, cap[6], total, ws));
    int64_t slots = 0;
    GP_CUDA(cudaMemcpyAsync(&slots, total, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    GP_TRY(ws.get(&a.hub_keys, (size_t)slots));
    GP_TRY(ws.zeros(&a.hub_vals, (size_t)slots));
    GP_TRY(ws.zeros(&a.hub_qv, (size_t)slots));
    GP_CUDA(cudaMemsetAsync(a.hub_keys, 0xff, sizeof(int32_t) * (size_t)slots, s));
    GP_TRY(ws.get(&a.hub_c0, (size_t)cap[6]));
    GP_TRY(ws.get(&a.hub_prefix, (size_t)cap[6] + 1));
    a.hub_of = hub_of;
    a.hub_base = hub_base;
  }
  // cooperative admission grid
  int coop_per_sm = 0;
  void *klarge = q ? (void *)k_contest_large<true> : (void *)k_contest_large<false>;
  GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&coop_per_sm, klarge, 256, 0));
  const int coop_grid = std::max(1, std::min(coop_per_sm, 2)) * nsm;
  GP_TRY(ws.get(&a.hist, (size_t)coop_grid * 256 + 16));
  GP_TRY(ws.get(&a.hoff, (size_t)coop_grid * 256 + 256 + 16));
  GridBarrier bar{&ctr->bar_count, &ctr->bar_gen, &ctr->err};

  const int ew = g.ew_mode();
  int st;
  if (q) {
    st = ew == 0 ? run_rounds<0, true>(a, cap, rounds, seed, act_buf, s, bar, coop_grid)
       : ew == 1 ? run_rounds<1, true>(a, cap, rounds, seed, act_buf, s, bar, coop_grid)
                 : run_rounds<2, true>(a, cap, rounds, seed, act_buf, s, bar, coop_grid);
  } else {
    st = ew == 0 ? run_rounds<0, false>(a, cap, rounds, seed, act_buf, s, bar, coop_grid)
       : ew == 1 ? run_rounds<1, false>(a, cap, rounds, seed, act_buf, s, bar, coop_grid)
                 : run_rounds<2, false>(a, cap, rounds, seed, act_buf, s, bar, coop_grid);
  }
  GP_TRY(st);
  GP_CUDA(cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  if (h.err) {
    set_error("label propagation: bounded device wait gave up");
    return GP_ERR_TIMEOUT;
  }
  if (profiling()) {
    static const char *names[kBins] = {"lp_choose_g4", "lp_choose_g8", "lp_choose_g16", "lp_choose_g32",
                                       "lp_choose_warp", "lp_choose_cta", "lp_choose_hub"};
    const int64_t ob = g.offset_bytes(), vb = g.vw_bytes(), eb = g.ew_bytes();
    for (int b = 0; b < kBins; b++) {
      const int64_t vis = (int64_t)h.bin_visits[b], edg = (int64_t)h.bin_edges[b];
      // algorithmic bytes: two offsets, own label, own weight, one label-weight read per vertex;
      // per entry: adjacency, neighbour label, edge weight (and score)
      const int64_t bytes = vis * (2 * ob + 4 + vb + 8) + edg * (8 + eb + (q ? 4 : 0));
      prof_add_counts(names[b], vis, edg, bytes);
    }
  }
  if (stats) {
    stats->rounds = (int64_t)h.rounds;
    stats->moves = (int64_t)h.moves;
    stats->movers = (int64_t)h.movers;
    int64_t vis = 0, edg = 0;
    for (int b = 0; b < 8; b++) {
      vis += (int64_t)h.bin_visits[b];
      edg += (int64_t)h.bin_edges[b];
    }
    stats->visits = vis;
    stats->edges = edg;
  }
  return GP_OK;
}

}  // namespace gp
