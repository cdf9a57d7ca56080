// contract.cu -- contraction of a clustering into the weighted quotient graph on the GPU.
//
// Method (Section III-A; Section IV-A "Parallel Contraction"): cluster ids are remapped to
// [0, n') by a prefix sum over an array holding ones at the used ids; each coarse vertex weighs the
// sum of its members; each coarse edge (a, b), a != b, weighs the sum of the fine edges between
// clusters a and b.
//
// GPU design: instead of the paper's concurrent hash table, the (cv, cu, omega) pairs are sorted
// and reduced in two levels. Fine vertices are bucketed by coarse id (a counting sort), which sorts
// the pairs by cv; within one coarse row the pairs are sorted by cu and equal keys are summed:
// in registers by one warp (<= 32 pairs), in shared memory by one CTA (<= 4096 pairs), or by a
// CTA-wide LSD radix sort in global memory for larger rows. Rows come out sorted by neighbour id,
// so the coarse CSR is canonical and independent of scheduling.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "contract.cuh"
#include "lp.cuh"
#include "sort.cuh"

namespace gp {

namespace {

constexpr int kRowSmall = 32;     // <= 32 pairs: one warp, registers
constexpr int kRowWarp = 256;     // <= 256 pairs: one warp, shared-memory hash of 512 slots
constexpr int kRowWarpBig = 1024; // <= 1024 pairs: one warp, shared-memory hash of 2048 slots
constexpr int kRowMedium = 4096;  // <= 4096 pairs: one CTA, shared-memory hash
constexpr int kRowThreads = 256;
constexpr int kWarpSlots = 2 * kRowWarp;
constexpr int kCtaSlots = 2 * kRowMedium;

__global__ void k_mark_used(const int32_t *labels, int64_t n, int64_t nl, uint32_t *used, int *bad) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int L = labels[v];
    if (L < 0 || L >= nl) {
      atomicExch(bad, 1);
      continue;
    }
    used[L] = 1;
  }
}

// Fine -> coarse map and, per coarse vertex, member count, weight and degree sum. Members of one
// cluster are mostly neighbours in id order, so the warp combines equal coarse ids before its atomics.
// A label outside [0, nl) sets *bad and maps its vertex to 0 (the caller reports the error).
__global__ void k_f2c(DGraph g, const int32_t *labels, int64_t nl, const int32_t *newid, int32_t *f2c, int64_t *cnt,
                      int64_t *cw, int64_t *dsum, int *bad) {
  const int lane = threadIdx.x & 31;
  for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x; v0 < g.n; v0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = v0 + threadIdx.x;
    bool ok = v < g.n;
    int cv = 0;
    long long c = 0, d = 0;
    if (ok) {
      const int L = labels[v];
      if (L < 0 || L >= nl) {
        atomicExch(bad, 1);
        f2c[v] = 0;
        ok = false;
      } else {
        cv = newid[L];
        f2c[v] = cv;
        c = g.vweight(v);
        d = g.row_begin(v + 1) - g.row_begin(v);
      }
    }
    const unsigned peers = __match_any_sync(kFull, ok ? cv : -1);
    if (!ok) continue;
    long long cs = 0, ds = 0;
    for (unsigned m = peers; m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      cs += __shfl_sync(peers, c, src);
      ds += __shfl_sync(peers, d, src);
    }
    if (lane == __ffs(peers) - 1) {
      atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[cv]), (unsigned long long)__popc(peers));
      atomicAdd(reinterpret_cast<unsigned long long *>(&cw[cv]), (unsigned long long)cs);
      atomicAdd(reinterpret_cast<unsigned long long *>(&dsum[cv]), (unsigned long long)ds);
    }
  }
}

__global__ void k_members(int64_t n, const int32_t *f2c, const int64_t *mstart, unsigned *fill, int32_t *members) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int cv = f2c[v];
    const unsigned pos = atomicAdd(&fill[cv], 1u);
    members[mstart[cv] + pos] = (int32_t)v;
  }
}

__global__ void k_max_i64(const int64_t *x, int64_t n, unsigned long long *out) {
  unsigned long long m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)x[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// nc_dev: the number of coarse vertices (device; the grid is sized for an upper bound)
__global__ void k_row_classify(const int64_t *nc_dev, const int64_t *dsum, int32_t *l0, int32_t *l1, int32_t *l2,
                               int32_t *l3, int32_t *l4, unsigned *counts) {
  const int64_t nc = *nc_dev;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < nc; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = base + threadIdx.x;
    int b = -1;
    if (c < nc) {
      const int64_t D = dsum[c];
      b = D <= kRowSmall ? 0 : (D <= kRowWarp ? 3 : (D <= kRowWarpBig ? 4 : (D <= kRowMedium ? 1 : 2)));
    }
    int32_t *lists[5] = {l0, l1, l2, l3, l4};
    for (int bb = 0; bb < 5; bb++) {
      const unsigned m = __ballot_sync(kFull, b == bb);
      if (!m) continue;
      const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
      unsigned pos = 0;
      if (lane == leader) pos = atomicAdd(&counts[bb], (unsigned)__popc(m));
      pos = __shfl_sync(kFull, pos, leader) + __popc(m & lanemask_lt());
      if (b == bb) lists[bb][pos] = (int32_t)c;
    }
  }
}

struct RowArgs {
  DGraph g;
  const int32_t *f2c;
  const int64_t *mstart;
  const int32_t *members;
  const int64_t *tstart;
  int32_t *okey;
  int64_t *oval;
  int64_t *rowcnt;
  const int32_t *list;
  const unsigned *count;
  const int64_t *dsum;
  int key_bits;
};

// Rows with at most 32 pairs: one warp gathers them into shared memory, sorts them in registers
// (bitonic network over the lanes) and sums runs of equal neighbour ids.
template <int EW>
__global__ void __launch_bounds__(256) k_row_warp(RowArgs a) {
  __shared__ int skey[8][32];
  __shared__ long long sval[8][32];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned cnt = *a.count;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned i = gw; i < cnt; i += nw) {
    const int cv = a.list[i];
    const int64_t mb = a.mstart[cv], me = a.mstart[cv + 1];
    int P = 0;
    for (int64_t m = mb; m < me; m++) {
      const int v = a.members[m];
      const int64_t b = a.g.row_begin(v), e = a.g.row_begin(v + 1);
      for (int64_t x = b; x < e; x += 32) {
        const int64_t j = x + lane;
        const bool valid = j < e;
        const int cu = valid ? a.f2c[__ldg(a.g.adj + j)] : -1;
        const bool keep = valid && cu != cv;
        const unsigned mask = __ballot_sync(kFull, keep);
        if (keep) {
          const int pos = P + __popc(mask & lanemask_lt());
          skey[wid][pos] = cu;
          sval[wid][pos] = load_ew<EW>(a.g.ew, j);
        }
        P += __popc(mask);
      }
    }
    __syncwarp();
    int key = lane < P ? skey[wid][lane] : INT_MAX;
    long long val = lane < P ? sval[wid][lane] : 0;
    __syncwarp();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int ok = __shfl_xor_sync(kFull, key, j);
        const long long ov = __shfl_xor_sync(kFull, val, j);
        const bool up = (lane & k) == 0;
        const bool lower = (lane & j) == 0;
        const bool take = lower ? (up ? ok < key : ok > key) : (up ? ok > key : ok < key);
        if (take) {
          key = ok;
          val = ov;
        }
      }
    }
    long long sum = 0;
#pragma unroll
    for (int j = 0; j < 32; j++) {
      const int kj = __shfl_sync(kFull, key, j);
      const long long vj = __shfl_sync(kFull, val, j);
      if (kj == key) sum += vj;
    }
    const int prev = __shfl_up_sync(kFull, key, 1);
    const bool head = lane < P && (lane == 0 || prev != key);
    const unsigned hm = __ballot_sync(kFull, head);
    if (head) {
      const int64_t pos = a.tstart[cv] + __popc(hm & lanemask_lt());
      a.okey[pos] = key;
      a.oval[pos] = sum;
    }
    if (lane == 0) a.rowcnt[cv] = __popc(hm);
  }
}



__device__ __forceinline__ unsigned row_slot(int cu) { return mix32((unsigned)cu); }

// Rows with 32 < pairs <= 256: one warp sums the pairs by neighbour id in a shared-memory hash
// table, compacts the distinct ids and sorts them (bitonic) before writing the row.
// Rows of up to S/2 pairs: one warp per row, an S-slot hash table per warp in shared memory (the
// CTA's warps are laid out one table after another). The warp walks the concatenated rows of 32
// members at a time, 64 entries per step (all lanes busy whatever the members' degrees, adjacency
// read contiguously); equal coarse neighbours of one step are combined in the warp before they touch
// the table.
// Table values: 32-bit counts with unit edge weights (a coarse entry counts at most the fine entries,
// fewer than 2^32), else 64-bit sums.
template <int EW>
using RowVal = typename std::conditional<EW == 0, unsigned, unsigned long long>::type;
template <int EW>
constexpr int row_slot_bytes() { return 4 + (int)sizeof(RowVal<EW>); }

template <int EW, int S>
__global__ void __launch_bounds__(kRowThreads) k_row_whash(RowArgs a) {
  using V = RowVal<EW>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nwb = blockDim.x >> 5;
  V *vals = reinterpret_cast<V *>(smem) + wid * S;
  int *keys = reinterpret_cast<int *>(smem + (size_t)nwb * S * sizeof(V)) + wid * S;
  for (int t = lane; t < S; t += 32) {
    keys[t] = -1;
    vals[t] = 0;
  }
  __syncwarp();
  const unsigned cnt = *a.count;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned i = gw; i < cnt; i += nw) {
    const int cv = a.list[i];
    const int64_t mb = a.mstart[cv], me = a.mstart[cv + 1];
    int cap = 64;
    while (cap < 2 * a.dsum[cv]) cap <<= 1;
    const unsigned mask = (unsigned)cap - 1;
    for (int64_t m0 = mb; m0 < me; m0 += 32) {
      // the warp walks the concatenation of the rows of members m0 .. m0+31, 64 entries per step
      const int64_t m = m0 + lane;
      int64_t rb = 0, deg = 0;
      if (m < me) {
        const int v = a.members[m];
        rb = a.g.row_begin(v);
        deg = a.g.row_begin(v + 1) - rb;
      }
      int64_t incl = deg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const int64_t excl = incl - deg;
      const int64_t total = __shfl_sync(kFull, incl, 31);
      for (int64_t t0 = 0; t0 < total; t0 += 64) {
        int cu[2];
        long long w[2];
        bool on[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int64_t t = t0 + h * 32 + lane;
          int j = 0;  // owner: the largest lane j with excl_j <= t
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int64_t ex = __shfl_sync(kFull, excl, j + step);
            if (j + step < 32 && ex <= t) j += step;
          }
          const int64_t x = __shfl_sync(kFull, rb, j) + (t - __shfl_sync(kFull, excl, j));
          on[h] = t < total;
          cu[h] = on[h] ? a.f2c[__ldg(a.g.adj + x)] : -1;
          w[h] = on[h] ? load_ew<EW>(a.g.ew, x) : 0;
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const bool ok = on[h] && cu[h] != cv;
          const unsigned peers = __match_any_sync(kFull, ok ? cu[h] : -1);
          // weights below 2^26 sum exactly in 32 bits over at most 32 lanes: one warp reduction
          const bool wide = EW != 0 && __any_sync(kFull, ok && (w[h] >= (1ll << 26) || w[h] < 0));
          if (!ok) continue;
          long long sum = 0;
          if constexpr (EW == 0) {
            sum = __popc(peers);
          } else if (!wide) {
            sum = (long long)__reduce_add_sync(peers, (unsigned)w[h]);
          } else {
            for (unsigned pm = peers; pm; pm &= pm - 1) sum += __shfl_sync(peers, w[h], __ffs(pm) - 1);
          }
          if (lane != __ffs(peers) - 1) continue;
          unsigned sl = row_slot(cu[h]) & mask;
          while (true) {
            const int k = atomicCAS(&keys[sl], -1, cu[h]);
            if (k == -1 || k == cu[h]) {
              atomicAdd(&vals[sl], (V)sum);
              break;
            }
            sl = (sl + 1) & mask;
          }
        }
      }
    }
    __syncwarp();
    // compact the used slots to the front (every lane reads its slot before anyone writes)
    int u = 0;
    for (int c0 = 0; c0 < cap; c0 += 32) {
      const int k = keys[c0 + lane];
      const V val = vals[c0 + lane];
      const unsigned hm = __ballot_sync(kFull, k >= 0);
      __syncwarp();
      if (k >= 0) {
        const int pos = u + __popc(hm & lanemask_lt());
        keys[pos] = k;
        vals[pos] = val;
      }
      u += __popc(hm);
      __syncwarp();
    }
    int Pp = 1;
    while (Pp < u) Pp <<= 1;
    for (int t = u + lane; t < cap; t += 32) {
      keys[t] = t < Pp ? INT_MAX : -1;
      vals[t] = 0;
    }
    __syncwarp();
    for (int k = 2; k <= Pp; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = lane; t < Pp / 2; t += 32) {
          const int lo = 2 * j * (t / j) + (t % j), hi = lo + j;
          const bool up = (lo & k) == 0;
          const int x = keys[lo], y = keys[hi];
          if ((x > y) == up && x != y) {
            keys[lo] = y;
            keys[hi] = x;
            const V vx = vals[lo];
            vals[lo] = vals[hi];
            vals[hi] = vx;
          }
        }
        __syncwarp();
      }
    }
    const int64_t dst = a.tstart[cv];
    for (int t = lane; t < u; t += 32) {
      a.okey[dst + t] = keys[t];
      a.oval[dst + t] = (int64_t)vals[t];
    }
    if (lane == 0) a.rowcnt[cv] = u;
    __syncwarp();
    for (int t = lane; t < Pp; t += 32) {
      keys[t] = -1;
      vals[t] = 0;
    }
    __syncwarp();
  }
}

// Rows with 256 < pairs <= 4096: the same with one CTA and a larger table.
template <int EW>
__global__ void __launch_bounds__(kRowThreads) k_row_cta(RowArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  long long *vals = reinterpret_cast<long long *>(smem);
  int *keys = reinterpret_cast<int *>(smem + kCtaSlots * 8);
  __shared__ long long tmp[32];
  __shared__ long long tot_s, carry_s;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int t = threadIdx.x; t < kCtaSlots; t += blockDim.x) {
    keys[t] = -1;
    vals[t] = 0;
  }
  __syncthreads();
  const unsigned cnt = *a.count;
  for (unsigned i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int cv = a.list[i];
    const int64_t mb = a.mstart[cv], me = a.mstart[cv + 1];
    int cap = 64;
    while (cap < 2 * a.dsum[cv]) cap <<= 1;
    const unsigned mask = (unsigned)cap - 1;
    for (int64_t m = mb + wid; m < me; m += nwarps) {
      const int v = a.members[m];
      const int64_t b = a.g.row_begin(v), e = a.g.row_begin(v + 1);
      for (int64_t x = b + lane; x < e; x += 32) {
        const int cu = a.f2c[__ldg(a.g.adj + x)];
        if (cu == cv) continue;
        const long long w = load_ew<EW>(a.g.ew, x);
        unsigned sl = row_slot(cu) & mask;
        while (true) {
          const int k = atomicCAS(&keys[sl], -1, cu);
          if (k == -1 || k == cu) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&vals[sl]), (unsigned long long)w);
            break;
          }
          sl = (sl + 1) & mask;
        }
      }
    }
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int c0 = 0; c0 < cap; c0 += blockDim.x) {
      const int t = c0 + threadIdx.x;
      const int k = t < cap ? keys[t] : -1;
      const long long val = t < cap ? vals[t] : 0;
      const long long ex = block_excl_scan64((long long)(k >= 0 ? 1 : 0), tmp, &tot_s);
      if (k >= 0) {
        keys[carry_s + ex] = k;
        vals[carry_s + ex] = val;
      }
      __syncthreads();
      if (threadIdx.x == 0) carry_s += tot_s;
      __syncthreads();
    }
    const int u = (int)carry_s;
    int Pp = 1;
    while (Pp < u) Pp <<= 1;
    for (int t = u + threadIdx.x; t < cap; t += blockDim.x) {
      keys[t] = t < Pp ? INT_MAX : -1;
      vals[t] = 0;
    }
    __syncthreads();
    for (int k = 2; k <= Pp; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < Pp / 2; t += blockDim.x) {
          const int lo = 2 * j * (t / j) + (t % j), hi = lo + j;
          const bool up = (lo & k) == 0;
          const int x = keys[lo], y = keys[hi];
          if ((x > y) == up && x != y) {
            keys[lo] = y;
            keys[hi] = x;
            const long long vx = vals[lo];
            vals[lo] = vals[hi];
            vals[hi] = vx;
          }
        }
        __syncthreads();
      }
    }
    const int64_t dst = a.tstart[cv];
    for (int t = threadIdx.x; t < u; t += blockDim.x) {
      a.okey[dst + t] = keys[t];
      a.oval[dst + t] = vals[t];
    }
    if (threadIdx.x == 0) a.rowcnt[cv] = u;
    __syncthreads();
    for (int t = threadIdx.x; t < Pp; t += blockDim.x) {
      keys[t] = -1;
      vals[t] = 0;
    }
    __syncthreads();
  }
}

// Rows with more than 4096 pairs: the pairs of all such rows are gathered into one array keyed by
// (row index, neighbour id), sorted together by a device-wide radix sort and reduced by key.
__global__ void k_large_index(const int32_t *list, const unsigned *count, int32_t *large_idx) {
  const unsigned cnt = *count;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    large_idx[list[i]] = (int32_t)i;
}

template <int EW>
__global__ void k_large_gather(DGraph g, const int32_t *f2c, const int32_t *large_idx, const int64_t *lofs,
                               unsigned long long *lfill, int kb, unsigned long long *keys,
                               unsigned long long *vals) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = gw; v < g.n; v += nw) {
    const int i = large_idx[f2c[v]];
    if (i < 0) continue;
    const int64_t b = g.row_begin(v), e = g.row_begin(v + 1);
    unsigned long long pos = 0;
    if (lane == 0) pos = atomicAdd(&lfill[i], (unsigned long long)(e - b));
    pos = __shfl_sync(kFull, pos, 0) + (unsigned long long)lofs[i];
    for (int64_t x = b + lane; x < e; x += 32) {
      const int cu = f2c[__ldg(g.adj + x)];
      keys[pos + (x - b)] = ((unsigned long long)i << kb) | (unsigned long long)(unsigned)cu;
      vals[pos + (x - b)] = (unsigned long long)load_ew<EW>(g.ew, x);
    }
  }
}

__global__ void k_large_heads(const unsigned long long *keys, int64_t N, int kb, const int32_t *list, int64_t *flag) {
  const unsigned long long mask = (1ull << kb) - 1;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[j];
    const int cv = list[k >> kb];
    const bool head = (int)(k & mask) != cv && (j == 0 || keys[j - 1] != k);
    flag[j] = head ? 1 : 0;
  }
}

// Sorted large-row pairs to coarse entries: every pair of a non-self run adds its weight to the run's
// output slot (the run's rank among its row's runs, from the head scan), a warp adding once per run it
// holds; the run's head writes the neighbour id. oval must be zero on entry.
__global__ void k_large_write(const unsigned long long *keys, const unsigned long long *vals, int64_t N, int kb,
                              const int32_t *list, const int64_t *uidx, const int64_t *lofs, const int64_t *tstart,
                              int32_t *okey, int64_t *oval) {
  const unsigned long long mask = (1ull << kb) - 1;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); j0 < N; j0 += stride) {
    const int64_t j = j0 + lane;
    bool on = false;
    unsigned long long out = ~0ull;
    long long v = 0;
    if (j < N) {
      const unsigned long long k = keys[j];
      const int64_t i = (int64_t)(k >> kb);
      const int cu = (int)(k & mask), cv = list[i];
      if (cu != cv) {
        on = true;
        const int64_t u1 = uidx[j + 1];
        out = (unsigned long long)(tstart[cv] + (u1 - 1 - uidx[lofs[i]]));
        v = (long long)vals[j];
        if (u1 != uidx[j]) okey[out] = cu;
      }
    }
    const unsigned peers = __match_any_sync(kFull, out);
    if (on) {
      long long sum = 0;
      for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, v, __ffs(m) - 1);
      if (lane == __ffs(peers) - 1) atomicAdd(reinterpret_cast<unsigned long long *>(&oval[out]), (unsigned long long)sum);
    }
  }
}

__global__ void k_large_counts(const int32_t *list, const unsigned *count, const int64_t *uidx, const int64_t *lofs,
                               int64_t *rowcnt) {
  const unsigned cnt = *count;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    rowcnt[list[i]] = uidx[lofs[i + 1]] - uidx[lofs[i]];
}

__global__ void k_large_sizes(const int32_t *list, const unsigned *count, const int64_t *dsum, int64_t *sz) {
  const unsigned cnt = *count;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    sz[i] = dsum[list[i]];
}

// Compaction of the rows into the coarse CSR: a warp per row of at most kCompactLong entries; longer
// rows (the large clusters of power-law graphs) are cut into items of kCompactLong entries that the
// CTAs take in turn, so that no single warp copies a row of millions of entries.
constexpr int64_t kCompactLong = 4096;

__global__ void k_compact_rows(int64_t nc, const int64_t *tstart, const int64_t *rowcnt, const int64_t *off,
                               const int32_t *okey, const int64_t *oval, int32_t *adj, int64_t *ew) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = gw; c < nc; c += nw) {
    const int64_t src = tstart[c], dst = off[c], len = rowcnt[c];
    if (len > kCompactLong) continue;
    for (int64_t t = lane; t < len; t += 32) {
      adj[dst + t] = okey[src + t];
      ew[dst + t] = oval[src + t];
    }
  }
}

// the long rows among the large ones: (coarse id << 32) | item, at most cap items
__global__ void k_compact_list(const int32_t *list, const unsigned *count, const int64_t *rowcnt,
                               unsigned long long *items, unsigned long long cap, unsigned long long *nitems) {
  const unsigned cnt = *count;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const int c = list[i];
    const int64_t len = rowcnt[c];
    if (len <= kCompactLong) continue;
    const unsigned long long nch = (unsigned long long)((len + kCompactLong - 1) / kCompactLong);
    const unsigned long long base = atomicAdd(nitems, nch);
    for (unsigned long long x = 0; x < nch && base + x < cap; x++) items[base + x] = ((unsigned long long)c << 32) | x;
  }
}

__global__ void k_compact_items(const unsigned long long *items, unsigned long long cap, const unsigned long long *nitems,
                                const int64_t *tstart, const int64_t *rowcnt, const int64_t *off, const int32_t *okey,
                                const int64_t *oval, int32_t *adj, int64_t *ew) {
  const unsigned long long nit = min(*nitems, cap);
  for (unsigned long long it = blockIdx.x; it < nit; it += gridDim.x) {
    const int64_t c = (int64_t)(items[it] >> 32);
    const int64_t b = (int64_t)(items[it] & 0xffffffffull) * kCompactLong;
    const int64_t e = min(rowcnt[c], b + kCompactLong);
    const int64_t src = tstart[c], dst = off[c];
    for (int64_t t = b + threadIdx.x; t < e; t += blockDim.x) {
      adj[dst + t] = okey[src + t];
      ew[dst + t] = oval[src + t];
    }
  }
}

template <class K>
void set_smem(K kernel, int bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int EW>
int build_rows(RowArgs a, const unsigned *counts_dev, const unsigned counts[5], int32_t *lists[5], cudaStream_t s) {
  const int nsm = num_sms();
  auto grid_for = [&](int64_t items, int per_block, int limit) {
    int64_t g = (items + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, limit));
  };
  ProfScope ps("contract_rows", s);
  if (counts[0]) {
    RowArgs b = a;
    b.list = lists[0];
    b.count = counts_dev + 0;
    (::gp::count_launch(), k_row_warp<EW><<<grid_for(counts[0], 8, nsm * 16), 256, 0, s>>>(b));
  }
  if (counts[3]) {
    RowArgs b = a;
    b.list = lists[3];
    b.count = counts_dev + 3;
    const int sm = (kRowThreads / 32) * kWarpSlots * row_slot_bytes<EW>();
    set_smem(k_row_whash<EW, kWarpSlots>, sm);
    (::gp::count_launch(), k_row_whash<EW, kWarpSlots><<<grid_for(counts[3], 8, nsm * (EW == 0 ? 6 : 4)), kRowThreads, sm, s>>>(b));
  }
  if (counts[4]) {
    RowArgs b = a;
    b.list = lists[4];
    b.count = counts_dev + 4;
    constexpr int kBigSlots = 2 * kRowWarpBig;
    const int sm = 4 * kBigSlots * row_slot_bytes<EW>();  // 4 warps per CTA
    set_smem(k_row_whash<EW, kBigSlots>, sm);
    (::gp::count_launch(), k_row_whash<EW, kBigSlots><<<grid_for(counts[4], 4, nsm * (EW == 0 ? 3 : 2)), 128, sm, s>>>(b));
  }
  if (counts[1]) {
    RowArgs b = a;
    b.list = lists[1];
    b.count = counts_dev + 1;
    const int sm = kCtaSlots * 12;
    set_smem(k_row_cta<EW>, sm);
    (::gp::count_launch(), k_row_cta<EW><<<grid_for(counts[1], 1, nsm * 2), kRowThreads, sm, s>>>(b));
  }
  GP_LAUNCH_CHECK();
  return GP_OK;
}

}  // namespace

int alloc_graph(OwnedGraph *g, int64_t n, int64_t m, cudaStream_t s) {
  g->n = n;
  g->m = m;
  g->off_bytes = sizeof(int64_t) * (size_t)(n + 1);
  g->adj_bytes = sizeof(int32_t) * (size_t)std::max<int64_t>(m, 1);
  g->vw_bytes = sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1);
  g->ew_bytes = sizeof(int64_t) * (size_t)std::max<int64_t>(m, 1);
  g->off = (int64_t *)dev_alloc(g->off_bytes, s);
  g->adj = (int32_t *)dev_alloc(g->adj_bytes, s);
  g->vw = (int64_t *)dev_alloc(g->vw_bytes, s);
  g->ew = (int64_t *)dev_alloc(g->ew_bytes, s);
  if (!g->off || !g->adj || !g->vw || !g->ew) {
    g->release(s);
    set_error("device allocation for a coarse graph failed");
    return GP_ERR_OOM;
  }
  return GP_OK;
}

int contract_graph(const DGraph &g, const int32_t *labels, int64_t nl, OwnedGraph *out, int32_t *f2c_user,
                   cudaStream_t s, const LpConfig *cfg, LpClassInfo *cls) {
  Workspace ws(s);
  const int nsm = num_sms();
  const int64_t n = g.n;
  auto grid_n = [&](int64_t items) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, nsm * 8));
  };
  if (n == 0) {
    GP_TRY(alloc_graph(out, 0, 0, s));
    GP_CUDA(cudaMemsetAsync(out->off, 0, sizeof(int64_t), s));
    return GP_OK;
  }
  // 1. used flags -> new ids by an exclusive prefix sum
  uint32_t *used;
  int32_t *newid;
  int *bad;
  int64_t *hdr;  // [0] = n', [1] = m'
  GP_TRY(ws.zeros(&used, (size_t)nl));
  GP_TRY(ws.get(&newid, (size_t)nl));
  GP_TRY(ws.zeros(&bad, 1));
  GP_TRY(ws.zeros(&hdr, 4));
  (::gp::count_launch(), k_mark_used<<<grid_n(n), 256, 0, s>>>(labels, n, nl, used, bad));
  GP_LAUNCH_CHECK();
  GP_TRY(scan_excl_u32(used, newid, nl, hdr, ws));
  // The coarse vertex count nc = hdr[0] stays on the device until the read back after step 4: the
  // arrays indexed by coarse vertex are sized for the bound min(n, nl) (zero beyond nc, so the scans
  // over the bound equal the scans over nc) and the row classification reads nc on the device.
  const int64_t ncb = std::max<int64_t>(1, std::min<int64_t>(n, nl));
  // 2. fine -> coarse map, member counts, coarse vertex weights, degree sums
  int32_t *f2c = f2c_user;
  if (!f2c) GP_TRY(ws.get(&f2c, (size_t)n));
  int64_t *cnt, *dsum, *mstart, *tstart, *cw;
  GP_TRY(ws.zeros(&cnt, (size_t)ncb + 1));
  GP_TRY(ws.zeros(&dsum, (size_t)ncb + 1));
  GP_TRY(ws.zeros(&cw, (size_t)ncb));
  GP_TRY(ws.get(&mstart, (size_t)ncb + 1));
  GP_TRY(ws.get(&tstart, (size_t)ncb + 1));
  (::gp::count_launch(), k_f2c<<<grid_n(n), 256, 0, s>>>(g, labels, nl, newid, f2c, cnt, cw, dsum, bad));
  GP_LAUNCH_CHECK();
  GP_TRY(scan_excl_i64(cnt, mstart, ncb, mstart + ncb, ws));
  GP_TRY(scan_excl_i64(dsum, tstart, ncb, tstart + ncb, ws));
  // 3. members bucketed by coarse id
  unsigned *fill;
  int32_t *members;
  GP_TRY(ws.zeros(&fill, (size_t)ncb));
  GP_TRY(ws.get(&members, (size_t)n));
  (::gp::count_launch(), k_members<<<grid_n(n), 256, 0, s>>>(n, f2c, mstart, fill, members));
  // 4. rows binned by pair count
  int32_t *lists[5];
  unsigned *counts_dev;
  for (int b = 0; b < 5; b++) GP_TRY(ws.get(&lists[b], (size_t)ncb));
  GP_TRY(ws.zeros(&counts_dev, 5));
  (::gp::count_launch(), k_row_classify<<<grid_n(ncb), 256, 0, s>>>(hdr, dsum, lists[0], lists[1], lists[2],
                                                                     lists[3], lists[4], counts_dev));
  GP_LAUNCH_CHECK();
  unsigned long long *maxvw_dev;
  GP_TRY(ws.zeros(&maxvw_dev, 1));
  (::gp::count_launch(), k_max_i64<<<grid_n(ncb), 256, 0, s>>>(cw, ncb, maxvw_dev));
  unsigned counts[5];
  unsigned long long maxvw = 0;
  int64_t hh[4];
  int hbad = 0;
  {
    Readback rb;
    rb.add(hh, hdr, sizeof(hh));
    rb.add(&hbad, bad, sizeof(int));
    rb.add(counts, counts_dev, sizeof(counts));
    rb.add(&maxvw, maxvw_dev, sizeof(maxvw));
    GP_TRY(rb.run(s));
  }
  if (hbad) {
    set_error("contract: a label is outside [0, n)");
    return GP_ERR_INVALID_ARG;
  }
  const int64_t nc = hh[0];
  RowArgs a;
  a.g = g;
  a.f2c = f2c;
  a.mstart = mstart;
  a.members = members;
  a.tstart = tstart;
  a.dsum = dsum;
  int kb = 0;
  while (kb < 31 && ((int64_t)1 << kb) < nc) kb++;
  a.key_bits = kb;
  GP_TRY(ws.get(&a.okey, (size_t)std::max<int64_t>(g.m, 1)));
  GP_TRY(ws.get(&a.oval, (size_t)std::max<int64_t>(g.m, 1)));
  GP_TRY(ws.get(&a.rowcnt, (size_t)nc + 1));
  const int ew = g.ew_mode();
  if (counts[2]) {
    // very large rows: gather, sort by (row, neighbour), reduce
    ProfScope ps("contract_large_rows", s);
    const unsigned R = counts[2];
    int64_t *sz, *lofs;
    GP_TRY(ws.get(&sz, (size_t)R));
    GP_TRY(ws.get(&lofs, (size_t)R + 1));
    (::gp::count_launch(), k_large_sizes<<<grid_n(R), 256, 0, s>>>(lists[2], counts_dev + 2, dsum, sz));
    GP_TRY(scan_excl_i64(sz, lofs, R, lofs + R, ws));
    int64_t N = 0;
    GP_CUDA(cudaMemcpyAsync(&N, lofs + R, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    int32_t *large_idx;
    unsigned long long *lfill, *k0, *v0, *k1, *v1;
    GP_TRY(ws.get(&large_idx, (size_t)nc));
    GP_CUDA(cudaMemsetAsync(large_idx, 0xff, sizeof(int32_t) * (size_t)nc, s));
    GP_TRY(ws.zeros(&lfill, (size_t)R));
    GP_TRY(ws.get(&k0, (size_t)N));
    GP_TRY(ws.get(&v0, (size_t)N));
    GP_TRY(ws.get(&k1, (size_t)N));
    GP_TRY(ws.get(&v1, (size_t)N));
    (::gp::count_launch(), k_large_index<<<grid_n(R), 256, 0, s>>>(lists[2], counts_dev + 2, large_idx));
    int rb = 0;
    while (rb < 31 && ((int64_t)1 << rb) < (int64_t)R) rb++;
    const int kbits = std::max(kb, 1);
    if (ew == 0)
      (::gp::count_launch(), k_large_gather<0><<<grid_n(n * 32), 256, 0, s>>>(g, f2c, large_idx, lofs, lfill, kbits, k0, v0));
    else if (ew == 1)
      (::gp::count_launch(), k_large_gather<1><<<grid_n(n * 32), 256, 0, s>>>(g, f2c, large_idx, lofs, lfill, kbits, k0, v0));
    else
      (::gp::count_launch(), k_large_gather<2><<<grid_n(n * 32), 256, 0, s>>>(g, f2c, large_idx, lofs, lfill, kbits, k0, v0));
    GP_LAUNCH_CHECK();
    bool in_tmp = false;
    GP_TRY(radix_sort_pairs(k0, v0, k1, v1, N, rb + kbits, &in_tmp, ws));
    unsigned long long *ks = in_tmp ? k1 : k0, *vs = in_tmp ? v1 : v0;
    int64_t *flag, *uidx;
    GP_TRY(ws.get(&flag, (size_t)N));
    GP_TRY(ws.get(&uidx, (size_t)N + 1));
    (::gp::count_launch(), k_large_heads<<<grid_n(N), 256, 0, s>>>(ks, N, kbits, lists[2], flag));
    GP_TRY(scan_excl_i64(flag, uidx, N, uidx + N, ws));
    // (the large rows' weights are summed into zeroed slots)
    GP_CUDA(cudaMemsetAsync(a.oval, 0, sizeof(int64_t) * (size_t)std::max<int64_t>(g.m, 1), s));
    (::gp::count_launch(), k_large_write<<<grid_n(N), 256, 0, s>>>(ks, vs, N, kbits, lists[2], uidx, lofs, tstart,
                                                                   a.okey, a.oval));
    (::gp::count_launch(), k_large_counts<<<grid_n(R), 256, 0, s>>>(lists[2], counts_dev + 2, uidx, lofs, a.rowcnt));
    GP_LAUNCH_CHECK();
  }
  GP_TRY(ew == 0 ? build_rows<0>(a, counts_dev, counts, lists, s)
       : ew == 1 ? build_rows<1>(a, counts_dev, counts, lists, s)
                 : build_rows<2>(a, counts_dev, counts, lists, s));
  // 5. coarse offsets from the unique counts, then compaction of the rows
  int64_t mc = 0;
  int64_t *off_tmp;
  GP_TRY(ws.get(&off_tmp, (size_t)nc + 1));
  GP_TRY(scan_excl_i64(a.rowcnt, off_tmp, nc, off_tmp + nc, ws));
  // the next level's LP degree classes need only the coarse offsets: computed here and read back
  // with the coarse entry count
  unsigned long long *cls_dev = nullptr;
  unsigned long long cls_words[kLpClassWords];
  if (cfg && cls) {
    GP_TRY(ws.get(&cls_dev, (size_t)kLpClassWords));
    DGraph cg;
    cg.n = nc;
    cg.off = off_tmp;
    cg.off64 = 1;
    GP_TRY(lp_classes_launch(cg, *cfg, cls_dev, ws));
  }
  {
    Readback rb;
    rb.add(&mc, off_tmp + nc, sizeof(int64_t));
    if (cls_dev) rb.add(cls_words, cls_dev, sizeof(cls_words));
    GP_TRY(rb.run(s));
  }
  if (cls_dev) lp_classes_from(cls_words, *cfg, cls);
  GP_TRY(alloc_graph(out, nc, mc, s));
  out->max_vw = (int64_t)maxvw;
  GP_CUDA(cudaMemcpyAsync(out->off, off_tmp, sizeof(int64_t) * (size_t)(nc + 1), cudaMemcpyDeviceToDevice, s));
  GP_CUDA(cudaMemcpyAsync(out->vw, cw, sizeof(int64_t) * (size_t)nc, cudaMemcpyDeviceToDevice, s));
  {
    ProfScope ps("contract_compact", s);
    (::gp::count_launch(), k_compact_rows<<<grid_n(nc * 32), 256, 0, s>>>(nc, tstart, a.rowcnt, out->off, a.okey, a.oval, out->adj, out->ew));
    if (counts[2]) {
      // items: at most one per kCompactLong coarse entries plus one per large row
      const unsigned long long cap = (unsigned long long)(mc / kCompactLong + counts[2] + 1);
      unsigned long long *items, *nitems;
      GP_TRY(ws.get(&items, (size_t)cap));
      GP_TRY(ws.zeros(&nitems, 1));
      (::gp::count_launch(), k_compact_list<<<grid_n(counts[2]), 256, 0, s>>>(lists[2], counts_dev + 2, a.rowcnt, items,
                                                                              cap, nitems));
      (::gp::count_launch(), k_compact_items<<<num_sms() * 8, 256, 0, s>>>(items, cap, nitems, tstart, a.rowcnt,
                                                                         out->off, a.okey, a.oval, out->adj, out->ew));
    }
  }
  GP_LAUNCH_CHECK();
  if (profiling()) {
    const int64_t rb = n * 2 * g.offset_bytes() + g.m * (4 + g.ew_bytes()) + g.m * 4;
    prof_add_counts("contract_rows", nc, g.m, rb);
    prof_add_counts("contract_compact", nc, mc, mc * 12 + nc * 8);
  }
  return GP_OK;  // stream-ordered: the temporary buffers are released on s after the kernels
}

}  // namespace gp
