// mls.cu -- multi-try k-way local search (MLS) on the GPU, after label-propagation refinement.
//
// Section III-C: localized k-way searches, each started from a single boundary vertex of a todo list,
// move the vertex of largest gain from a priority queue seeded with the start vertex and its
// neighbours, queue the neighbours of moved vertices, respect the balance bound and keep the best
// prefix of their moves. Section IV-C, Algorithm 1 (PerformMoves / ApplyMoves): searches run in
// parallel on the partition of the local iteration's start and only record their moves; the recorded
// sequences are then applied one after another with every gain recomputed on the current partition,
// each sequence up to its best prefix. Local iterations repeat on the moved vertices while their gain
// exceeds alpha of the global iteration's gain; global iterations restart from all boundary vertices.
//
// GPU form:
//   * PerformMoves: one warp per search, all searches of a local iteration in one launch. A warp keeps
//     its whole search state in shared memory: the queue (an unsorted array; the maximum is found by a
//     warp reduction over (gain, H(s, w, 0), -w)), its moves and a small hash map of the blocks they
//     changed (the search's view of the partition), its copy of the block weights, and a per-block
//     connection array for gain computations (each lane adds its neighbours' weights with shared-memory
//     atomics, then the lanes reduce over the blocks). Each search writes its best prefix to its own
//     slot range, so the sequences keep the todo order.
//   * ApplyMoves: one CTA walks the sequences in todo order (the non-empty ones found 256 at a time by a
//     block scan), recomputes each move's gain with a block-wide sum over the vertex's row, and applies
//     the best prefix; block weights live in shared memory.
//   * Todo lists: boundary (or moved) flags compacted in vertex order, then a stable radix sort by
//     H(s, v, 1) -- the order the oracle uses.
// The readings the paper leaves open (fixed search bounds instead of the adaptive stopping rule, no
// global moved bitmap during a local iteration, the degree bound, the hash orders) are those of the
// CPU oracle; results are bit-identical to it.
#include <algorithm>
#include <vector>

#include "gp_internal.cuh"
#include "mls.cuh"
#include "sort.cuh"

namespace gp {
namespace {

constexpr int kMlsWarps = 4;
constexpr int kMlsThreads = kMlsWarps * 32;
constexpr int kMaxMoves = 64;
constexpr int kQCap = 256;
constexpr int kMaxK = 256;
constexpr int kMovedSlots = 128;  // hash map of moved vertices (at most kMaxMoves entries)
constexpr int kApplyThreads = 256;

struct WarpState {
  long long qg[kQCap];
  unsigned long long qh[kQCap];
  long long bw[kMaxK];
  long long conn[kMaxK];
  int qv[kQCap];
  int mv[kMaxMoves], mto[kMaxMoves], mfrom[kMaxMoves];
  int hk[kMovedSlots], hb[kMovedSlots];
  int qn, nm;
};

struct MlsArgs {
  DGraph g;
  const int32_t *part;
  const int64_t *bw;  // block weights at the local iteration's start
  int k;
  int64_t lmax;
  uint64_t smix;  // mix64(s)
  int max_moves, fruitless, queue_cap, max_degree;
};

__device__ __forceinline__ uint64_t hkey(uint64_t smix, uint64_t a, uint64_t b) { return mix64(mix64(smix ^ a) ^ b); }

__device__ __forceinline__ int moved_block(const WarpState &W, int u) {
  unsigned sl = mix32((unsigned)u) & (kMovedSlots - 1);
  while (true) {
    const int key = W.hk[sl];
    if (key == u) return W.hb[sl];
    if (key < 0) return -1;
    sl = (sl + 1) & (kMovedSlots - 1);
  }
}

__device__ __forceinline__ int view_block(const MlsArgs &A, const WarpState &W, int u) {
  const int b = W.nm ? moved_block(W, u) : -1;
  return b >= 0 ? b : A.part[u];
}

__device__ __forceinline__ int64_t degree_of(const DGraph &g, int v) { return g.row_begin(v + 1) - g.row_begin(v); }

// Best move of x in the warp's view (all lanes call; results are uniform). Returns movable.
template <int EW>
__device__ bool gain_of(const MlsArgs &A, WarpState &W, int x, int *to_out, long long *gain_out) {
  const int lane = threadIdx.x & 31;
  for (int b = lane; b < A.k; b += 32) W.conn[b] = 0;
  __syncwarp();
  const int64_t rb = A.g.row_begin(x), re = A.g.row_begin(x + 1);
  for (int64_t e = rb + lane; e < re; e += 32) {
    const int u = __ldg(A.g.adj + e);
    atomicAdd(reinterpret_cast<unsigned long long *>(&W.conn[view_block(A, W, u)]),
              (unsigned long long)load_ew<EW>(A.g.ew, e));
  }
  __syncwarp();
  const int a = view_block(A, W, x);
  const long long cx = A.g.vweight(x);
  const uint64_t hx = mix64(A.smix ^ (uint64_t)(uint32_t)x);
  long long bc = -1;
  uint64_t bh = 0;
  int bb = -1;
  for (int b = lane; b < A.k; b += 32) {
    const long long c = W.conn[b];
    if (b == a || c <= 0 || W.bw[b] + cx > A.lmax) continue;
    const uint64_t h = mix64(hx ^ (uint64_t)b);
    if (bb < 0 || c > bc || (c == bc && (h > bh || (h == bh && b < bb)))) {
      bc = c;
      bh = h;
      bb = b;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long c2 = __shfl_xor_sync(kFull, bc, o);
    const uint64_t h2 = __shfl_xor_sync(kFull, bh, o);
    const int b2 = __shfl_xor_sync(kFull, bb, o);
    if (b2 >= 0 && (bb < 0 || c2 > bc || (c2 == bc && (h2 > bh || (h2 == bh && b2 < bb))))) {
      bc = c2;
      bh = h2;
      bb = b2;
    }
  }
  const long long own = W.conn[a];
  __syncwarp();
  if (bb < 0) return false;
  *to_out = bb;
  *gain_out = bc - own;
  return true;
}

__device__ __forceinline__ int queue_find(const WarpState &W, int x) {
  int at = -1;
  for (int base = 0; base < W.qn; base += 32) {
    const int i = base + (threadIdx.x & 31);
    const unsigned m = __ballot_sync(kFull, i < W.qn && W.qv[i] == x);
    if (m) {
      at = base + __ffs(m) - 1;
      break;
    }
  }
  return at;
}

__device__ __forceinline__ void queue_remove(WarpState &W, int i) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    const int last = W.qn - 1;
    W.qv[i] = W.qv[last];
    W.qg[i] = W.qg[last];
    W.qh[i] = W.qh[last];
    W.qn = last;
  }
  __syncwarp();
}

template <int EW>
__device__ void try_insert(const MlsArgs &A, WarpState &W, int x) {
  if (degree_of(A.g, x) > A.max_degree) return;
  if (W.nm && moved_block(W, x) >= 0) return;
  if (queue_find(W, x) >= 0) return;
  if (W.qn >= A.queue_cap) return;
  int to;
  long long gain;
  if (!gain_of<EW>(A, W, x, &to, &gain)) return;
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    W.qv[W.qn] = x;
    W.qg[W.qn] = gain;
    W.qh[W.qn] = hkey(A.smix, (uint64_t)(uint32_t)x, 0);
    W.qn += 1;
  }
  __syncwarp();
}

// PerformMoves: one warp per todo vertex; seq[i * max_moves + j] = (vertex, from, to) of the best prefix,
// len[i] its length.
template <int EW>
__global__ void __launch_bounds__(kMlsThreads) k_mls_search(MlsArgs A, const int32_t *todo, int64_t m, int3 *seq,
                                                            int32_t *len) {
  extern __shared__ __align__(16) unsigned char smem[];
  WarpState &W = reinterpret_cast<WarpState *>(smem)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * kMlsWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kMlsWarps;
  for (int64_t i = gw; i < m; i += nw) {
    const int v = todo[i];
    const int64_t dv = degree_of(A.g, v);
    if (dv == 0 || dv > A.max_degree) {
      if (lane == 0) len[i] = 0;
      continue;
    }
    for (int b = lane; b < A.k; b += 32) W.bw[b] = A.bw[b];
    for (int t = lane; t < kMovedSlots; t += 32) W.hk[t] = -1;
    if (lane == 0) {
      W.qn = 0;
      W.nm = 0;
    }
    __syncwarp();
    try_insert<EW>(A, W, v);
    for (int64_t e = A.g.row_begin(v); e < A.g.row_begin(v + 1); e++) try_insert<EW>(A, W, __ldg(A.g.adj + e));
    long long cum = 0, best = 0;
    int best_len = 0, fruitless = 0;
    while (W.qn > 0 && W.nm < A.max_moves) {
      // the queue's maximum by (gain, hash, -vertex)
      long long bg = 0;
      uint64_t bh = 0;
      int bx = -1, bi = -1;
      for (int j = lane; j < W.qn; j += 32) {
        const long long gq = W.qg[j];
        const uint64_t hq = W.qh[j];
        const int xq = W.qv[j];
        if (bi < 0 || gq > bg || (gq == bg && (hq > bh || (hq == bh && xq < bx)))) {
          bg = gq;
          bh = hq;
          bx = xq;
          bi = j;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long g2 = __shfl_xor_sync(kFull, bg, o);
        const uint64_t h2 = __shfl_xor_sync(kFull, bh, o);
        const int x2 = __shfl_xor_sync(kFull, bx, o);
        const int i2 = __shfl_xor_sync(kFull, bi, o);
        if (i2 >= 0 && (bi < 0 || g2 > bg || (g2 == bg && (h2 > bh || (h2 == bh && x2 < bx))))) {
          bg = g2;
          bh = h2;
          bx = x2;
          bi = i2;
        }
      }
      const int x = bx;
      queue_remove(W, bi);
      int to;
      long long gain;
      if (!gain_of<EW>(A, W, x, &to, &gain)) continue;
      const int a = view_block(A, W, x);
      const long long cx = A.g.vweight(x);
      __syncwarp();
      if (lane == 0) {
        const int j = W.nm;
        W.mv[j] = x;
        W.mfrom[j] = a;
        W.mto[j] = to;
        unsigned sl = mix32((unsigned)x) & (kMovedSlots - 1);
        while (W.hk[sl] >= 0) sl = (sl + 1) & (kMovedSlots - 1);
        W.hk[sl] = x;
        W.hb[sl] = to;
        W.bw[a] -= cx;
        W.bw[to] += cx;
        W.nm = j + 1;
      }
      __syncwarp();
      cum += gain;
      if (cum > best) {
        best = cum;
        best_len = W.nm;
        fruitless = 0;
      } else if (++fruitless >= A.fruitless) {
        break;
      }
      for (int64_t e = A.g.row_begin(x); e < A.g.row_begin(x + 1); e++) {
        const int u = __ldg(A.g.adj + e);
        if (degree_of(A.g, u) > A.max_degree || moved_block(W, u) >= 0) continue;
        const int j = queue_find(W, u);
        if (j >= 0) {
          int tu;
          long long gu;
          if (gain_of<EW>(A, W, u, &tu, &gu)) {
            __syncwarp();
            if (lane == 0) W.qg[j] = gu;
            __syncwarp();
          } else {
            queue_remove(W, j);
          }
        } else {
          try_insert<EW>(A, W, u);
        }
      }
    }
    const int L = best > 0 ? best_len : 0;
    for (int j = lane; j < L; j += 32) seq[i * A.max_moves + j] = make_int3(W.mv[j], W.mfrom[j], W.mto[j]);
    if (lane == 0) len[i] = L;
    __syncwarp();
  }
}

__device__ __forceinline__ long long block_sum_ll(long long x, long long *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  long long t = 0;
  for (int w = 0; w < kApplyThreads / 32; w++) t += red[w];
  __syncthreads();
  return t;
}

// ApplyMoves: one CTA, sequences in todo order. out[0] += gain, out[1] += applied moves.
template <int EW>
__global__ void __launch_bounds__(kApplyThreads) k_mls_apply(DGraph g, int32_t *part, int64_t *bw_g, int k,
                                                             int64_t lmax, const int3 *seq, const int32_t *len,
                                                             int64_t m, int max_moves, uint32_t *moved,
                                                             long long *out) {
  __shared__ long long bw[kMaxK];
  __shared__ long long red[kApplyThreads / 32];
  __shared__ int idx[kApplyThreads];
  __shared__ int nidx;
  __shared__ int ok;
  __shared__ long long cum, best, gain_total, moves_total;
  __shared__ int best_len, napplied;
  for (int b = threadIdx.x; b < k; b += kApplyThreads) bw[b] = bw_g[b];
  if (threadIdx.x == 0) {
    gain_total = 0;
    moves_total = 0;
  }
  __syncthreads();
  for (int64_t base = 0; base < m; base += kApplyThreads) {
    const int64_t i = base + threadIdx.x;
    const bool ne = i < m && len[i] > 0;
    if (threadIdx.x == 0) nidx = 0;
    __syncthreads();
    // the non-empty sequences of this tile, in order
    const unsigned bal = __ballot_sync(kFull, ne);
    __shared__ int wbase[kApplyThreads / 32];
    if ((threadIdx.x & 31) == 0) wbase[threadIdx.x >> 5] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int s = 0;
      for (int w = 0; w < kApplyThreads / 32; w++) {
        const int c = wbase[w];
        wbase[w] = s;
        s += c;
      }
      nidx = s;
    }
    __syncthreads();
    if (ne) idx[wbase[threadIdx.x >> 5] + __popc(bal & lanemask_lt())] = (int)threadIdx.x;
    __syncthreads();
    for (int q = 0; q < nidx; q++) {
      const int64_t si = base + idx[q];
      const int L = len[si];
      if (threadIdx.x == 0) {
        cum = 0;
        best = 0;
        best_len = 0;
        napplied = 0;
      }
      __syncthreads();
      for (int j = 0; j < L; j++) {
        const int3 mvj = seq[si * max_moves + j];
        const int w = mvj.x, from = mvj.y, to = mvj.z;
        const long long cw = g.vweight(w);
        if (threadIdx.x == 0) ok = !(moved[w] || part[w] != from || bw[to] + cw > lmax);
        __syncthreads();
        if (!ok) break;
        long long gsum = 0;
        for (int64_t e = g.row_begin(w) + threadIdx.x; e < g.row_begin(w + 1); e += kApplyThreads) {
          const int b = part[__ldg(g.adj + e)];
          const long long we = load_ew<EW>(g.ew, e);
          if (b == to) gsum += we;
          if (b == from) gsum -= we;
        }
        gsum = block_sum_ll(gsum, red);
        if (threadIdx.x == 0) {
          part[w] = to;
          bw[from] -= cw;
          bw[to] += cw;
          napplied = j + 1;
          cum += gsum;
          if (cum > best) {
            best = cum;
            best_len = j + 1;
          }
        }
        __syncthreads();
      }
      // roll back the moves after the best prefix, mark the applied ones
      if (threadIdx.x == 0) {
        for (int j = napplied - 1; j >= best_len; j--) {
          const int3 mvj = seq[si * max_moves + j];
          const long long cw = g.vweight(mvj.x);
          part[mvj.x] = mvj.y;
          bw[mvj.z] -= cw;
          bw[mvj.y] += cw;
        }
        for (int j = 0; j < best_len; j++) moved[seq[si * max_moves + j].x] = 1;
        gain_total += best;
        moves_total += best_len;
      }
      __syncthreads();
    }
  }
  for (int b = threadIdx.x; b < k; b += kApplyThreads) bw_g[b] = bw[b];
  if (threadIdx.x == 0) {
    out[0] += gain_total;
    out[1] += moves_total;
  }
}

__global__ void k_boundary_flags(DGraph g, const int32_t *part, int max_degree, uint32_t *flags) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rb = g.row_begin(v), re = g.row_begin(v + 1);
    uint32_t f = 0;
    if (re - rb <= max_degree) {
      const int a = part[v];
      for (int64_t e = rb; e < re; e++)
        if (part[g.adj[e]] != a) {
          f = 1;
          break;
        }
    }
    flags[v] = f;
  }
}

// keys[r] = H(s, v, 1), vals[r] = v for every flagged v at rank r (ranks in vertex order)
__global__ void k_todo_keys(int64_t n, const uint32_t *flags, const int32_t *rank, uint64_t smix,
                            unsigned long long *keys, unsigned long long *vals) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (!flags[v]) continue;
    keys[rank[v]] = hkey(smix, (uint64_t)v, 1);
    vals[rank[v]] = (unsigned long long)v;
  }
}

__global__ void k_vals_to_i32(const unsigned long long *vals, int64_t m, int32_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)vals[i];
}

__global__ void k_mls_block_weights(DGraph g, const int32_t *part, int64_t *bw) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long *>(&bw[part[v]]), (unsigned long long)g.vweight(v));
}

int grid_of(int64_t items, int threads) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + threads - 1) / threads, (int64_t)num_sms() * 8));
}

// todo = flagged vertices ordered by H(s, v, 1) (ties: smaller v); returns the count via *m_out
int build_todo(int64_t n, uint32_t *flags, uint64_t s, int32_t *rank, unsigned long long *keys,
               unsigned long long *vals, unsigned long long *keys2, unsigned long long *vals2, int32_t *todo,
               int64_t *m_out, Workspace &ws) {
  cudaStream_t st = ws.stream();
  int64_t *tot;
  GP_TRY(ws.get(&tot, 1));
  GP_TRY(scan_excl_u32(flags, rank, n, tot, ws));
  int64_t m = 0;
  GP_CUDA(cudaMemcpyAsync(&m, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaStreamSynchronize(st));
  *m_out = m;
  if (m == 0) return GP_OK;
  (count_launch(), k_todo_keys<<<grid_of(n, 256), 256, 0, st>>>(n, flags, rank, mix64(s), keys, vals));
  GP_LAUNCH_CHECK();
  bool in_tmp = false;
  GP_TRY(radix_sort_pairs(keys, vals, keys2, vals2, m, 64, &in_tmp, ws));
  (count_launch(), k_vals_to_i32<<<grid_of(m, 256), 256, 0, st>>>(in_tmp ? vals2 : vals, m, todo));
  GP_LAUNCH_CHECK();
  return GP_OK;
}

}  // namespace

void mls_default_params(MlsParams *p) {
  p->global_iters = 3;
  p->alpha_pct = 10;
  p->max_local = 16;
  p->max_moves = 64;
  p->fruitless = 16;
  p->queue_cap = 256;
  p->max_degree = 1024;
}

int run_mls(const DGraph &g, int k, int64_t lmax, uint64_t seed, const MlsParams &p, int32_t *part, MlsStats *out,
            cudaStream_t s) {
  if (out) *out = MlsStats();
  if (g.n <= 0 || p.global_iters <= 0) return GP_OK;
  if (k > kMaxK || p.max_moves < 1 || p.max_moves > kMaxMoves || p.queue_cap < 1 || p.queue_cap > kQCap ||
      p.fruitless < 1 || p.max_degree < 0) {
    set_error("multi-try local search: k <= 256, 1 <= max_moves <= 64, 1 <= queue_cap <= 256, fruitless >= 1");
    return GP_ERR_UNSUPPORTED;
  }
  Workspace ws(s);
  const int64_t n = g.n;
  uint32_t *flags;
  int32_t *rank, *todo, *len;
  unsigned long long *keys, *vals, *keys2, *vals2;
  int64_t *bw;
  long long *acc;
  int3 *seq;
  GP_TRY(ws.get(&flags, (size_t)n));
  GP_TRY(ws.get(&rank, (size_t)n));
  GP_TRY(ws.get(&todo, (size_t)n));
  GP_TRY(ws.get(&len, (size_t)n));
  GP_TRY(ws.get(&keys, (size_t)n));
  GP_TRY(ws.get(&vals, (size_t)n));
  GP_TRY(ws.get(&keys2, (size_t)n));
  GP_TRY(ws.get(&vals2, (size_t)n));
  GP_TRY(ws.zeros(&bw, (size_t)k));
  GP_TRY(ws.zeros(&acc, 2));
  const int gn = grid_of(n, 256);
  (count_launch(), k_mls_block_weights<<<gn, 256, 0, s>>>(g, part, bw));
  GP_LAUNCH_CHECK();
  const size_t smem = sizeof(WarpState) * kMlsWarps;
  const int ew = g.ew_mode();
  static bool attr_set[3] = {false, false, false};
  if (!attr_set[ew]) {
    if (ew == 0) GP_CUDA(cudaFuncSetAttribute(k_mls_search<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (ew == 1) GP_CUDA(cudaFuncSetAttribute(k_mls_search<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (ew == 2) GP_CUDA(cudaFuncSetAttribute(k_mls_search<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set[ew] = true;
  }
  MlsStats st;
  size_t seq_cap = 0;
  for (int gi = 0; gi < p.global_iters; gi++) {
    uint64_t sl = hash3(seed, (uint64_t)gi, 5);
    (count_launch(), k_boundary_flags<<<gn, 256, 0, s>>>(g, part, (int)p.max_degree, flags));
    GP_LAUNCH_CHECK();
    int64_t m = 0;
    GP_TRY(build_todo(n, flags, sl, rank, keys, vals, keys2, vals2, todo, &m, ws));
    int64_t total = 0;
    for (int li = 0; li < p.max_local && m > 0; li++) {
      if ((size_t)m * p.max_moves > seq_cap) {
        seq_cap = (size_t)m * p.max_moves;
        GP_TRY(ws.get(&seq, seq_cap));
      }
      MlsArgs A;
      A.g = g;
      A.part = part;
      A.bw = bw;
      A.k = k;
      A.lmax = lmax;
      A.smix = mix64(sl);
      A.max_moves = (int)p.max_moves;
      A.fruitless = (int)p.fruitless;
      A.queue_cap = (int)p.queue_cap;
      A.max_degree = (int)p.max_degree;
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((m + kMlsWarps - 1) / kMlsWarps,
                                                                    (int64_t)num_sms() * 8));
      {
        ProfScope ps("mls_search", s);
        if (ew == 0) (count_launch(), k_mls_search<0><<<grid, kMlsThreads, smem, s>>>(A, todo, m, seq, len));
        else if (ew == 1) (count_launch(), k_mls_search<1><<<grid, kMlsThreads, smem, s>>>(A, todo, m, seq, len));
        else (count_launch(), k_mls_search<2><<<grid, kMlsThreads, smem, s>>>(A, todo, m, seq, len));
        GP_LAUNCH_CHECK();
      }
      GP_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (size_t)n, s));  // now: moved in this local iteration
      GP_CUDA(cudaMemsetAsync(acc, 0, sizeof(long long) * 2, s));
      {
        ProfScope ps("mls_apply", s);
        if (ew == 0) (count_launch(), k_mls_apply<0><<<1, kApplyThreads, 0, s>>>(g, part, bw, k, lmax, seq, len, m, (int)p.max_moves, flags, acc));
        else if (ew == 1) (count_launch(), k_mls_apply<1><<<1, kApplyThreads, 0, s>>>(g, part, bw, k, lmax, seq, len, m, (int)p.max_moves, flags, acc));
        else (count_launch(), k_mls_apply<2><<<1, kApplyThreads, 0, s>>>(g, part, bw, k, lmax, seq, len, m, (int)p.max_moves, flags, acc));
        GP_LAUNCH_CHECK();
      }
      long long h[2];
      GP_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaStreamSynchronize(s));
      st.searches += m;
      st.moves += h[1];
      st.local_iters += 1;
      const int64_t gain = h[0];
      const bool more = gain > 0 && 100 * gain > p.alpha_pct * total;
      total += gain;
      if (!more) break;
      sl = hash3(sl, (uint64_t)li + 1, 6);
      GP_TRY(build_todo(n, flags, sl, rank, keys, vals, keys2, vals2, todo, &m, ws));
    }
    st.gain += total;
  }
  if (out) *out = st;
  return GP_OK;
}

}  // namespace gp
