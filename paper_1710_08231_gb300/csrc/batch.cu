// batch.cu -- partitioning many independent graphs together.
//
// The graphs are stored as one disjoint union (vertex ids offset per graph) and the multilevel scheme
// runs once on the union: contraction, degree-0 stripping, projection and evaluation need nothing
// special because clusters never span graphs and contraction keeps every graph's vertices contiguous
// and in order. Label propagation and initial partitioning run each graph as an independent problem of
// a shared launch, with the graph's own seeds, bounds and local ids, so every graph is partitioned
// exactly as gp_partition would partition it alone. A graph that has finished coarsening passes
// through the remaining levels unchanged (its vertices keep their own labels) and is refined only at
// its own levels.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "contract.cuh"
#include "gp_internal.cuh"
#include "ip.cuh"
#include "lp.cuh"
#include "mlp.cuh"

namespace gp {
LpConfig schedule_for_batch(const gp_params *p);

namespace {

struct BatchDesc {
  const void *off;
  const int32_t *adj;
  const void *vw;
  const void *ew;
  int off64, vw64, ew64, pad;
  int64_t n, m;
};

__device__ __forceinline__ int find_graph(const int64_t *base, int count, int64_t x) {
  int lo = 0, hi = count;  // largest i with base[i] <= x
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (base[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Warp-aggregated atomics: every lane calls; lanes with `on` add (or max/min) their value into the
// element at `addr`, one atomic per distinct address in the warp. Graphs of a union are contiguous,
// so the 32 vertices of a warp mostly update the same per-graph counter.
__device__ __forceinline__ void wadd(unsigned long long *addr, bool on, unsigned long long val) {
  const unsigned peers = __match_any_sync(kFull, on ? (unsigned long long)addr : 0ull);
  if (!on) return;
  unsigned long long sum = 0;
  for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, val, __ffs(m) - 1);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1 && sum) atomicAdd(addr, sum);
}
__device__ __forceinline__ void wmax(unsigned long long *addr, bool on, unsigned long long val) {
  const unsigned peers = __match_any_sync(kFull, on ? (unsigned long long)addr : 0ull);
  if (!on) return;
  unsigned long long mx = 0;
  for (unsigned m = peers; m; m &= m - 1) mx = max(mx, __shfl_sync(peers, val, __ffs(m) - 1));
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(addr, mx);
}
__device__ __forceinline__ void wmin(unsigned long long *addr, bool on, unsigned long long val) {
  const unsigned peers = __match_any_sync(kFull, on ? (unsigned long long)addr : 0ull);
  if (!on) return;
  unsigned long long mn = ~0ull;
  for (unsigned m = peers; m; m &= m - 1) mn = min(mn, __shfl_sync(peers, val, __ffs(m) - 1));
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicMin(addr, mn);
}

// Grid-stride loop in which every lane of a warp runs the same iterations (warp collectives inside).
#define FOR_WARP_UNIFORM(i, n, valid)                                                                     \
  for (int64_t i##0 = blockIdx.x * (int64_t)blockDim.x; i##0 < (n); i##0 += (int64_t)gridDim.x * blockDim.x) \
    for (int64_t i = i##0 + threadIdx.x, valid = i < (n); valid >= 0; valid = -1)

__global__ void k_union_rows(const BatchDesc *d, int count, const int64_t *vb, const int64_t *eb, int64_t N,
                             int64_t *off, int64_t *vw, bool want_vw) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int gi = find_graph(vb, count, v);
    const int64_t l = v - vb[gi];
    const BatchDesc D = d[gi];
    const int64_t o = D.off64 ? static_cast<const int64_t *>(D.off)[l] : (int64_t) static_cast<const int32_t *>(D.off)[l];
    off[v] = eb[gi] + o;
    if (want_vw) {
      vw[v] = D.vw ? (D.vw64 ? static_cast<const int64_t *>(D.vw)[l] : (int64_t) static_cast<const int32_t *>(D.vw)[l]) : 1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) off[N] = eb[count];
}

__global__ void k_union_entries(const BatchDesc *d, int count, const int64_t *vb, const int64_t *eb, int64_t M,
                                int32_t *adj, int64_t *ew, bool want_ew) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M; e += (int64_t)gridDim.x * blockDim.x) {
    const int gi = find_graph(eb, count, e);
    const int64_t l = e - eb[gi];
    const BatchDesc D = d[gi];
    adj[e] = (int32_t)(D.adj[l] + vb[gi]);
    if (want_ew) {
      ew[e] = D.ew ? (D.ew64 ? static_cast<const int64_t *>(D.ew)[l] : (int64_t) static_cast<const int32_t *>(D.ew)[l]) : 1;
    }
  }
}

// out[i] = src[idx[i]] (idx[i] may equal the array length; then out[i] = tail)
__global__ void k_gather_at(const int32_t *src, const int64_t *idx, int count, int64_t len, int64_t tail, int64_t *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = idx[i] >= len ? tail : (int64_t)src[idx[i]];
}

// first[gi] = smallest coarse id of graph gi's vertices (coarse ids of one graph are contiguous, and
// below those of the next graph, but f2c of the graph's first vertex need not be the smallest)
__global__ void k_graph_first(const int32_t *f2c, const int64_t *vb, int count, int64_t n, unsigned long long *first) {
  FOR_WARP_UNIFORM(v, n, ok) {
    const int gi = ok ? find_graph(vb, count, v) : 0;
    wmin(&first[gi], ok, ok ? (unsigned long long)f2c[v] : 0);
  }
}

__global__ void k_gather_off(const int64_t *off, const int64_t *idx, int count, int64_t *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) out[i] = off[idx[i]];
}

__global__ void k_graph_vstats(DGraph g, const int64_t *vb, int count, unsigned long long *maxc,
                               unsigned long long *wsum) {
  FOR_WARP_UNIFORM(v, g.n, ok) {
    const int gi = ok ? find_graph(vb, count, v) : 0;
    const unsigned long long c = ok ? (unsigned long long)g.vweight(v) : 0;
    if (maxc) wmax(&maxc[gi], ok, c);
    if (wsum) wadd(&wsum[gi], ok, c);
  }
}

__global__ void k_iota_i32(int32_t *x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (int32_t)i;
}

__global__ void k_vw_i64(DGraph g, int64_t *out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = g.vweight(v);
}

// Block weights and cut of every (graph, try) partition of the coarsest union level.
struct TryEval {
  int32_t *parts;   // tries * n of the graph
  int64_t n, vbase;
  int k;
  int64_t *bw;      // tries * k
};

__global__ void k_try_eval(DGraph g, const int64_t *vb, int count, const TryEval *te, int tries,
                           unsigned long long *cut2) {
  FOR_WARP_UNIFORM(v, g.n, ok) {
    const int gi = ok ? find_graph(vb, count, v) : 0;
    const TryEval T = te[gi];
    const int64_t l = v - T.vbase;
    for (int t = 0; t < tries; t++) {
      const int32_t *p = T.parts + (size_t)t * T.n;
      const int pv = ok ? p[l] : 0;
      wadd(reinterpret_cast<unsigned long long *>(&T.bw[(size_t)t * T.k + pv]), ok,
           ok ? (unsigned long long)g.vweight(v) : 0);
      if (!cut2) continue;
      long long c = 0;
      if (ok)
        for (int64_t j = g.row_begin(v); j < g.row_begin(v + 1); j++)
          if (p[g.adj[j] - T.vbase] != pv) c += g.eweight(j);
      wadd(&cut2[(size_t)gi * tries + t], ok && c, (unsigned long long)c);
    }
  }
}

// Union partition (local block ids) -> per-graph block weights (bwoff[gi] .. + k_gi) and doubled cuts.
__global__ void k_union_eval(DGraph g, const int64_t *vb, int count, const int32_t *part, const int64_t *bwoff,
                             int64_t *bw, unsigned long long *cut2) {
  FOR_WARP_UNIFORM(v, g.n, ok) {
    const int gi = ok ? find_graph(vb, count, v) : 0;
    const int pv = ok ? part[v] : 0;
    wadd(reinterpret_cast<unsigned long long *>(&bw[bwoff[gi] + pv]), ok, ok ? (unsigned long long)g.vweight(v) : 0);
    if (cut2) {
      long long c = 0;
      if (ok)
        for (int64_t j = g.row_begin(v); j < g.row_begin(v + 1); j++)
          if (part[g.adj[j]] != pv) c += g.eweight(j);
      wadd(&cut2[gi], ok && c, (unsigned long long)c);
    }
  }
}

// Copies each graph's best try into the union partition of the coarsest level.
__global__ void k_pick_tries(const int64_t *vb, int count, int64_t N, const TryEval *te, const int *best,
                             int32_t *part) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int gi = find_graph(vb, count, v);
    const TryEval T = te[gi];
    part[v] = T.parts[(size_t)best[gi] * T.n + (v - T.vbase)];
  }
}

// Degree-0 vertices of every graph (unit weights): water-filling of the graph's kept block weights.
__global__ void k_batch_place(DGraph g0, const int64_t *vb, int count, const int32_t *rank, const int64_t *rank_at_vb,
                              const int32_t *part_stripped, const int64_t *bwoff, const int64_t *bw, const int *kk,
                              int32_t *part) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g0.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int gi = find_graph(vb, count, v);
    const int64_t d = g0.row_begin(v + 1) - g0.row_begin(v);
    if (d > 0) {
      part[v] = part_stripped[rank[v]];
      continue;
    }
    const long long j = (long long)(v - vb[gi]) - ((long long)rank[v] - rank_at_vb[gi]);
    const int64_t *b = bw + bwoff[gi];
    const int k = kk[gi];
    long long bmin = LLONG_MAX;
    for (int x = 0; x < k; x++) bmin = min(bmin, (long long)b[x]);
    auto F = [&](long long xl) {
      long long s = 0;
      for (int x = 0; x < k; x++) s += xl > b[x] ? xl - b[x] : 0;
      return s;
    };
    long long lo = bmin, hi = bmin + j + 1;
    while (hi - lo > 1) {
      const long long mid = lo + (hi - lo) / 2;
      if (F(mid) <= j) lo = mid;
      else hi = mid;
    }
    long long rem = j - F(lo);
    int pick = 0;
    for (int x = 0; x < k; x++)
      if (b[x] <= lo) {
        if (rem == 0) {
          pick = x;
          break;
        }
        rem--;
      }
    part[v] = pick;
  }
}

// Degree-0 vertices with general weights: one thread per graph applies the greedy rule in id order.
__global__ void k_batch_place_seq(DGraph g0, const int64_t *vb, int count, const int32_t *rank,
                                  const int32_t *part_stripped, const int64_t *bwoff, int64_t *bw, const int *kk,
                                  int32_t *part) {
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < count; gi += gridDim.x * blockDim.x) {
    int64_t *b = bw + bwoff[gi];
    const int k = kk[gi];
    for (int64_t v = vb[gi]; v < vb[gi + 1]; v++) {
      if (g0.row_begin(v + 1) > g0.row_begin(v)) {
        part[v] = part_stripped[rank[v]];
        continue;
      }
      int best = 0;
      for (int x = 1; x < k; x++)
        if (b[x] < b[best]) best = x;
      part[v] = best;
      b[best] += g0.vweight(v);
    }
  }
}

struct CopyOut {
  int32_t *dst;
  int64_t vbase, n;
};

__global__ void k_copy_out(const int32_t *part, const CopyOut *co, int count) {
  for (int gi = blockIdx.y; gi < count; gi += gridDim.y) {
    const CopyOut C = co[gi];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C.n; i += (int64_t)gridDim.x * blockDim.x)
      C.dst[i] = part[C.vbase + i];
  }
}

int gridn(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, num_sms() * 8)); }

double now_ms_b() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Local view of graph gi of a union level: offsets and vertex weights shifted to its first vertex.
DGraph view_of(const DGraph &u, int64_t vbase, int64_t n) {
  DGraph d = u;
  d.n = n;
  d.off = static_cast<const char *>(u.off) + vbase * (u.off64 ? 8 : 4);
  if (u.vw) d.vw = static_cast<const char *>(u.vw) + vbase * (u.vw64 ? 8 : 4);
  return d;
}

template <class T>
int to_device(Workspace &ws, const std::vector<T> &h, T **d, cudaStream_t s) {
  GP_TRY(ws.get(d, std::max<size_t>(h.size(), 1)));
  if (!h.empty()) GP_CUDA(cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
  return GP_OK;
}

// Runs LP jobs in one launch (small jobs share blocks).
int run_lp_chunks(std::vector<LpJob> &jobs, cudaStream_t s, const LpConfig &cfg) {
  if (jobs.empty()) return GP_OK;
  return run_lp_multi(jobs.data(), (int)jobs.size(), s, cfg);
}

}  // namespace

int partition_batch_device(const gp_batch_item *items, int count, const gp_params *pp, gp_result *res,
                           cudaStream_t s) {
  const double t0 = now_ms_b();
  gp_params p;
  if (pp) p = *pp;
  else gp_default_params(&p);
  if (p.ip_tries < 1 || p.ip_tries > 16 || p.cluster_div < 1 || p.max_levels < 0 || p.max_levels > 64) {
    set_error("gp_partition_batch: params out of range");
    return GP_ERR_INVALID_ARG;
  }
  if (p.coarsen != GP_COARSEN_LP) {
    set_error("gp_partition_batch: only LP clustering coarsens a batch");
    return GP_ERR_INVALID_ARG;
  }
  if (p.mode != GP_MODE_PLAIN && p.mode != GP_MODE_LEARNED) {
    set_error("gp_partition_batch: mode must be plain or learned");
    return GP_ERR_INVALID_ARG;
  }
  if (p.mode == GP_MODE_LEARNED && !p.mlp) {
    set_error("gp_partition_batch: learned mode needs params.mlp");
    return GP_ERR_INVALID_ARG;
  }
  const bool learned = p.mode == GP_MODE_LEARNED;
  const LpConfig cfg = schedule_for_batch(&p);
  const int tries = (int)p.ip_tries;
  Workspace ws(s);
  // ---- level-0 union
  std::vector<BatchDesc> hd(count);
  std::vector<int64_t> vb(count + 1, 0), eb(count + 1, 0);
  bool any_vw = false, any_ew = false;
  for (int i = 0; i < count; i++) {
    const gp_graph &g = items[i].g;
    if (g.n < 0 || g.m_dir < 0 || (g.n > 0 && !g.offsets) || (g.m_dir > 0 && !g.adj) || !items[i].part_out ||
        items[i].k < 1 || items[i].k > g.n || !(items[i].eps >= 0.0)) {
      set_error("gp_partition_batch: item " + std::to_string(i) + " is invalid");
      return GP_ERR_INVALID_ARG;
    }
    hd[i] = BatchDesc{g.offsets, g.adj, g.vwgt, g.ewgt, g.offsets_64 ? 1 : 0, g.vwgt_64 ? 1 : 0, g.ewgt_64 ? 1 : 0,
                      0, g.n, g.m_dir};
    vb[i + 1] = vb[i] + g.n;
    eb[i + 1] = eb[i] + g.m_dir;
    any_vw |= g.vwgt != nullptr;
    any_ew |= g.ewgt != nullptr;
  }
  const int64_t N = vb[count], M = eb[count];
  if (N >= ((int64_t)1 << 31) - 1) {
    set_error("gp_partition_batch: the union of the graphs must have fewer than 2^31 - 1 vertices");
    return GP_ERR_UNSUPPORTED;
  }
  BatchDesc *d_desc;
  int64_t *d_vb, *d_eb, *u_off, *u_vw = nullptr, *u_ew = nullptr;
  int32_t *u_adj;
  GP_TRY(to_device(ws, hd, &d_desc, s));
  GP_TRY(to_device(ws, vb, &d_vb, s));
  GP_TRY(to_device(ws, eb, &d_eb, s));
  GP_TRY(ws.get(&u_off, (size_t)N + 1));
  GP_TRY(ws.get(&u_adj, (size_t)std::max<int64_t>(M, 1)));
  if (any_vw) GP_TRY(ws.get(&u_vw, (size_t)std::max<int64_t>(N, 1)));
  if (any_ew) GP_TRY(ws.get(&u_ew, (size_t)std::max<int64_t>(M, 1)));
  (::gp::count_launch(), k_union_rows<<<gridn(N), 256, 0, s>>>(d_desc, count, d_vb, d_eb, N, u_off, u_vw, any_vw));
  if (M > 0) (::gp::count_launch(), k_union_entries<<<gridn(M), 256, 0, s>>>(d_desc, count, d_vb, d_eb, M, u_adj, u_ew, any_ew));
  GP_LAUNCH_CHECK();
  DGraph U0;
  U0.n = N;
  U0.m = M;
  U0.off = u_off;
  U0.off64 = 1;
  U0.adj = u_adj;
  U0.vw = u_vw;
  U0.vw64 = 1;
  U0.ew = u_ew;
  U0.ew64 = 1;
  // per-graph totals and Lmax
  unsigned long long *wsum;
  GP_TRY(ws.zeros(&wsum, (size_t)count));
  if (N > 0) (::gp::count_launch(), k_graph_vstats<<<gridn(N), 256, 0, s>>>(U0, d_vb, count, nullptr, wsum));
  std::vector<unsigned long long> hw(count);
  GP_CUDA(cudaMemcpyAsync(hw.data(), wsum, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  std::vector<int64_t> lmax(count), Tstop(count);
  for (int i = 0; i < count; i++) {
    std::memset(&res[i], 0, sizeof(gp_result));
    const int64_t ceil_avg = ((int64_t)hw[i] + items[i].k - 1) / items[i].k;
    lmax[i] = (int64_t)((1.0 + items[i].eps) * (double)ceil_avg);
    res[i].lmax = lmax[i];
    Tstop[i] = std::max<int64_t>(p.coarse_min, p.coarse_per_k * (int64_t)items[i].k);
  }
  // ---- degree-0 vertices
  Stripped st;
  GP_TRY(strip_isolated(U0, &st, ws, s));
  std::vector<int64_t> vb0(count + 1);
  int64_t *d_rank_at = nullptr;
  if (st.n_iso > 0) {
    GP_TRY(ws.get(&d_rank_at, (size_t)count + 1));
    (::gp::count_launch(), k_gather_at<<<gridn(count + 1), 256, 0, s>>>(st.rank, d_vb, count + 1, N, st.n0, d_rank_at));
    GP_CUDA(cudaMemcpyAsync(vb0.data(), d_rank_at, sizeof(int64_t) * (count + 1), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
  } else {
    vb0 = vb;
  }
  for (int i = 0; i < count; i++) {
    res[i].n_isolated = (vb[i + 1] - vb[i]) - (vb0[i + 1] - vb0[i]);
    res[i].level_n[0] = vb0[i + 1] - vb0[i];
  }
  // ---- coarsening on the union
  std::vector<DGraph> G{st.g0};
  std::vector<std::vector<int64_t>> VB{vb0};
  std::vector<OwnedGraph> owned;
  std::vector<int32_t *> f2c;
  owned.reserve(64);
  std::vector<int> clev(count, 0);
  std::vector<char> active(count, 0);
  for (int i = 0; i < count; i++) active[i] = (vb0[i + 1] - vb0[i]) > Tstop[i];
  std::vector<int64_t> lp_edges(count, 0), lp_moves(count, 0);
  struct Cleanup {
    std::vector<OwnedGraph> *o;
    cudaStream_t s;
    ~Cleanup() {
      for (auto &g : *o) g.release(s);
    }
  } cleanup{&owned, s};
  int32_t *labels = nullptr;
  int64_t *lw = nullptr;
  int32_t *q = nullptr;
  if (st.n0 > 0) {
    GP_TRY(ws.get(&labels, (size_t)st.n0));
    GP_TRY(ws.get(&lw, (size_t)st.n0));
    if (learned) GP_TRY(ws.get(&q, (size_t)std::max<int64_t>(st.g0.m, 1)));
  }
  const double t_c0 = now_ms_b();
  unsigned long long *maxc_d;
  GP_TRY(ws.get(&maxc_d, (size_t)count));
  int64_t *d_vbl;
  GP_TRY(ws.get(&d_vbl, (size_t)count + 1));
  unsigned long long *first_d;
  GP_TRY(ws.get(&first_d, (size_t)count));
  for (int l = 0; l < p.max_levels && st.n0 > 0; l++) {
    bool any = false;
    for (int i = 0; i < count; i++) any |= active[i] != 0;
    if (!any) break;
    const DGraph gl = G.back();                  // copies: G and VB grow below
    const std::vector<int64_t> vbl = VB.back();
    GP_CUDA(cudaMemcpyAsync(d_vbl, vbl.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
    GP_CUDA(cudaMemsetAsync(maxc_d, 0, sizeof(unsigned long long) * count, s));
    (::gp::count_launch(), k_graph_vstats<<<gridn(gl.n), 256, 0, s>>>(gl, d_vbl, count, maxc_d, nullptr));
    (::gp::count_launch(), k_iota_i32<<<gridn(gl.n), 256, 0, s>>>(labels, gl.n));
    (::gp::count_launch(), k_vw_i64<<<gridn(gl.n), 256, 0, s>>>(gl, lw));
    GP_LAUNCH_CHECK();
    std::vector<unsigned long long> hmax(count);
    GP_CUDA(cudaMemcpyAsync(hmax.data(), maxc_d, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (learned) GP_TRY(mlp_score(gl, l, static_cast<const gp_mlp *>(p.mlp), nullptr, q, s));
    std::vector<LpJob> jobs;
    std::vector<gp_lp_stats> stats(count);
    std::vector<int> job_graph;
    for (int i = 0; i < count; i++) {
      if (!active[i]) continue;
      LpJob j;
      j.g = view_of(gl, vbl[i], vbl[i + 1] - vbl[i]);
      j.vbase = vbl[i];
      j.lbase = vbl[i];
      j.q = q;
      j.labels = labels;
      j.lw = lw;
      j.nl = vbl[i + 1] - vbl[i];
      j.U = std::max<int64_t>((int64_t)hmax[i], lmax[i] / p.cluster_div);
      j.rounds = (int)p.rounds_coarsen;
      j.seed = hash3(items[i].seed, (uint64_t)l, 1);
      j.stats = &stats[i];
      j.singletons = true;
      jobs.push_back(j);
      job_graph.push_back(i);
    }
    GP_TRY(run_lp_chunks(jobs, s, cfg));
    for (int i : job_graph) {
      lp_edges[i] += stats[i].edges;
      lp_moves[i] += stats[i].moves;
    }
    owned.emplace_back();
    int32_t *map;
    GP_TRY(ws.get(&map, (size_t)gl.n));
    GP_TRY(contract_graph(gl, labels, gl.n, &owned.back(), map, s));
    f2c.push_back(map);
    // first coarse id of every graph; a graph without vertices starts where the next one starts
    std::vector<unsigned long long> hfirst(count);
    GP_CUDA(cudaMemsetAsync(first_d, 0xff, sizeof(unsigned long long) * count, s));
    if (gl.n > 0) (::gp::count_launch(), k_graph_first<<<gridn(gl.n), 256, 0, s>>>(map, d_vbl, count, gl.n, first_d));
    GP_LAUNCH_CHECK();
    GP_CUDA(cudaMemcpyAsync(hfirst.data(), first_d, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> nvb(count + 1);
    nvb[count] = owned.back().n;
    for (int i = count - 1; i >= 0; i--) nvb[i] = vbl[i + 1] > vbl[i] ? (int64_t)hfirst[i] : nvb[i + 1];
    for (int i = 0; i < count; i++)
      if (nvb[i] > nvb[i + 1] || nvb[i + 1] - nvb[i] > vbl[i + 1] - vbl[i] ||
          (vbl[i + 1] > vbl[i] && nvb[i + 1] == nvb[i])) {
        set_error("gp_partition_batch: coarse vertex ranges of the graphs are inconsistent");
        return GP_ERR_INTERNAL;
      }
    G.push_back(owned.back().view());
    VB.push_back(nvb);
    for (int i = 0; i < count; i++) {
      if (!active[i]) continue;
      const int64_t nb4 = vbl[i + 1] - vbl[i], naf = nvb[i + 1] - nvb[i];
      clev[i] = l + 1;
      res[i].level_n[l + 1] = naf;
      if (100 * naf > p.stall_pct * nb4 || naf <= Tstop[i] || l + 1 >= p.max_levels) active[i] = 0;
    }
  }
  const int L = (int)f2c.size();
  const double t_ip0 = now_ms_b();
  // ---- initial partitioning of every graph's coarsest level (the union's last level)
  const DGraph &gc = G.back();
  const std::vector<int64_t> &vbc = VB.back();
  std::vector<IpJob> ipj;
  std::vector<int32_t *> parts(count, nullptr);
  std::vector<TryEval> te(count);
  std::vector<int64_t> kk64(count), bwoff(count + 1, 0);
  for (int i = 0; i < count; i++) bwoff[i + 1] = bwoff[i] + items[i].k;
  int64_t *tbw;
  GP_TRY(ws.zeros(&tbw, (size_t)bwoff[count] * tries));
  std::vector<int> kint(count);
  for (int i = 0; i < count; i++) {
    kint[i] = items[i].k;
    const int64_t ni = vbc[i + 1] - vbc[i];
    GP_TRY(ws.get(&parts[i], (size_t)std::max<int64_t>(ni, 1) * tries));
    te[i] = TryEval{parts[i], ni, vbc[i], items[i].k, tbw + bwoff[i] * tries};
    if (ni == 0) continue;
    IpJob j;
    j.g = view_of(gc, vbc[i], ni);
    j.vbase = vbc[i];
    j.k = items[i].k;
    j.lmax = lmax[i];
    j.seed = items[i].seed;
    j.level = clev[i];
    j.parts = parts[i];
    ipj.push_back(j);
  }
  if (!ipj.empty()) GP_TRY(initial_partition_multi(ipj.data(), (int)ipj.size(), tries, (int)p.repair_rounds, s));
  // LP refinement of every try
  TryEval *d_te;
  GP_TRY(to_device(ws, te, &d_te, s));
  int64_t *d_vbc;
  GP_TRY(to_device(ws, vbc, &d_vbc, s));
  // block weights of the unrefined tries (label weights of their LP refinement)
  if (gc.n > 0) (::gp::count_launch(), k_try_eval<<<gridn(gc.n), 256, 0, s>>>(gc, d_vbc, count, d_te, tries, nullptr));
  std::vector<LpJob> rj;
  std::vector<gp_lp_stats> rstats((size_t)count * tries);
  for (int i = 0; i < count; i++) {
    const int64_t ni = vbc[i + 1] - vbc[i];
    if (ni == 0 || p.rounds_refine <= 0) continue;
    const uint64_t seed_i = items[i].seed;
    for (int t = 0; t < tries; t++) {
      const uint64_t s_try = hash3(seed_i, (uint64_t)clev[i], (uint64_t)(4 + t));
      LpJob j;
      j.g = view_of(gc, vbc[i], ni);
      j.vbase = vbc[i];
      j.lbase = 0;
      j.labels = parts[i] + (size_t)t * ni - vbc[i];  // indexed by union vertex id
      j.lw = te[i].bw + (size_t)t * items[i].k;
      j.nl = items[i].k;
      j.U = lmax[i];
      j.rounds = (int)p.rounds_refine;
      j.seed = hash3(s_try, (uint64_t)clev[i], 3);
      j.stats = &rstats[(size_t)i * tries + t];
      rj.push_back(j);
    }
  }
  GP_TRY(run_lp_chunks(rj, s, cfg));
  for (int i = 0; i < count; i++)
    for (int t = 0; t < tries; t++) {
      lp_edges[i] += rstats[(size_t)i * tries + t].edges;
      lp_moves[i] += rstats[(size_t)i * tries + t].moves;
    }
  // cuts and block weights of the refined tries
  unsigned long long *tcut;
  GP_TRY(ws.zeros(&tcut, (size_t)count * tries));
  GP_CUDA(cudaMemsetAsync(tbw, 0, sizeof(int64_t) * (size_t)bwoff[count] * tries, s));
  if (gc.n > 0) (::gp::count_launch(), k_try_eval<<<gridn(gc.n), 256, 0, s>>>(gc, d_vbc, count, d_te, tries, tcut));
  GP_LAUNCH_CHECK();
  std::vector<unsigned long long> htcut((size_t)count * tries);
  std::vector<int64_t> htbw((size_t)bwoff[count] * tries);
  GP_CUDA(cudaMemcpyAsync(htcut.data(), tcut, sizeof(unsigned long long) * htcut.size(), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaMemcpyAsync(htbw.data(), tbw, sizeof(int64_t) * htbw.size(), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  std::vector<int> best(count, 0);
  for (int i = 0; i < count; i++) {
    int64_t bc = -1, bimb = 0;
    for (int t = 0; t < tries; t++) {
      const int64_t cut = (int64_t)(htcut[(size_t)i * tries + t] / 2);
      int64_t mx = 0;
      for (int b = 0; b < items[i].k; b++) mx = std::max(mx, htbw[bwoff[i] * tries + (size_t)t * items[i].k + b]);
      const int64_t imb = mx > lmax[i] ? 1 : 0;
      res[i].try_cut[t] = cut;
      res[i].try_imbalanced[t] = imb;
      if (bc < 0 || cut < bc || (cut == bc && imb < bimb)) {
        bc = cut;
        bimb = imb;
        best[i] = t;
      }
    }
    res[i].best_try = best[i];
  }
  int *d_best;
  GP_TRY(to_device(ws, best, &d_best, s));
  int32_t *cur, *nxt;
  GP_TRY(ws.get(&cur, (size_t)std::max<int64_t>(st.n0, 1)));
  GP_TRY(ws.get(&nxt, (size_t)std::max<int64_t>(st.n0, 1)));
  if (gc.n > 0) (::gp::count_launch(), k_pick_tries<<<gridn(gc.n), 256, 0, s>>>(d_vbc, count, gc.n, d_te, d_best, cur));
  GP_LAUNCH_CHECK();
  const double t_r0 = now_ms_b();
  // ---- uncoarsening: project everything, refine the graphs whose own level this is
  // Block weights per graph: the best try's, then each refinement's final label weights. Projection
  // keeps every block's weight, so they are never recomputed on the way up.
  int64_t *d_bwoff, *lbw;
  GP_TRY(to_device(ws, bwoff, &d_bwoff, s));
  {
    std::vector<int64_t> h((size_t)std::max<int64_t>(bwoff[count], 1), 0);
    for (int i = 0; i < count; i++)
      for (int b = 0; b < items[i].k; b++)
        h[bwoff[i] + b] = htbw[(size_t)bwoff[i] * tries + (size_t)best[i] * items[i].k + b];
    GP_TRY(to_device(ws, h, &lbw, s));
  }
  for (int l = L - 1; l >= 0; l--) {
    const DGraph &gl = G[l];
    const std::vector<int64_t> &vbl = VB[l];
    GP_TRY(project(cur, f2c[l], gl.n, nxt, s));
    std::swap(cur, nxt);
    std::vector<LpJob> uj;
    std::vector<gp_lp_stats> ustats(count);
    std::vector<int> ug;
    for (int i = 0; i < count; i++) {
      if (l >= clev[i]) continue;  // not one of this graph's levels: it passes through unchanged
      const int64_t ni = vbl[i + 1] - vbl[i];
      if (ni == 0 || p.rounds_refine <= 0) continue;
      LpJob j;
      j.g = view_of(gl, vbl[i], ni);
      j.vbase = vbl[i];
      j.lbase = 0;
      j.labels = cur;
      j.lw = lbw + bwoff[i];
      j.nl = items[i].k;
      j.U = lmax[i];
      j.rounds = (int)p.rounds_refine;
      j.seed = hash3(items[i].seed, (uint64_t)l, 2);
      j.stats = &ustats[i];
      uj.push_back(j);
      ug.push_back(i);
    }
    GP_TRY(run_lp_chunks(uj, s, cfg));
    for (int i : ug) {
      lp_edges[i] += ustats[i].edges;
      lp_moves[i] += ustats[i].moves;
    }
  }
  // ---- degree-0 vertices and final evaluation on the input union
  int32_t *fullp;
  GP_TRY(ws.get(&fullp, (size_t)std::max<int64_t>(N, 1)));
  if (st.n_iso > 0) {
    // (lbw holds the block weights of the kept vertices per graph)
    int *d_k;
    GP_TRY(to_device(ws, kint, &d_k, s));
    if (!any_vw)
      (::gp::count_launch(), k_batch_place<<<gridn(N), 256, 0, s>>>(U0, d_vb, count, st.rank, d_rank_at, cur, d_bwoff, lbw, d_k, fullp));
    else
      (::gp::count_launch(), k_batch_place_seq<<<gridn(count), 256, 0, s>>>(U0, d_vb, count, st.rank, cur, d_bwoff, lbw, d_k, fullp));
    GP_LAUNCH_CHECK();
  } else if (N > 0) {
    GP_CUDA(cudaMemcpyAsync(fullp, cur, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToDevice, s));
  }
  unsigned long long *fcut;
  GP_TRY(ws.zeros(&fcut, (size_t)count));
  GP_CUDA(cudaMemsetAsync(lbw, 0, sizeof(int64_t) * (size_t)bwoff[count], s));
  if (N > 0) (::gp::count_launch(), k_union_eval<<<gridn(N), 256, 0, s>>>(U0, d_vb, count, fullp, d_bwoff, lbw, fcut));
  std::vector<CopyOut> co(count);
  for (int i = 0; i < count; i++) co[i] = CopyOut{items[i].part_out, vb[i], vb[i + 1] - vb[i]};
  CopyOut *d_co;
  GP_TRY(to_device(ws, co, &d_co, s));
  (::gp::count_launch(), k_copy_out<<<dim3(64, std::min(count, 65535)), 256, 0, s>>>(fullp, d_co, count));
  GP_LAUNCH_CHECK();
  std::vector<unsigned long long> hcut(count);
  std::vector<int64_t> hbw(bwoff[count]);
  GP_CUDA(cudaMemcpyAsync(hcut.data(), fcut, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaMemcpyAsync(hbw.data(), lbw, sizeof(int64_t) * hbw.size(), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  // CSR entries of every graph at every level (all union levels have int64 offsets)
  std::vector<std::vector<int64_t>> EB(G.size());
  {
    int64_t *d_idx, *d_out;
    GP_TRY(ws.get(&d_idx, (size_t)count + 1));
    GP_TRY(ws.get(&d_out, (size_t)(count + 1) * G.size()));
    for (size_t l = 0; l < G.size(); l++) {
      GP_CUDA(cudaMemcpyAsync(d_idx, VB[l].data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
      (::gp::count_launch(), k_gather_off<<<gridn(count + 1), 256, 0, s>>>(static_cast<const int64_t *>(G[l].off), d_idx, count + 1,
                                                                           d_out + (count + 1) * l));
    }
    std::vector<int64_t> h((size_t)(count + 1) * G.size());
    GP_CUDA(cudaMemcpyAsync(h.data(), d_out, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    for (size_t l = 0; l < G.size(); l++) EB[l].assign(h.begin() + (count + 1) * l, h.begin() + (count + 1) * (l + 1));
  }
  const double t_end = now_ms_b();
  for (int i = 0; i < count; i++) {
    gp_result &r = res[i];
    r.cut = (int64_t)(hcut[i] / 2);
    int64_t mx = 0;
    for (int b = 0; b < items[i].k; b++) mx = std::max(mx, hbw[bwoff[i] + b]);
    r.max_block_weight = mx;
    r.imbalanced = mx > lmax[i] ? 1 : 0;
    r.levels = clev[i];
    for (int l = 0; l <= clev[i] && l < 65; l++) {
      r.level_n[l] = VB[l][i + 1] - VB[l][i];
      r.level_m[l] = EB[l][i + 1] - EB[l][i];
    }
    r.lp_edges = lp_edges[i];
    r.lp_moves = lp_moves[i];
    if (learned) r.learned_cut = r.cut;
    else r.plain_cut = r.cut;
    r.ms_total = t_end - t0;
    r.ms_coarsen = t_ip0 - t_c0;
    r.ms_initial = t_r0 - t_ip0;
    r.ms_refine = t_end - t_r0;
  }
  GP_TRY(prof_flush(s));
  return GP_OK;
}

}  // namespace gp

extern "C" int gp_partition_batch(const gp_batch_item *items, int32_t count, const gp_params *params, gp_result *res,
                                  gp_stream stream) {
  if (count < 0 || (count > 0 && (!items || !res))) {
    gp::set_error("gp_partition_batch: items and res are required");
    return GP_ERR_INVALID_ARG;
  }
  if (count == 0) return GP_OK;
  const int st = gp::partition_batch_device(items, count, params, res, (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  return st;
}
