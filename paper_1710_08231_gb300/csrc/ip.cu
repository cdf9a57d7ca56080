// ip.cu -- initial partitioning of the coarsest graph, evaluation, projection and degree-0 vertices.
//
// Initial partitioning (Section III-B, Section IV-B): the coarsest graph is partitioned several
// times independently and the best result is kept; each try is a recursive bisection into
// ceil(k/2) and floor(k/2) blocks. KaHIP's bisection with local search and flows is external to the
// paper; this library's bisection is deterministic: BFS from the vertex of minimum
// H(s_try, depth, v), a second BFS from the farthest vertex found (ties: smaller id), vertices
// ordered by (distance, id) with unreachable ones last, side 0 the shortest prefix whose weight
// reaches ceil(k/2)/k of the set. All sets of one recursion depth are split together (their BFS
// runs are one multi-source BFS restricted to each set), one CTA per try, tries in parallel.
// A balance repair then moves vertices out of overloaded blocks (Section II-A: a block is
// overloaded when heavier than Lmax).
// Projection (Section III-C): a fine vertex takes the block of its coarse representative.
#include <algorithm>
#include <climits>
#include <vector>

#include "block_sort.cuh"
#include "ip.cuh"
#include "lp.cuh"

namespace gp {

namespace {

constexpr int kIpThreads = 1024;

// One graph of an initial-partitioning launch: a local view (offsets and vertex weights shifted to its
// first vertex; adjacency holds global ids, minus vbase gives local ids), its parameters and where its
// tries' partitions and scratch live.
struct IpGraph {
  DGraph g;
  int64_t vbase;
  int k;
  int level;
  int64_t lmax;
  uint64_t seed;
  int32_t *parts;     // tries * n
  int64_t ns;         // per-try stride of n-sized scratch: max(n, k)
  int64_t scr_off;    // offset of this graph's n-sized scratch (tries * ns)
  int64_t kscr_off;   // offset of this graph's k-sized scratch (tries * k)
  int64_t conn_off;   // offset of this graph's repair connection scratch (tries * kIpThreads * k)
};

struct IpArgs {
  const IpGraph *graphs;
  const int *block_graph;
  const int *block_try;
  int repair_rounds;
  int32_t *gk;               // n-sized scratch arrays
  int32_t *dist;
  int32_t *qa, *qb;
  unsigned long long *ka, *kb;
  int32_t *va, *vb;
  int32_t *mv_t;
  long long *mv_g;
  uint8_t *flag;
  int64_t smem_ns;           // > 0: the bisection keeps part, gk, dist and both BFS queues of every try
                             // in dynamic shared memory (every graph of the launch has ns <= smem_ns)
  int smem_sort;             // with smem_ns: the sort's key and value arrays are in shared memory too
  long long *gws;            // k-sized scratch arrays
  unsigned long long *gminh;
  int *gstart;
  unsigned long long *gfar;
  long long *bw;
  long long *conn;
  int *err;
};

// Multi-source BFS restricted to same-set vertices (part equal, set still being split).
__device__ void set_bfs(const DGraph &g, int64_t vbase, int32_t *part, int32_t *gk, int32_t *dist, int32_t *qa,
                        int32_t *qb, int nf) {
  __shared__ int s_next;
  while (nf > 0) {
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    // one warp per frontier vertex, lanes over its row
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = wid; i < nf; i += nw) {
      const int x = qa[i];
      const int px = part[x];
      const int dx = dist[x];
      const int64_t b = g.row_begin(x), e = g.row_begin(x + 1);
      for (int64_t j = b + lane; j < e; j += 32) {
        const int u = (int)(g.adj[j] - vbase);
        if (gk[u] <= 1 || part[u] != px) continue;
        if (atomicCAS(&dist[u], -1, dx + 1) == -1) qb[atomicAdd(&s_next, 1)] = u;
      }
    }
    __syncthreads();
    nf = s_next;
    int32_t *t = qa;
    qa = qb;
    qb = t;
    __syncthreads();
  }
}

// Per-vertex state of a bisection in shared memory: 5 arrays of ns int32 (part, gk, dist, qa, qb), and
// for ns <= kIpSmemSortNs also the sort's keys and values (2 x ns uint64 + 2 x ns int32) after them.
constexpr int64_t kIpSmemMaxNs = 8192;
constexpr int64_t kIpSmemSortNs = 4096;
constexpr size_t ip_state_bytes(int64_t ns) { return ((size_t)ns * 5 * sizeof(int32_t) + 15) & ~size_t(15); }
constexpr size_t ip_smem_bytes(int64_t ns, bool sort) {
  return ip_state_bytes(ns) + (sort ? (size_t)ns * (2 * sizeof(unsigned long long) + 2 * sizeof(int32_t)) : 0);
}

__global__ void __launch_bounds__(kIpThreads, 2) k_bisect(IpArgs a) {
  extern __shared__ __align__(16) unsigned char ip_dsm[];
  __shared__ BlockSortSmem sm;
  __shared__ int s_any, s_maxd;
  const IpGraph &G = a.graphs[a.block_graph[blockIdx.x]];
  const int t = a.block_try[blockIdx.x];
  const DGraph g = G.g;
  const int n = (int)g.n, k = G.k;
  const size_t ns = (size_t)G.ns;
  const size_t so = (size_t)G.scr_off + (size_t)t * ns, ko = (size_t)G.kscr_off + (size_t)t * k;
  int32_t *const part_out = G.parts + (size_t)t * n;
  int32_t *part = part_out, *gk = a.gk + so, *dist = a.dist + so;
  int32_t *qa = a.qa + so, *qb = a.qb + so;
  if (a.smem_ns > 0) {
    // small coarsest graphs: the BFS state lives in shared memory (the partition is copied out at
    // the end)
    int32_t *sp = reinterpret_cast<int32_t *>(ip_dsm);
    part = sp;
    gk = sp + ns;
    dist = sp + 2 * ns;
    qa = sp + 3 * ns;
    qb = sp + 4 * ns;
  }
  unsigned long long *ka = a.ka + so, *kb = a.kb + so;
  int32_t *va = a.va + so, *vb = a.vb + so;
  if (a.smem_sort) {
    unsigned char *sb = ip_dsm + ip_state_bytes((int64_t)ns);
    ka = reinterpret_cast<unsigned long long *>(sb);
    kb = ka + ns;
    va = reinterpret_cast<int32_t *>(kb + ns);
    vb = va + ns;
  }
  long long *gws = a.gws + ko;
  unsigned long long *gminh = a.gminh + ko, *gfar = a.gfar + ko;
  int *gstart = a.gstart + ko;
  const uint64_t s_try = hash3(G.seed, (uint64_t)G.level, (uint64_t)(4 + t));
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    part[v] = 0;
    gk[v] = k;
  }
  __syncthreads();
  for (int depth = 0; depth < 64; depth++) {
    if (threadIdx.x == 0) {
      s_any = 0;
      s_maxd = 0;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x)
      if (gk[v] > 1) s_any = 1;
    __syncthreads();
    if (!s_any) break;
    for (int b = threadIdx.x; b < k; b += blockDim.x) {
      gws[b] = 0;
      gminh[b] = ~0ull;
      gstart[b] = INT_MAX;
      gfar[b] = 0;
    }
    __syncthreads();
    const uint64_t hd = mix64(mix64(s_try) ^ (uint64_t)depth);
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      if (gk[v] <= 1) continue;
      const int b = part[v];
      atomicAdd(reinterpret_cast<unsigned long long *>(&gws[b]), (unsigned long long)g.vweight(v));
      atomicMin(&gminh[b], (unsigned long long)mix64(hd ^ (uint64_t)v));
      dist[v] = -1;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      if (gk[v] <= 1) continue;
      const int b = part[v];
      if (mix64(hd ^ (uint64_t)v) == gminh[b]) atomicMin(&gstart[b], v);
    }
    __syncthreads();
    // BFS 1 from the start vertex of every set
    int nf = block_compact(k, [&](int b) { return gstart[b] != INT_MAX; }, qa, sm);
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
      const int v = gstart[qa[i]];
      qa[i] = v;
      dist[v] = 0;
    }
    __syncthreads();
    set_bfs(g, G.vbase, part, gk, dist, qa, qb, nf);
    // farthest vertex per set, ties by smaller id
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      if (gk[v] <= 1 || dist[v] < 0) continue;
      atomicMax(&gfar[part[v]], ((unsigned long long)dist[v] << 32) | (unsigned long long)(0x7fffffff - v));
    }
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x)
      if (gk[v] > 1) dist[v] = -1;
    __syncthreads();
    nf = block_compact(k, [&](int b) { return gfar[b] != 0; }, qa, sm);
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
      const int v = 0x7fffffff - (int)(gfar[qa[i]] & 0xffffffffull);
      qa[i] = v;
      dist[v] = 0;
    }
    __syncthreads();
    set_bfs(g, G.vbase, part, gk, dist, qa, qb, nf);
    // order the vertices of every set by (set, unreachable, distance), stable in id order
    const int na = block_compact(n, [&](int v) { return gk[v] > 1; }, va, sm);
    for (int i = threadIdx.x; i < na; i += blockDim.x) atomicMax(&s_maxd, dist[va[i]]);
    __syncthreads();
    const int db = bits_of((unsigned long long)s_maxd + 1);
    const int kbits = bits_of((unsigned long long)(k > 1 ? k - 1 : 0));
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
      const int v = va[i];
      const int dv = dist[v];
      const unsigned long long unreach = dv < 0 ? 1ull : 0ull;
      ka[i] = ((unsigned long long)part[v] << (db + 1)) | (unreach << db) | (unsigned long long)(dv < 0 ? 0 : dv);
    }
    __syncthreads();
    const bool in_b = block_radix_sort(ka, va, kb, vb, na, kbits + db + 1, sm);
    unsigned long long *ks = in_b ? kb : ka;
    int32_t *vs = in_b ? vb : va;
    // side 0: shortest prefix of the set whose weight reaches ceil(kS/2)/kS of the set
    block_seg_scan(
        na, [&](int p) { return (int)(ks[p] >> (db + 1)); },
        [&](int p) { return g.vweight(vs[p]); },
        [&](int p, long long excl, long long) {
          const int v = vs[p];
          const int base = (int)(ks[p] >> (db + 1));
          const int kS = gk[v];
          const int k0 = (kS + 1) / 2, k1 = kS / 2;
          const __int128 lhs = (__int128)excl * kS, rhs = (__int128)gws[base] * k0;
          if (lhs < rhs) {
            gk[v] = k0;
          } else {
            part[v] = base + k0;
            gk[v] = k1;
          }
        },
        sm);
    __syncthreads();
  }
  if (a.smem_ns > 0) {
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x) part_out[v] = part[v];
  }
}

// Balance repair (one CTA per try).
__global__ void __launch_bounds__(kIpThreads) k_repair(IpArgs a) {
  __shared__ BlockSortSmem sm;
  __shared__ int s_over, s_light, s_applied;
  __shared__ long long s_gmin, s_gmax;
  const IpGraph &G = a.graphs[a.block_graph[blockIdx.x]];
  const int t = a.block_try[blockIdx.x];
  const DGraph g = G.g;
  const int n = (int)g.n, k = G.k;
  const int64_t lmax = G.lmax, vbase = G.vbase;
  const size_t ns = (size_t)G.ns;
  const size_t so = (size_t)G.scr_off + (size_t)t * ns, ko = (size_t)G.kscr_off + (size_t)t * k;
  int32_t *part = G.parts + (size_t)t * n;
  unsigned long long *ka = a.ka + so, *kb = a.kb + so;
  int32_t *va = a.va + so, *vb = a.vb + so;
  int32_t *mv_t = a.mv_t + so;
  long long *mv_g = a.mv_g + so;
  uint8_t *flag = a.flag + so;
  int32_t *list2 = a.qa + so;
  long long *bw = a.bw + ko;
  long long *conn = a.conn + (size_t)G.conn_off + ((size_t)t * blockDim.x + threadIdx.x) * (size_t)k;
  const int kbits = bits_of((unsigned long long)(k > 1 ? k - 1 : 0));
  for (int b = 0; b < k; b++) conn[b] = 0;
  for (int rr = 0; rr < a.repair_rounds; rr++) {
    for (int b = threadIdx.x; b < k; b += blockDim.x) bw[b] = 0;
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x)
      atomicAdd(reinterpret_cast<unsigned long long *>(&bw[part[v]]), (unsigned long long)g.vweight(v));
    __syncthreads();
    if (threadIdx.x == 0) {
      int over = 0, light = 0;
      for (int b = 0; b < k; b++) {
        if (bw[b] > lmax) over = 1;
        if (bw[b] < bw[light]) light = b;
      }
      s_over = over;
      s_light = light;
      s_applied = 0;
      s_gmin = LLONG_MAX;
      s_gmax = LLONG_MIN;
    }
    __syncthreads();
    if (!s_over) break;
    // per vertex of an overloaded block: target and gain
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      mv_t[v] = -1;
      const int P = part[v];
      if (bw[P] <= lmax) continue;
      const long long cv = g.vweight(v);
      const int64_t b = g.row_begin(v), e = g.row_begin(v + 1);
      for (int64_t j = b; j < e; j++) conn[part[g.adj[j] - vbase]] += g.eweight(j);
      int best = -1;
      for (int64_t j = b; j < e; j++) {
        const int B = part[g.adj[j] - vbase];
        if (B == P || conn[B] <= 0 || bw[B] + cv > lmax) continue;
        if (best < 0 || conn[B] > conn[best] || (conn[B] == conn[best] && B < best)) best = B;
      }
      if (best < 0 && s_light != P && bw[s_light] + cv <= lmax) best = s_light;
      if (best >= 0) {
        mv_t[v] = best;
        mv_g[v] = conn[best] - conn[P];
        atomicMin(&s_gmin, mv_g[v]);
        atomicMax(&s_gmax, mv_g[v]);
      }
      for (int64_t j = b; j < e; j++) conn[part[g.adj[j] - vbase]] = 0;
    }
    __syncthreads();
    const int nm = block_compact(n, [&](int v) { return mv_t[v] >= 0; }, va, sm);
    if (nm == 0) break;
    const unsigned long long grange = (unsigned long long)(s_gmax - s_gmin);
    const int gb = bits_of(grange);
    if (kbits + gb > 64) {
      if (threadIdx.x == 0) atomicExch(a.err, GP_ERR_UNSUPPORTED);
      return;
    }
    // per target: (gain desc, id asc) -- input is in id order, the sort is stable
    for (int i = threadIdx.x; i < nm; i += blockDim.x) {
      const int v = va[i];
      ka[i] = ((unsigned long long)mv_t[v] << gb) | (unsigned long long)(s_gmax - mv_g[v]);
    }
    __syncthreads();
    bool in_b = block_radix_sort(ka, va, kb, vb, nm, kbits + gb, sm);
    unsigned long long *ks = in_b ? kb : ka;
    int32_t *vs = in_b ? vb : va;
    for (int v = threadIdx.x; v < n; v += blockDim.x) flag[v] = 0;
    __syncthreads();
    block_seg_scan(
        nm, [&](int p) { return (int)(ks[p] >> gb); }, [&](int p) { return g.vweight(vs[p]); },
        [&](int p, long long, long long incl) {
          const int v = vs[p];
          if (bw[mv_t[v]] + incl <= lmax) flag[v] = 1;
        },
        sm);
    __syncthreads();
    // per source: take movers while the source is still overloaded
    const int na = block_compact(n, [&](int v) { return flag[v] != 0; }, list2, sm);
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
      const int v = list2[i];
      ka[i] = ((unsigned long long)part[v] << gb) | (unsigned long long)(s_gmax - mv_g[v]);
      va[i] = v;
    }
    __syncthreads();
    in_b = block_radix_sort(ka, va, kb, vb, na, kbits + gb, sm);
    ks = in_b ? kb : ka;
    vs = in_b ? vb : va;
    block_seg_scan(
        na, [&](int p) { return (int)(ks[p] >> gb); }, [&](int p) { return g.vweight(vs[p]); },
        [&](int p, long long excl, long long) {
          const int v = vs[p];
          const int P = (int)(ks[p] >> gb);
          flag[v] = (bw[P] - excl > lmax) ? 2 : 0;
        },
        sm);
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x)
      if (flag[v] == 2) {
        part[v] = mv_t[v];
        s_applied = 1;
      }
    __syncthreads();
    if (!s_applied) break;
  }
}

// Rows up to kCutSmall entries: a thread each; longer rows (hubs of power-law graphs, whose walk by one
// thread would decide the kernel's duration) are left to k_cut_big.
constexpr int64_t kCutSmall = 256;

__global__ void k_cut(DGraph g, const int32_t *part, unsigned long long *acc) {
  __shared__ long long sh[32];
  long long s = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int pv = part[v];
    const int64_t b = g.row_begin(v), e = g.row_begin(v + 1);
    if (e - b > kCutSmall) continue;
    for (int64_t j = b; j < e; j++)
      if (part[g.adj[j]] != pv) s += g.eweight(j);
  }
  s = warp_sum64(s);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[wid] = s;
  __syncthreads();
  if (wid == 0) {
    long long x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
    x = warp_sum64(x);
    if (lane == 0 && x) atomicAdd(acc, (unsigned long long)x);
  }
}

// Rows above kCutSmall entries are cut into items of kCutChunk entries, listed first so that every CTA
// takes items in turn (the long rows of power-law graphs sit at small ids: tiles of vertices would leave
// them to a few CTAs).
constexpr int64_t kCutChunk = 4096;

__global__ void k_cut_list(DGraph g, unsigned long long *items, unsigned long long cap, unsigned long long *cnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = g.row_begin(v + 1) - g.row_begin(v);
    if (d <= kCutSmall) continue;
    const unsigned long long nch = (unsigned long long)((d + kCutChunk - 1) / kCutChunk);
    const unsigned long long base = atomicAdd(cnt, nch);
    for (unsigned long long c = 0; c < nch && base + c < cap; c++) items[base + c] = ((unsigned long long)v << 32) | c;
  }
}

__global__ void k_cut_items(DGraph g, const int32_t *part, const unsigned long long *items, unsigned long long cap,
                            const unsigned long long *cnt, unsigned long long *acc) {
  __shared__ long long sh[32];
  const unsigned long long nit = min(*cnt, cap);  // (the list is sized for every row of the graph)
  long long s = 0;
  for (unsigned long long i = blockIdx.x; i < nit; i += gridDim.x) {
    const unsigned long long it = items[i];
    const int64_t v = (int64_t)(it >> 32);
    const int pv = part[v];
    const int64_t b = g.row_begin(v) + (int64_t)(it & 0xffffffffull) * kCutChunk;
    const int64_t e = min(g.row_begin(v + 1), b + kCutChunk);
    // four entries per thread in flight
    for (int64_t j0 = b; j0 < e; j0 += 4 * (int64_t)blockDim.x) {
      int a[4];
#pragma unroll
      for (int x = 0; x < 4; x++) {
        const int64_t j = j0 + x * (int64_t)blockDim.x + threadIdx.x;
        a[x] = j < e ? __ldg(g.adj + j) : -1;
      }
#pragma unroll
      for (int x = 0; x < 4; x++) {
        const int64_t j = j0 + x * (int64_t)blockDim.x + threadIdx.x;
        if (a[x] >= 0 && part[a[x]] != pv) s += g.eweight(j);
      }
    }
  }
  s = warp_sum64(s);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[wid] = s;
  __syncthreads();
  if (wid == 0) {
    long long x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
    x = warp_sum64(x);
    if (lane == 0 && x) atomicAdd(acc, (unsigned long long)x);
  }
}

__global__ void k_project(const int32_t *coarse, const int32_t *f2c, int64_t n, int32_t *fine) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    fine[v] = coarse[f2c[v]];
}

__global__ void k_vw_stats(DGraph g, unsigned long long *mx, unsigned long long *sum) {
  unsigned long long m = 0, s = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long c = (unsigned long long)g.vweight(v);
    m = max(m, c);
    s += c;
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = max(m, __shfl_xor_sync(kFull, m, o));
    s += __shfl_xor_sync(kFull, s, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(mx, m);
    atomicAdd(sum, s);
  }
}

// Keep flags (degree > 0) and degrees; with `acc`, also acc[0] = max c(v) over the kept vertices and
// acc[1] = sum of c(v) over all vertices.
__global__ void k_deg_flags(DGraph g, uint32_t *keep, int64_t *deg0, unsigned long long *acc) {
  unsigned long long m = 0, sum = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = g.row_begin(v + 1) - g.row_begin(v);
    keep[v] = d > 0 ? 1u : 0u;
    deg0[v] = d;
    if (acc) {
      const unsigned long long c = (unsigned long long)g.vweight(v);
      if (d > 0) m = max(m, c);
      sum += c;
    }
  }
  if (!acc) return;
  for (int o = 16; o > 0; o >>= 1) {
    m = max(m, __shfl_xor_sync(kFull, m, o));
    sum += __shfl_xor_sync(kFull, sum, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (m) atomicMax(&acc[0], m);
    if (sum) atomicAdd(&acc[1], sum);
  }
}

// Degree-0 vertices own no CSR entries, so the kept vertices' rows keep their entries in the same
// order: the stripped offsets are the kept vertices' offsets, the stripped adjacency is the renamed
// adjacency and the edge weights are unchanged.
__global__ void k_strip_rows(DGraph g, const int32_t *rank, const uint32_t *keep, int64_t n0, int64_t *off0,
                             void *vw0) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[v]) continue;
    const int r = rank[v];
    off0[r] = g.row_begin(v);
    if (vw0) {
      if (g.vw64) static_cast<int64_t *>(vw0)[r] = static_cast<const int64_t *>(g.vw)[v];
      else static_cast<int32_t *>(vw0)[r] = static_cast<const int32_t *>(g.vw)[v];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) off0[n0] = g.row_begin(g.n);
}

__global__ void k_strip_adj(const int32_t *adj, int64_t m, const int32_t *rank, int32_t *adj0) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
    adj0[j] = rank[adj[j]];
}

// Degree-0 vertex placement with unit weights, closed form of the greedy rule: at water level x
// every block of weight <= x receives one vertex, blocks in id order. F(x) = sum_b max(0, x - bw_b)
// vertices are placed before level x; vertex j (0-based, ascending id) is placed at the level x with
// F(x) <= j < F(x+1), into the (j - F(x))-th block (by id) among those with bw_b <= x.
__global__ void k_place_unit(DGraph g, const int32_t *rank, const int32_t *part0, const int64_t *iso_idx,
                             const long long *bw, int64_t k, int32_t *part_full) {
  long long bmin = LLONG_MAX;
  for (int64_t b = 0; b < k; b++) bmin = min(bmin, bw[b]);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int r = rank[v];
    if (r >= 0) {
      part_full[v] = part0[r];
      continue;
    }
    const long long j = iso_idx[v];
    long long lo = bmin, hi = bmin + j + 1;  // F(lo) = 0 <= j; F(hi) > j
    auto F = [&](long long x) {
      long long s = 0;
      for (int64_t b = 0; b < k; b++) s += x > bw[b] ? x - bw[b] : 0;
      return s;
    };
    while (hi - lo > 1) {
      const long long mid = lo + (hi - lo) / 2;
      if (F(mid) <= j) lo = mid;
      else hi = mid;
    }
    long long rem = j - F(lo);
    int pick = 0;
    for (int64_t b = 0; b < k; b++)
      if (bw[b] <= lo) {
        if (rem == 0) {
          pick = (int)b;
          break;
        }
        rem--;
      }
    part_full[v] = pick;
  }
}

// Degree-0 vertices with general weights: one thread applies the greedy rule in id order.
__global__ void k_place_seq(DGraph g, const int32_t *rank, const int32_t *part0, long long *bw, int64_t k,
                            int32_t *part_full) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int64_t v = 0; v < g.n; v++) {
    const int r = rank[v];
    if (r >= 0) {
      part_full[v] = part0[r];
      continue;
    }
    int b = 0;
    for (int64_t x = 1; x < k; x++)
      if (bw[x] < bw[b]) b = (int)x;
    part_full[v] = b;
    bw[b] += g.vweight(v);
  }
}

// rank_out[v] = rank[v] for vertices with neighbours, -1 otherwise; iso_idx[v] = v - rank[v]
// (the number of degree-0 vertices before v, since rank counts the kept vertices before v).
__global__ void k_mark_rank(DGraph g, const int32_t *rank, int32_t *rank_out, int64_t *iso_idx) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = g.row_begin(v + 1) - g.row_begin(v);
    rank_out[v] = d > 0 ? rank[v] : -1;
    iso_idx[v] = v - rank[v];
  }
}

int grid_for_n(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8));
}

}  // namespace

int initial_partition_multi(const IpJob *jobs, int njobs, int tries, int repair_rounds, cudaStream_t s,
                            int *err_dev) {
  if (njobs <= 0) return GP_OK;
  Workspace ws(s);
  std::vector<IpGraph> hg(njobs);
  std::vector<int> bgraph, btry;
  int64_t scr = 0, kscr = 0, cscr = 0;
  for (int j = 0; j < njobs; j++) {
    const IpJob &jb = jobs[j];
    if (jb.g.n >= (1 << 30)) {
      set_error("initial partitioning supports coarsest graphs below 2^30 vertices");
      return GP_ERR_UNSUPPORTED;
    }
    IpGraph &G = hg[j];
    G.g = jb.g;
    G.vbase = jb.vbase;
    G.k = jb.k;
    G.level = jb.level;
    G.lmax = jb.lmax;
    G.seed = jb.seed;
    G.parts = jb.parts;
    G.ns = std::max<int64_t>(std::max<int64_t>(jb.g.n, jb.k), 1);
    G.scr_off = scr;
    G.kscr_off = kscr;
    G.conn_off = cscr;
    scr += (int64_t)tries * G.ns;
    kscr += (int64_t)tries * jb.k;
    cscr += (int64_t)tries * kIpThreads * jb.k;
    for (int t = 0; t < tries; t++) {
      bgraph.push_back(j);
      btry.push_back(t);
    }
  }
  IpArgs a;
  a.repair_rounds = repair_rounds;
  GP_TRY(ws.get(&a.gk, (size_t)scr));
  GP_TRY(ws.get(&a.dist, (size_t)scr));
  GP_TRY(ws.get(&a.qa, (size_t)scr));
  GP_TRY(ws.get(&a.qb, (size_t)scr));
  GP_TRY(ws.get(&a.ka, (size_t)scr));
  GP_TRY(ws.get(&a.kb, (size_t)scr));
  GP_TRY(ws.get(&a.va, (size_t)scr));
  GP_TRY(ws.get(&a.vb, (size_t)scr));
  GP_TRY(ws.get(&a.mv_t, (size_t)scr));
  GP_TRY(ws.get(&a.mv_g, (size_t)scr));
  GP_TRY(ws.get(&a.flag, (size_t)scr));
  GP_TRY(ws.get(&a.gws, (size_t)kscr));
  GP_TRY(ws.get(&a.gminh, (size_t)kscr));
  GP_TRY(ws.get(&a.gstart, (size_t)kscr));
  GP_TRY(ws.get(&a.gfar, (size_t)kscr));
  GP_TRY(ws.get(&a.bw, (size_t)kscr));
  GP_TRY(ws.get(&a.conn, (size_t)cscr));
  GP_TRY(ws.zeros(&a.err, 1));
  IpGraph *graphs_dev;
  int *bg_dev, *bt_dev;
  GP_TRY(ws.get(&graphs_dev, hg.size()));
  GP_TRY(ws.get(&bg_dev, bgraph.size()));
  GP_TRY(ws.get(&bt_dev, btry.size()));
  GP_CUDA(cudaMemcpyAsync(graphs_dev, hg.data(), sizeof(IpGraph) * hg.size(), cudaMemcpyHostToDevice, s));
  GP_CUDA(cudaMemcpyAsync(bg_dev, bgraph.data(), sizeof(int) * bgraph.size(), cudaMemcpyHostToDevice, s));
  GP_CUDA(cudaMemcpyAsync(bt_dev, btry.data(), sizeof(int) * btry.size(), cudaMemcpyHostToDevice, s));
  a.graphs = graphs_dev;
  a.block_graph = bg_dev;
  a.block_try = bt_dev;
  const int grid = (int)bgraph.size();
  int64_t max_ns = 0;
  for (const IpGraph &G : hg) max_ns = std::max<int64_t>(max_ns, G.ns);
  a.smem_ns = max_ns <= kIpSmemMaxNs ? max_ns : 0;
  a.smem_sort = max_ns <= kIpSmemSortNs ? 1 : 0;
  const size_t dsm = a.smem_ns > 0 ? ip_smem_bytes(a.smem_ns, a.smem_sort != 0) : 0;
  if (dsm > 0) {  // (per call: the attribute belongs to the current device)
    const size_t cap = std::max(ip_smem_bytes(kIpSmemMaxNs, false), ip_smem_bytes(kIpSmemSortNs, true));
    GP_CUDA(cudaFuncSetAttribute(k_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
  }
  (::gp::count_launch(), k_bisect<<<grid, kIpThreads, dsm, s>>>(a));
  GP_LAUNCH_CHECK();
  (::gp::count_launch(), k_repair<<<grid, kIpThreads, 0, s>>>(a));
  GP_LAUNCH_CHECK();
  if (err_dev) {
    GP_CUDA(cudaMemcpyAsync(err_dev, a.err, sizeof(int), cudaMemcpyDeviceToDevice, s));
    return GP_OK;
  }
  int err = 0;
  GP_CUDA(cudaMemcpyAsync(&err, a.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  if (err) {
    set_error("initial partitioning: gain range too wide for the repair sort keys");
    return err;
  }
  return GP_OK;
}

int initial_partition(const DGraph &g, int k, int64_t lmax, uint64_t seed, int level, int tries, int repair_rounds,
                      int32_t *parts, cudaStream_t s, int *err_dev) {
  IpJob j;
  j.g = g;
  j.vbase = 0;
  j.k = k;
  j.lmax = lmax;
  j.seed = seed;
  j.level = level;
  j.parts = parts;
  return initial_partition_multi(&j, 1, tries, repair_rounds, s, err_dev);
}

int eval_cut_launch(const DGraph &g, const int32_t *part, int64_t k, unsigned long long *acc_dev, int64_t *bw_dev,
                    cudaStream_t s) {
  GP_CUDA(cudaMemsetAsync(acc_dev, 0, sizeof(unsigned long long), s));
  if (g.n > 0) {
    Workspace ws(s);
    unsigned long long *items, *cnt;
    // items: at most one per kCutChunk entries plus one per row above kCutSmall
    const unsigned long long cap = (unsigned long long)(g.m / kCutChunk + g.m / (kCutSmall + 1) + 1);
    GP_TRY(ws.get(&items, (size_t)cap));
    GP_TRY(ws.zeros(&cnt, 1));
    (::gp::count_launch(), k_cut<<<grid_for_n(g.n), 256, 0, s>>>(g, part, acc_dev));
    (::gp::count_launch(), k_cut_list<<<grid_for_n(g.n), 256, 0, s>>>(g, items, cap, cnt));
    (::gp::count_launch(), k_cut_items<<<num_sms() * 8, 256, 0, s>>>(g, part, items, cap, cnt, acc_dev));
    GP_LAUNCH_CHECK();
  }
  if (bw_dev) GP_TRY(block_weights(g, part, k, bw_dev, nullptr, s));
  return GP_OK;
}

int eval_cut(const DGraph &g, const int32_t *part, int64_t k, int64_t *cut_host, int64_t *bw_dev, cudaStream_t s) {
  Workspace ws(s);
  unsigned long long *acc;
  GP_TRY(ws.get(&acc, 1));
  GP_TRY(eval_cut_launch(g, part, k, acc, bw_dev, s));
  unsigned long long h = 0;
  GP_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  *cut_host = (int64_t)(h / 2);
  return GP_OK;
}

int project(const int32_t *coarse, const int32_t *f2c, int64_t n, int32_t *fine, cudaStream_t s) {
  if (n == 0) return GP_OK;
  (::gp::count_launch(), k_project<<<grid_for_n(n), 256, 0, s>>>(coarse, f2c, n, fine));
  GP_LAUNCH_CHECK();
  return GP_OK;
}

int vertex_weight_stats(const DGraph &g, int64_t *maxc, int64_t *total, cudaStream_t s) {
  Workspace ws(s);
  unsigned long long *d;
  GP_TRY(ws.zeros(&d, 2));
  if (g.n > 0) {
    (::gp::count_launch(), k_vw_stats<<<grid_for_n(g.n), 256, 0, s>>>(g, d, d + 1));
    GP_LAUNCH_CHECK();
  }
  unsigned long long h[2];
  GP_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  if (maxc) *maxc = (int64_t)h[0];
  if (total) *total = (int64_t)h[1];
  return GP_OK;
}

int strip_isolated(const DGraph &g, Stripped *out, Workspace &ws, cudaStream_t s, int64_t *W_out,
                   int64_t *maxc_kept_out, const LpConfig *cfg, LpClassInfo *cls) {
  out->g0 = g;
  out->n0 = g.n;
  out->n_iso = 0;
  out->rank = nullptr;
  if (W_out) *W_out = 0;
  if (maxc_kept_out) *maxc_kept_out = 0;
  if (g.n == 0) return GP_OK;
  uint32_t *keep;
  int64_t *deg, *total;
  int32_t *rank;
  GP_TRY(ws.get(&keep, (size_t)g.n));
  GP_TRY(ws.get(&deg, (size_t)g.n));
  GP_TRY(ws.get(&rank, (size_t)g.n));
  // total[0] = kept vertices, total[1] = max kept weight, total[2] = total weight (one read back)
  GP_TRY(ws.zeros(&total, 3));
  const bool stats = W_out || maxc_kept_out;
  (::gp::count_launch(), k_deg_flags<<<grid_for_n(g.n), 256, 0, s>>>(
                             g, keep, deg, stats ? reinterpret_cast<unsigned long long *>(total + 1) : nullptr));
  GP_LAUNCH_CHECK();
  GP_TRY(scan_excl_u32(keep, rank, g.n, total, ws));
  // the LP degree classes of g, valid for the level-0 graph when no vertex is stripped
  unsigned long long *cls_dev = nullptr;
  unsigned long long cls_words[kLpClassWords];
  if (cfg && cls) {
    GP_TRY(ws.get(&cls_dev, (size_t)kLpClassWords));
    GP_TRY(lp_classes_launch(g, *cfg, cls_dev, ws));
  }
  int64_t h[3] = {0, 0, 0};
  Readback rb;
  rb.add(h, total, sizeof(h));
  if (cls_dev) rb.add(cls_words, cls_dev, sizeof(cls_words));
  GP_TRY(rb.run(s));
  const int64_t n0 = h[0];
  if (maxc_kept_out) *maxc_kept_out = h[1];
  if (W_out) *W_out = h[2];
  if (cls_dev && n0 == g.n) lp_classes_from(cls_words, *cfg, cls);
  if (n0 == g.n) return GP_OK;
  out->n0 = n0;
  out->n_iso = g.n - n0;
  out->rank = rank;
  // rank of kept vertices = exclusive count of kept before v; degree-0 ones are marked -1 later
  int64_t *off0;
  GP_TRY(ws.get(&off0, (size_t)n0 + 1));
  void *vw0 = nullptr;
  if (g.vw) {
    if (g.vw64) {
      int64_t *p;
      GP_TRY(ws.get(&p, (size_t)std::max<int64_t>(n0, 1)));
      vw0 = p;
    } else {
      int32_t *p;
      GP_TRY(ws.get(&p, (size_t)std::max<int64_t>(n0, 1)));
      vw0 = p;
    }
  }
  int32_t *adj0;
  GP_TRY(ws.get(&adj0, (size_t)std::max<int64_t>(g.m, 1)));
  (::gp::count_launch(), k_strip_rows<<<grid_for_n(g.n), 256, 0, s>>>(g, rank, keep, n0, off0, vw0));
  if (g.m > 0) (::gp::count_launch(), k_strip_adj<<<grid_for_n(g.m), 256, 0, s>>>(g.adj, g.m, rank, adj0));
  GP_LAUNCH_CHECK();
  DGraph d;
  d.n = n0;
  d.m = g.m;
  d.off = off0;
  d.off64 = 1;
  d.adj = adj0;
  d.vw = vw0;
  d.vw64 = g.vw64;
  d.ew = g.ew;  // same entries in the same order
  d.ew64 = g.ew64;
  out->g0 = d;
  return GP_OK;
}

int place_isolated(const DGraph &g, const Stripped &st, const int32_t *part0, int64_t k, int32_t *part_full,
                   cudaStream_t s) {
  Workspace ws(s);
  if (st.n_iso == 0) {
    if (g.n) GP_CUDA(cudaMemcpyAsync(part_full, part0, sizeof(int32_t) * (size_t)g.n, cudaMemcpyDeviceToDevice, s));
    return GP_OK;
  }
  // block weights of the kept vertices
  long long *bw;
  GP_TRY(ws.zeros(&bw, (size_t)k));
  GP_TRY(block_weights(st.g0, part0, k, reinterpret_cast<int64_t *>(bw), nullptr, s));
  // rank[v] becomes -1 for degree-0 vertices; iso_idx[v] = number of degree-0 vertices before v
  int32_t *rank;
  int64_t *iso_idx;
  GP_TRY(ws.get(&rank, (size_t)g.n));
  GP_TRY(ws.get(&iso_idx, (size_t)g.n));
  (::gp::count_launch(), k_mark_rank<<<grid_for_n(g.n), 256, 0, s>>>(g, st.rank, rank, iso_idx));
  GP_LAUNCH_CHECK();
  if (!g.vw) {
    (::gp::count_launch(), k_place_unit<<<grid_for_n(g.n), 256, 0, s>>>(g, rank, part0, iso_idx, bw, k, part_full));
  } else {
    (::gp::count_launch(), k_place_seq<<<1, 32, 0, s>>>(g, rank, part0, bw, k, part_full));
  }
  GP_LAUNCH_CHECK();
  return GP_OK;
}

}  // namespace gp
