// partition.cpp -- oracle: initial partitioning, balance repair, evaluation and the multilevel driver.
//
// TEST INFRASTRUCTURE ONLY (CPU oracle; shares no code with the GPU library).
//
// The multilevel scheme (Section I, Section III): coarsen by label-propagation clustering and
// contraction until the graph is small, partition the coarsest graph several times and keep the
// best (Section III-B, Section IV-B: max(p, I) tries, I = 4), then project the partition level by
// level ("a vertex in the finer graph is assigned the block of its coarse representative",
// Section III-C) and improve it with label propagation under U = Lmax (Section IV-C, 25 iterations,
// Section VI "Algorithm Configuration"). Multi-try local search is not part of this path.
//
// Readings of what the paper leaves open:
//   * cluster bound U = max(max_v c(v), floor(Lmax / f)), f = 14;
//   * coarsening stops when n <= T = max(2000, 64 k), when a contraction keeps more than 95% of the
//     vertices (that level is kept), or after 64 contractions;
//   * degree-0 vertices are removed before coarsening and, after refinement, given in ascending id
//     order to the block of minimum weight (ties: smaller block id);
//   * the initial partitioner (KaHIP's, Section III-B, is external) is a deterministic recursive
//     bisection into ceil(k/2) and floor(k/2) blocks: BFS from the vertex of minimum
//     H(s_try, depth, v), a second BFS from the farthest vertex found (ties: smaller id), vertices
//     ordered by (distance, id) with unreachable ones last, side 0 the shortest prefix whose weight
//     reaches the ceil(k/2)/k share; then balance repair, then LP refinement;
//   * the best try is the minimum of (cut, imbalanced, try index);
//   * with coarsen_mode = 1 the clustering of each level is the matching of match.cpp (same bound U,
//     rounds_coarsen rounds at most, the same seed H(seed, l, 1)) instead of label propagation;
//   * with mls != 0, multi-try k-way local search (mls.cpp, seed H(seed, l, 7)) follows the LP
//     refinement of every level, the coarsest one (after the best try is kept) included.
// Seeds: coarsening LP at level l uses H(seed, l, 1); refinement at level l uses H(seed, l, 2); IP
// try t on the coarsest level c uses s_try = H(seed, c, 4 + t) and refines with H(s_try, c, 3).
#include <algorithm>
#include <numeric>
#include <vector>

#include "oracle.h"

namespace {

struct OwnedGraph {
  int64_t n = 0, m = 0;
  std::vector<int64_t> off, vw, ew;
  std::vector<int32_t> adj;
  or_graph view() const {
    or_graph g;
    g.n = n;
    g.m_dir = m;
    g.off = off.data();
    g.adj = adj.data();
    g.vw = vw.data();
    g.ew = ew.data();
    return g;
  }
};

inline int64_t vweight(const or_graph *g, int64_t v) { return g->vw ? g->vw[v] : 1; }
inline int64_t eweight(const or_graph *g, int64_t e) { return g->ew ? g->ew[e] : 1; }

// Breadth-first distances from src inside the vertex set marked with `stamp`; -1 = unreachable.
void bfs_in_set(const or_graph *g, int32_t src, const std::vector<int64_t> &mark, int64_t stamp,
                std::vector<int64_t> &dist) {
  std::vector<int32_t> queue;
  dist[src] = 0;
  queue.push_back(src);
  for (size_t h = 0; h < queue.size(); h++) {
    const int32_t x = queue[h];
    for (int64_t e = g->off[x]; e < g->off[x + 1]; e++) {
      const int32_t u = g->adj[e];
      if (mark[u] != stamp || dist[u] >= 0) continue;
      dist[u] = dist[x] + 1;
      queue.push_back(u);
    }
  }
}

struct Bisector {
  const or_graph *g;
  uint64_t s_try;
  int32_t *part;
  std::vector<int64_t> mark, dist;
  int64_t next_stamp = 1;

  // S: vertices (ascending id) to split into kS blocks numbered base .. base+kS-1.
  void run(std::vector<int32_t> S, int64_t kS, int64_t base, int64_t depth) {
    if (kS == 1) {
      for (int32_t v : S) part[v] = (int32_t)base;
      return;
    }
    const int64_t k0 = (kS + 1) / 2, k1 = kS / 2;
    std::vector<int32_t> side0, side1;
    if (!S.empty()) {
      const int64_t stamp = next_stamp++;
      int64_t WS = 0;
      for (int32_t v : S) {
        mark[v] = stamp;
        WS += vweight(g, v);
      }
      // Start vertex: minimum H(s_try, depth, v), ties by id.
      int32_t start = S[0];
      uint64_t hs = or_hash3(s_try, (uint64_t)depth, (uint64_t)S[0]);
      for (int32_t v : S) {
        const uint64_t h = or_hash3(s_try, (uint64_t)depth, (uint64_t)v);
        if (h < hs) {
          hs = h;
          start = v;
        }
      }
      for (int32_t v : S) dist[v] = -1;
      bfs_in_set(g, start, mark, stamp, dist);
      // Pseudo-peripheral vertex: farthest from start, ties by smaller id.
      int32_t far = start;
      for (int32_t v : S)
        if (dist[v] > dist[far]) far = v;
      for (int32_t v : S) dist[v] = -1;
      bfs_in_set(g, far, mark, stamp, dist);
      std::vector<int32_t> order(S);
      std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        const bool ra = dist[a] >= 0, rb = dist[b] >= 0;
        if (ra != rb) return ra;  // reachable first
        if (ra && dist[a] != dist[b]) return dist[a] < dist[b];
        return a < b;
      });
      // Side 0: the shortest prefix P with c(P) >= WS * k0 / kS.
      int64_t acc = 0;
      size_t cut_at = order.size();
      for (size_t i = 0; i < order.size(); i++) {
        acc += vweight(g, order[i]);
        if (acc * kS >= WS * k0) {
          cut_at = i + 1;
          break;
        }
      }
      side0.assign(order.begin(), order.begin() + (long)cut_at);
      side1.assign(order.begin() + (long)cut_at, order.end());
      std::sort(side0.begin(), side0.end());
      std::sort(side1.begin(), side1.end());
    }
    run(side0, k0, base, depth + 1);
    run(side1, k1, base + k0, depth + 1);
  }
};

}  // namespace

extern "C" int64_t or_cut(const or_graph *g, const int32_t *part, int64_t k, int64_t *bw) {
  if (bw) {
    for (int64_t b = 0; b < k; b++) bw[b] = 0;
    for (int64_t v = 0; v < g->n; v++) bw[part[v]] += vweight(g, v);
  }
  int64_t twice = 0;
  for (int64_t v = 0; v < g->n; v++)
    for (int64_t e = g->off[v]; e < g->off[v + 1]; e++)
      if (part[v] != part[g->adj[e]]) twice += eweight(g, e);
  return twice / 2;
}

extern "C" int or_bisect(const or_graph *g, int64_t k, uint64_t s_try, int32_t *part) {
  Bisector b;
  b.g = g;
  b.s_try = s_try;
  b.part = part;
  b.mark.assign(g->n, 0);
  b.dist.assign(g->n, -1);
  std::vector<int32_t> all(g->n);
  std::iota(all.begin(), all.end(), 0);
  b.run(all, k, 0, 0);
  return 0;
}

// Balance repair: vertices of overloaded blocks move to the eligible neighbouring block of largest
// connection (ties: smaller id), else to the lightest block when it can take them. Movers are
// admitted per target in (gain desc, id asc) order while the target stays <= Lmax, and a source
// stops giving vertices once it is <= Lmax.
extern "C" int64_t or_repair(const or_graph *g, int64_t k, int64_t lmax, int64_t max_rounds,
                             int32_t *part) {
  const int64_t n = g->n;
  std::vector<int64_t> bw(k);
  for (int64_t rr = 0; rr < max_rounds; rr++) {
    std::fill(bw.begin(), bw.end(), 0);
    for (int64_t v = 0; v < n; v++) bw[part[v]] += vweight(g, v);
    if (*std::max_element(bw.begin(), bw.end()) <= lmax) return rr;
    int64_t lightest = 0;
    for (int64_t b = 1; b < k; b++)
      if (bw[b] < bw[lightest]) lightest = b;
    struct M {
      int32_t v, from, to;
      int64_t gain;
    };
    std::vector<M> movers;
    std::vector<int64_t> conn(k, 0);
    for (int64_t v = 0; v < n; v++) {
      const int32_t P = part[v];
      if (bw[P] <= lmax) continue;
      const int64_t cv = vweight(g, v);
      for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) conn[part[g->adj[e]]] += eweight(g, e);
      int32_t best = -1;
      for (int64_t B = 0; B < k; B++) {
        if (B == P || conn[B] <= 0 || bw[B] + cv > lmax) continue;
        if (best < 0 || conn[B] > conn[best]) best = (int32_t)B;
      }
      if (best < 0 && lightest != P && bw[lightest] + cv <= lmax) best = (int32_t)lightest;
      if (best >= 0) movers.push_back({(int32_t)v, P, best, conn[best] - conn[P]});
      for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) conn[part[g->adj[e]]] = 0;
    }
    auto order = [](const M &a, const M &b) {
      if (a.gain != b.gain) return a.gain > b.gain;
      return a.v < b.v;
    };
    // Per target: longest prefix that fits.
    std::stable_sort(movers.begin(), movers.end(), [&](const M &a, const M &b) {
      if (a.to != b.to) return a.to < b.to;
      return order(a, b);
    });
    std::vector<M> into;
    for (size_t i = 0; i < movers.size();) {
      size_t j = i;
      int64_t acc = 0;
      bool open = true;
      for (; j < movers.size() && movers[j].to == movers[i].to; j++) {
        acc += vweight(g, movers[j].v);
        if (open && bw[movers[j].to] + acc <= lmax) into.push_back(movers[j]);
        else open = false;
      }
      i = j;
    }
    // Per source: take movers while the source is still overloaded.
    std::stable_sort(into.begin(), into.end(), [&](const M &a, const M &b) {
      if (a.from != b.from) return a.from < b.from;
      return order(a, b);
    });
    int64_t applied = 0;
    for (size_t i = 0; i < into.size();) {
      size_t j = i;
      int64_t removed = 0;
      for (; j < into.size() && into[j].from == into[i].from; j++) {
        if (bw[into[j].from] - removed > lmax) {
          removed += vweight(g, into[j].v);
          part[into[j].v] = into[j].to;
          applied++;
        }
      }
      i = j;
    }
    if (applied == 0) return rr + 1;
  }
  return max_rounds;
}

extern "C" void or_default_params(or_params *p) {
  p->cluster_div = 14;
  p->rounds_coarsen = 10;
  p->rounds_refine = 25;
  p->coarse_min = 2000;
  p->coarse_per_k = 64;
  p->stall_pct = 95;
  p->max_levels = 64;
  p->ip_tries = 4;
  p->repair_rounds = 16;
  p->coarsen_mode = 0;
  p->mls = 0;
  p->lp_async = 0;
}

extern "C" int or_partition(const or_graph *g, int64_t k, double eps, uint64_t seed,
                            const or_params *pp, const int32_t *const *q_levels, int64_t n_q_levels,
                            int32_t *part, or_result *res) {
  or_params p;
  if (pp) p = *pp;
  else or_default_params(&p);
  const int64_t n = g->n;
  if (k < 1 || eps < 0.0 || k > n || p.ip_tries < 1 || p.ip_tries > 16) return -1;
  *res = or_result();
  int64_t W = 0;
  for (int64_t v = 0; v < n; v++) W += vweight(g, v);
  const int64_t lmax = or_lmax(W, k, eps);
  res->lmax = lmax;

  // Remove degree-0 vertices: level 0 is the graph induced by the others, ids by rank.
  std::vector<int64_t> rank(n, -1);
  int64_t n0 = 0;
  for (int64_t v = 0; v < n; v++)
    if (g->off[v + 1] > g->off[v]) rank[v] = n0++;
  res->n_isolated = n - n0;
  std::vector<OwnedGraph> G(1);
  {
    OwnedGraph &L0 = G[0];
    L0.n = n0;
    L0.off.assign(n0 + 1, 0);
    L0.vw.resize(n0);
    for (int64_t v = 0; v < n; v++)
      if (rank[v] >= 0) {
        L0.off[rank[v] + 1] = g->off[v + 1] - g->off[v];
        L0.vw[rank[v]] = vweight(g, v);
      }
    for (int64_t i = 0; i < n0; i++) L0.off[i + 1] += L0.off[i];
    L0.m = L0.off[n0];
    L0.adj.resize(L0.m);
    L0.ew.resize(L0.m);
    for (int64_t v = 0; v < n; v++) {
      if (rank[v] < 0) continue;
      int64_t pos = L0.off[rank[v]];
      for (int64_t e = g->off[v]; e < g->off[v + 1]; e++, pos++) {
        L0.adj[pos] = (int32_t)rank[g->adj[e]];
        L0.ew[pos] = eweight(g, e);
      }
    }
  }
  std::vector<std::vector<int32_t>> f2c;
  std::vector<int32_t> cur;  // partition of the current level graph

  if (n0 > 0) {
    // Coarsening.
    const int64_t T = std::max(p.coarse_min, p.coarse_per_k * k);
    while (G.back().n > T && (int64_t)f2c.size() < p.max_levels) {
      const int64_t l = (int64_t)f2c.size();
      const or_graph gl = G.back().view();
      int64_t maxc = 0;
      for (int64_t v = 0; v < gl.n; v++) maxc = std::max(maxc, gl.vw[v]);
      const int64_t U = std::max(maxc, lmax / p.cluster_div);
      std::vector<int32_t> labels(gl.n);
      std::iota(labels.begin(), labels.end(), 0);
      std::vector<int64_t> lw(gl.vw, gl.vw + gl.n);
      const int32_t *q = nullptr;
      if (q_levels) {
        if (l >= n_q_levels) return -2;
        q = q_levels[l];
      }
      if (p.coarsen_mode == 1) {
        or_match(&gl, U, p.rounds_coarsen, or_hash3(seed, (uint64_t)l, 1), labels.data(), nullptr);
      } else {
        or_lp_stats ls;
        if (p.lp_async)
          or_lp_async(&gl, labels.data(), lw.data(), gl.n, U, p.rounds_coarsen, or_hash3(seed, (uint64_t)l, 1), &ls);
        else
          or_lp(&gl, q, labels.data(), lw.data(), gl.n, U, p.rounds_coarsen, or_hash3(seed, (uint64_t)l, 1), &ls);
        res->lp_edges += ls.edges;
      }
      OwnedGraph c;
      c.off.resize(gl.n + 1);
      c.adj.resize(gl.m_dir);
      c.vw.resize(gl.n);
      c.ew.resize(gl.m_dir);
      std::vector<int32_t> map(gl.n);
      or_contract(&gl, labels.data(), gl.n, &c.n, &c.m, c.off.data(), c.adj.data(), c.vw.data(),
                  c.ew.data(), map.data());
      c.off.resize(c.n + 1);
      c.adj.resize(c.m);
      c.vw.resize(c.n);
      c.ew.resize(c.m);
      const int64_t n_before = gl.n;
      G.push_back(std::move(c));
      f2c.push_back(std::move(map));
      if (100 * G.back().n > p.stall_pct * n_before) break;
    }
    const int64_t levels = (int64_t)f2c.size();
    // Initial partitioning: best of ip_tries tries.
    const or_graph gc = G.back().view();
    int64_t best_cut = -1, best_imb = 0;
    for (int64_t t = 0; t < p.ip_tries; t++) {
      const uint64_t s_try = or_hash3(seed, (uint64_t)levels, (uint64_t)(4 + t));
      std::vector<int32_t> pt(gc.n);
      or_bisect(&gc, k, s_try, pt.data());
      or_repair(&gc, k, lmax, p.repair_rounds, pt.data());
      std::vector<int64_t> bw(k);
      or_cut(&gc, pt.data(), k, bw.data());
      or_lp_stats ls;
      if (p.lp_async)
        or_lp_async(&gc, pt.data(), bw.data(), k, lmax, p.rounds_refine, or_hash3(s_try, (uint64_t)levels, 3), &ls);
      else
        or_lp(&gc, nullptr, pt.data(), bw.data(), k, lmax, p.rounds_refine, or_hash3(s_try, (uint64_t)levels, 3),
              &ls);
      res->lp_edges += ls.edges;
      const int64_t cut = or_cut(&gc, pt.data(), k, bw.data());
      const int64_t imb = *std::max_element(bw.begin(), bw.end()) > lmax ? 1 : 0;
      res->try_cut[t] = cut;
      res->try_imbalanced[t] = imb;
      if (best_cut < 0 || cut < best_cut || (cut == best_cut && imb < best_imb)) {
        best_cut = cut;
        best_imb = imb;
        res->best_try = t;
        cur = pt;
      }
    }
    or_mls_params mp;
    or_mls_default_params(&mp);
    mp.global_iters = p.mls;
    if (p.mls) {
      const or_graph gcv = G.back().view();
      or_mls(&gcv, k, lmax, or_hash3(seed, (uint64_t)levels, 7), &mp, cur.data(), nullptr);
    }
    // Uncoarsening: project, then refine.
    for (int64_t l = levels - 1; l >= 0; l--) {
      const or_graph gl = G[l].view();
      std::vector<int32_t> fine(gl.n);
      for (int64_t v = 0; v < gl.n; v++) fine[v] = cur[f2c[l][v]];
      std::vector<int64_t> bw(k);
      or_cut(&gl, fine.data(), k, bw.data());
      or_lp_stats ls;
      if (p.lp_async)
        or_lp_async(&gl, fine.data(), bw.data(), k, lmax, p.rounds_refine, or_hash3(seed, (uint64_t)l, 2), &ls);
      else
        or_lp(&gl, nullptr, fine.data(), bw.data(), k, lmax, p.rounds_refine, or_hash3(seed, (uint64_t)l, 2), &ls);
      res->lp_edges += ls.edges;
      if (p.mls) or_mls(&gl, k, lmax, or_hash3(seed, (uint64_t)l, 7), &mp, fine.data(), nullptr);
      cur.swap(fine);
    }
    res->levels = levels;
  }
  for (size_t l = 0; l < G.size() && l < 65; l++) {
    res->level_n[l] = G[l].n;
    res->level_m[l] = G[l].m;
  }
  // Degree-0 vertices: ascending id order, each to the currently lightest block.
  std::vector<int64_t> bw(k, 0);
  for (int64_t v = 0; v < n; v++)
    if (rank[v] >= 0) {
      part[v] = cur[rank[v]];
      bw[part[v]] += vweight(g, v);
    }
  for (int64_t v = 0; v < n; v++) {
    if (rank[v] >= 0) continue;
    int64_t b = 0;
    for (int64_t x = 1; x < k; x++)
      if (bw[x] < bw[b]) b = x;
    part[v] = (int32_t)b;
    bw[b] += vweight(g, v);
  }
  res->cut = or_cut(g, part, k, nullptr);
  res->max_block_weight = *std::max_element(bw.begin(), bw.end());
  res->imbalanced = res->max_block_weight > lmax ? 1 : 0;
  return 0;
}
