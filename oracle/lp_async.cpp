// lp_async.cpp -- oracle: the paper's sequential label propagation order (a comparator).
//
// TEST INFRASTRUCTURE ONLY (CPU oracle; shares no code with the GPU library).
//
// Section III-A ("Clustering") describes size-constrained label propagation as a sequential,
// in-place (Gauss-Seidel) sweep: all vertices start in a queue in increasing order of their degrees;
// an iteration visits the queued vertices in that order, each moves at once to the eligible cluster of
// strongest connection (a cluster stays within U), and the neighbours of moved vertices are queued for
// the next iteration; it stops after l iterations or an iteration without moves. Section IV-A runs it
// asynchronously on packets of the degree-sorted order with the cluster sizes updated by compare-and-
// swap. This function is that sequential order; the GPU's asynchronous form reproduces it exactly when
// it runs on a single warp, and is a non-deterministic comparator for the library's deterministic
// Jacobi rounds otherwise.
//
// Readings: the order is (degree, id) ascending and the same in every iteration (restricted to the
// queued vertices); ties go to the own label, then to the larger H(seed, v, L), then to the smaller L
// (the paper breaks ties at random); a vertex is queued for the next iteration when a neighbour moved.
#include <algorithm>
#include <map>
#include <numeric>
#include <vector>

#include "oracle.h"

namespace {
inline int64_t vweight(const or_graph *g, int64_t v) { return g->vw ? g->vw[v] : 1; }
inline int64_t eweight(const or_graph *g, int64_t e) { return g->ew ? g->ew[e] : 1; }
}  // namespace

extern "C" int or_lp_async(const or_graph *g, int32_t *labels, int64_t *lw, int64_t nl, int64_t U, int64_t rounds,
                           uint64_t seed, or_lp_stats *st) {
  (void)nl;
  const int64_t n = g->n;
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return g->off[a + 1] - g->off[a] < g->off[b + 1] - g->off[b];
  });
  std::vector<uint8_t> active(n, 1), next(n, 0);
  or_lp_stats s = {0, 0, 0, 0, 0};
  for (int64_t r = 0; r < rounds; r++) {
    int64_t moves = 0;
    std::fill(next.begin(), next.end(), 0);
    for (int32_t v : order) {
      if (!active[v]) continue;
      s.visits++;
      s.edges += g->off[v + 1] - g->off[v];
      std::map<int32_t, int64_t> conn;
      for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) conn[labels[g->adj[e]]] += eweight(g, e);
      const int32_t own = labels[v];
      const int64_t own_conn = conn.count(own) ? conn[own] : 0;
      const int64_t cv = vweight(g, v);
      int32_t best = -1;
      int64_t best_conn = 0;
      uint64_t best_h = 0;
      for (const auto &kv : conn) {
        const int32_t L = kv.first;
        if (L == own || kv.second <= own_conn || lw[L] + cv > U) continue;
        const uint64_t h = or_hash3(seed, (uint64_t)v, (uint64_t)L);
        bool better;
        if (best < 0) better = true;
        else if (kv.second != best_conn) better = kv.second > best_conn;
        else if (h != best_h) better = h > best_h;
        else better = L < best;
        if (better) {
          best = L;
          best_conn = kv.second;
          best_h = h;
        }
      }
      if (best < 0) continue;
      s.movers++;
      lw[own] -= cv;
      lw[best] += cv;
      labels[v] = best;
      moves++;
      for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) next[g->adj[e]] = 1;
    }
    s.rounds = r + 1;
    s.moves += moves;
    active.swap(next);
    if (moves == 0) break;
  }
  if (st) *st = s;
  return 0;
}
