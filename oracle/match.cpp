// match.cpp -- oracle: matching-based clustering for the coarsening phase.
//
// TEST INFRASTRUCTURE ONLY (CPU oracle; shares no code with the GPU library).
//
// The paper's clustering (Section III-A) names matching algorithms -- clusters of size two -- as the
// other family of clusterings, and its conclusion (Section VII) plans a high-quality parallel matching
// for the coarsening of mesh-like graphs. The paper fixes no algorithm; the reading implemented here
// is a deterministic handshake matching with the edge rating
//     rho(u, v) = omega(u, v)^2 / (c(u) c(v))
// (heavier edges between lighter vertices first):
//   * every round, each unmatched vertex v proposes to its best unmatched neighbour u with
//     c(v) + c(u) <= U: largest rho, then larger H(seed, min(u,v), max(u,v)), then smaller u;
//     the ratings are compared exactly, omega1^2 c(u2) against omega2^2 c(u1) in 128-bit integers;
//   * v and u are matched when they propose to each other; all decisions of a round read the
//     matching at its start;
//   * rounds repeat until one matches nothing or `rounds` rounds have run;
//   * the clustering is label(v) = min(v, mate(v)) for matched v, else v, and contracts like any
//     clustering (Section III-A).
#include <vector>

#include "oracle.h"

namespace {
inline int64_t vweight(const or_graph *g, int64_t v) { return g->vw ? g->vw[v] : 1; }
inline int64_t eweight(const or_graph *g, int64_t e) { return g->ew ? g->ew[e] : 1; }
typedef unsigned __int128 u128;
}  // namespace

extern "C" int or_match(const or_graph *g, int64_t U, int64_t rounds, uint64_t seed, int32_t *labels,
                        or_match_stats *st) {
  const int64_t n = g->n;
  std::vector<int32_t> mate(n, -1), prop(n, -1);
  or_match_stats s = {0, 0};
  for (int64_t r = 0; r < rounds; r++) {
    // proposals from the matching at the start of the round
    for (int64_t v = 0; v < n; v++) {
      prop[v] = -1;
      if (mate[v] >= 0) continue;
      const int64_t cv = vweight(g, v);
      int32_t best = -1;
      int64_t best_w = 0, best_c = 0;
      uint64_t best_h = 0;
      for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) {
        const int32_t u = g->adj[e];
        if (mate[u] >= 0) continue;
        const int64_t cu = vweight(g, u);
        if (cv + cu > U) continue;
        const int64_t w = eweight(g, e);
        const uint64_t h = or_hash3(seed, (uint64_t)(v < u ? v : u), (uint64_t)(v < u ? u : v));
        bool better;
        if (best < 0) {
          better = true;
        } else {
          // w^2 / cu against best_w^2 / best_c (c(v) is common)
          const u128 a = (u128)(uint64_t)w * (uint64_t)w * (uint64_t)best_c;
          const u128 b = (u128)(uint64_t)best_w * (uint64_t)best_w * (uint64_t)cu;
          if (a != b) better = a > b;
          else if (h != best_h) better = h > best_h;
          else better = u < best;
        }
        if (better) {
          best = u;
          best_w = w;
          best_c = cu;
          best_h = h;
        }
      }
      prop[v] = best;
    }
    int64_t pairs = 0;
    for (int64_t v = 0; v < n; v++) {
      const int32_t u = prop[v];
      if (u >= 0 && prop[u] == (int32_t)v) {
        mate[v] = u;
        if (v < u) pairs++;
      }
    }
    s.rounds = r + 1;
    s.pairs += pairs;
    if (pairs == 0) break;
  }
  for (int64_t v = 0; v < n; v++) labels[v] = mate[v] >= 0 && mate[v] < v ? mate[v] : (int32_t)v;
  if (st) *st = s;
  return 0;
}
