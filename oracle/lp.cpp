// lp.cpp -- oracle: hash and size-constrained label propagation.
//
// TEST INFRASTRUCTURE ONLY. This file is part of the CPU oracle that the tests, the smoke check and
// the benchmark's CPU-baseline leg use to check the GPU library. It shares no code with that library.
//
// Label propagation with a size constraint follows Section III-A ("Clustering"): a vertex moves to
// the eligible cluster of strongest connection, where a cluster is eligible if it does not exceed
// the bound U once the vertex joins; neighbours of moved vertices become active for the next
// iteration. Used as a local search (Section III-C, Section IV-C) it starts from a partition and
// uses U = Lmax. The deterministic readings (the paper randomises ties and visits vertices
// asynchronously, Section III and Section IV-A) are:
//   * each round has two Jacobi sub-rounds; vertex v takes part in sub-round bit(r,v) = H(s,r,v)>>63,
//     and all decisions of a sub-round read the labels and label weights of its start;
//   * the own label wins every tie, so a move needs a strictly positive gain;
//   * among other labels: larger connection, then (learned) larger sum of edge scores, then larger
//     H(s,v,L), then smaller L;
//   * movers to one target are admitted in (gain desc, [learned: score sum desc,] id asc) order while
//     the snapshot weight plus the admitted weight stays <= U (the CAS of Section IV-A made
//     deterministic); departures are not credited; a rejected mover stays;
//   * a vertex is active in round r+1 iff one of its neighbours moved in round r (round 0: all).
// Hash: SplitMix64's output function (Steele, Lea & Flood, OOPSLA 2014), H(a,b,c)=mix(mix(mix(a)^b)^c).
#include <algorithm>
#include <map>
#include <vector>

#include "oracle.h"

extern "C" uint64_t or_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

extern "C" uint64_t or_hash3(uint64_t a, uint64_t b, uint64_t c) {
  return or_mix64(or_mix64(or_mix64(a) ^ b) ^ c);
}

extern "C" int64_t or_lmax(int64_t total_weight, int64_t k, double eps) {
  // Section II-A: Lmax = (1+eps) * ceil(c(V)/k), rounded down to an integer weight.
  int64_t ceil_avg = (total_weight + k - 1) / k;
  return (int64_t)((1.0 + eps) * (double)ceil_avg);
}

namespace {

struct Mover {
  int32_t v;
  int32_t target;
  int64_t gain;
  int64_t qsum;
};

inline int64_t vweight(const or_graph *g, int64_t v) { return g->vw ? g->vw[v] : 1; }
inline int64_t eweight(const or_graph *g, int64_t e) { return g->ew ? g->ew[e] : 1; }

}  // namespace

extern "C" int or_lp(const or_graph *g, const int32_t *q, int32_t *labels, int64_t *lw, int64_t nl,
                     int64_t U, int64_t rounds, uint64_t seed, or_lp_stats *st) {
  const int64_t n = g->n;
  or_lp_stats stats = {0, 0, 0, 0, 0};
  std::vector<uint8_t> active(n, 1), next_active(n, 0);
  for (int64_t r = 0; r < rounds; r++) {
    int64_t moves_this_round = 0;
    std::fill(next_active.begin(), next_active.end(), 0);
    for (int s = 0; s < 2; s++) {
      // Snapshot at the start of the sub-round.
      std::vector<int32_t> snap(labels, labels + n);
      std::vector<int64_t> snap_w(lw, lw + nl);
      std::vector<Mover> movers;
      for (int64_t v = 0; v < n; v++) {
        if (r > 0 && !active[v]) continue;
        if ((int)(or_hash3(seed, (uint64_t)r, (uint64_t)v) >> 63) != s) continue;
        stats.visits++;
        stats.edges += g->off[v + 1] - g->off[v];
        // Connection strength omega({(v,u) : u in N(v) and C[u] = L}) per neighbouring label L.
        std::map<int32_t, std::pair<int64_t, int64_t>> conn;
        for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) {
          int32_t L = snap[g->adj[e]];
          conn[L].first += eweight(g, e);
          conn[L].second += q ? (int64_t)q[e] : 0;
        }
        const int32_t own = snap[v];
        const int64_t own_conn = conn.count(own) ? conn[own].first : 0;
        const int64_t cv = vweight(g, v);
        bool found = false;
        int32_t best = -1;
        int64_t best_conn = 0, best_q = 0;
        uint64_t best_h = 0;
        for (const auto &kv : conn) {
          const int32_t L = kv.first;
          const int64_t cw = kv.second.first, cq = kv.second.second;
          if (L == own) continue;
          if (cw <= own_conn) continue;          // the own label wins ties
          if (snap_w[L] + cv > U) continue;     // not eligible: L would exceed U
          const uint64_t h = or_hash3(seed, (uint64_t)v, (uint64_t)L);
          bool better;
          if (!found) better = true;
          else if (cw != best_conn) better = cw > best_conn;
          else if (cq != best_q) better = cq > best_q;
          else if (h != best_h) better = h > best_h;
          else better = L < best;
          if (better) {
            found = true;
            best = L;
            best_conn = cw;
            best_q = cq;
            best_h = h;
          }
        }
        if (found) movers.push_back({(int32_t)v, best, best_conn - own_conn, best_q});
      }
      stats.movers += (int64_t)movers.size();
      // Admission: per target, in (gain desc, qsum desc, id asc) order, the longest prefix that fits.
      std::sort(movers.begin(), movers.end(), [](const Mover &a, const Mover &b) {
        if (a.target != b.target) return a.target < b.target;
        if (a.gain != b.gain) return a.gain > b.gain;
        if (a.qsum != b.qsum) return a.qsum > b.qsum;
        return a.v < b.v;
      });
      std::vector<Mover> admitted;
      size_t i = 0;
      while (i < movers.size()) {
        size_t j = i;
        const int32_t T = movers[i].target;
        int64_t acc = 0;
        bool open = true;
        while (j < movers.size() && movers[j].target == T) {
          acc += vweight(g, movers[j].v);
          if (open && snap_w[T] + acc <= U) admitted.push_back(movers[j]);
          else open = false;
          j++;
        }
        i = j;
      }
      // Apply the admitted moves; neighbours of moved vertices become active next round.
      for (const Mover &m : admitted) {
        const int64_t cv = vweight(g, m.v);
        lw[labels[m.v]] -= cv;
        lw[m.target] += cv;
        labels[m.v] = m.target;
        for (int64_t e = g->off[m.v]; e < g->off[m.v + 1]; e++) next_active[g->adj[e]] = 1;
        moves_this_round++;
      }
    }
    stats.rounds = r + 1;
    stats.moves += moves_this_round;
    active.swap(next_active);
    if (moves_this_round == 0) break;
  }
  if (st) *st = stats;
  return 0;
}
