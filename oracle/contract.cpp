// contract.cpp -- oracle: contraction of a clustering into the weighted quotient graph.
//
// TEST INFRASTRUCTURE ONLY (CPU oracle; shares no code with the GPU library).
//
// Section III-A defines the coarse graph: one vertex per cluster whose weight is the cluster's
// weight, and an edge between two clusters whose weight is the total weight of the fine edges
// between them. Section IV-A ("Parallel Contraction") gives the three phases followed here:
//   1. remap cluster ids to [0, n') by a prefix sum over an array holding a one at every used id
//      (so the new id of a cluster is the rank of its label among the used labels);
//   2. accumulate the weight of every cut pair (C[v], C[u]), C[v] != C[u];
//   3. build the coarse CSR.
// Phase 2 here uses a counting sort of the vertices by coarse id and a dense marker array per coarse
// row instead of a hash table; rows are then sorted by neighbour id so the output is canonical.
#include <algorithm>
#include <vector>

#include "oracle.h"

extern "C" int or_contract(const or_graph *g, const int32_t *labels, int64_t nl, int64_t *n_out,
                           int64_t *m_out, int64_t *off_out, int32_t *adj_out, int64_t *vw_out,
                           int64_t *ew_out, int32_t *f2c) {
  const int64_t n = g->n;
  // Phase 1: ones at used ids, exclusive prefix sum -> new ids.
  std::vector<int64_t> used(nl, 0);
  for (int64_t v = 0; v < n; v++) {
    if (labels[v] < 0 || labels[v] >= nl) return -1;
    used[labels[v]] = 1;
  }
  std::vector<int64_t> new_id(nl, 0);
  int64_t n_coarse = 0;
  for (int64_t L = 0; L < nl; L++) {
    new_id[L] = n_coarse;
    n_coarse += used[L];
  }
  for (int64_t v = 0; v < n; v++) f2c[v] = (int32_t)new_id[labels[v]];
  // Coarse vertex weights.
  for (int64_t c = 0; c < n_coarse; c++) vw_out[c] = 0;
  for (int64_t v = 0; v < n; v++) vw_out[f2c[v]] += g->vw ? g->vw[v] : 1;
  // Members of each coarse vertex (counting sort by coarse id).
  std::vector<int64_t> start(n_coarse + 1, 0);
  for (int64_t v = 0; v < n; v++) start[f2c[v] + 1]++;
  for (int64_t c = 0; c < n_coarse; c++) start[c + 1] += start[c];
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  std::vector<int32_t> members(n);
  for (int64_t v = 0; v < n; v++) members[fill[f2c[v]]++] = (int32_t)v;
  // Phases 2 and 3: per coarse row, accumulate weights of cut pairs with a dense marker array.
  std::vector<int64_t> slot(n_coarse, -1);
  std::vector<std::pair<int32_t, int64_t>> row;
  int64_t m = 0;
  off_out[0] = 0;
  for (int64_t c = 0; c < n_coarse; c++) {
    row.clear();
    for (int64_t t = start[c]; t < start[c + 1]; t++) {
      const int32_t v = members[t];
      for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) {
        const int32_t cu = f2c[g->adj[e]];
        if (cu == c) continue;  // intra-cluster edge: not part of the quotient graph
        const int64_t w = g->ew ? g->ew[e] : 1;
        if (slot[cu] < 0) {
          slot[cu] = (int64_t)row.size();
          row.push_back({cu, w});
        } else {
          row[slot[cu]].second += w;
        }
      }
    }
    std::sort(row.begin(), row.end());
    for (const auto &p : row) {
      adj_out[m] = p.first;
      ew_out[m] = p.second;
      slot[p.first] = -1;
      m++;
    }
    off_out[c + 1] = m;
  }
  *n_out = n_coarse;
  *m_out = m;
  return 0;
}
