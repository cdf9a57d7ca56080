// mls.cpp -- oracle: multi-try k-way local search (MLS) after label-propagation refinement.
//
// TEST INFRASTRUCTURE ONLY (CPU oracle; shares no code with the GPU library).
//
// Section III-C describes MLS: instead of starting one k-way FM search from all boundary vertices,
// it repeatedly starts a localized search from a single boundary vertex taken from a todo list; the
// search puts the start vertex and its neighbours into a priority queue keyed by gain, moves the
// vertex of maximum gain, inserts unmarked neighbours of moved vertices and updates the keys of queued
// ones, respects the balance bound, stops by a stopping rule, and keeps the best prefix of its moves.
// A local iteration repeats this until the todo list is empty; moved vertices form the next todo list
// while the gain of a local iteration exceeds 10% of the gain of the global iteration so far; three
// global iterations start from all boundary vertices. Section IV-C parallelises it (Algorithm 1):
// searches (PerformMoves) run concurrently on the partition as it was at the start of the local
// iteration and only record their moves; ApplyMoves then applies the recorded sequences one after
// another, recomputing every gain on the current partition and applying only the best prefix.
//
// Readings of what the paper leaves open (the GPU path implements the same):
//   * todo lists are ordered by H(s, v, 1) ascending, then v (the paper shuffles randomly); global
//     iteration g uses s = H(seed, g, 5) for its first local iteration, and local iteration l + 1 uses
//     H(s_l, l + 1, 6) where s_l is the seed of local iteration l;
//   * all searches of a local iteration read the partition and block weights of its start; a search
//     starts at every todo vertex (no global "moved" bitmap during the searches: conflicts between
//     searches are resolved by ApplyMoves, which stops applying a sequence at the first move whose
//     vertex an earlier sequence of the same local iteration moved or whose source block changed);
//   * gain(w) in a search's view: the best target b != a = block(w) among blocks adjacent to w with
//     weight(b) + c(w) <= Lmax, by larger connection, then larger H(s, w, b), then smaller b;
//     gain = conn(w, b) - conn(w, a); w is movable iff such a b exists;
//   * queue order: larger gain, then larger H(s, w, 0), then smaller w; on extraction the gain and target
//     are recomputed in the current view (block weights may have changed) and the vertex is dropped if
//     it is no longer movable;
//   * the adaptive stopping rule of Osipov and Sanders is replaced by fixed bounds: a search stops after
//     `max_moves` moves or `fruitless` consecutive moves that do not improve its best prefix; the
//     queue holds at most `queue_cap` vertices (further insertions are skipped);
//   * "marked" is read as "queued or already moved by this search": when a vertex moves, each of its
//     neighbours that is queued gets its key recomputed (and leaves the queue if no longer movable),
//     and each one that is neither queued nor moved is inserted if movable (the start vertex and its
//     neighbours are inserted the same way, in row order);
//   * vertices of degree > `max_degree` are never queued or moved (hubs of power-law graphs would make
//     a single search cost the square of their degree);
//   * a search keeps its best prefix only when that prefix has positive gain;
//   * a local iteration continues to the next while 100 * gain > alpha_pct * (gain of the global
//     iteration so far), at most `max_local` local iterations.
#include <algorithm>
#include <cstring>
#include <map>
#include <set>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "oracle.h"

namespace {

inline int64_t vweight(const or_graph *g, int64_t v) { return g->vw ? g->vw[v] : 1; }
inline int64_t eweight(const or_graph *g, int64_t e) { return g->ew ? g->ew[e] : 1; }
inline int64_t degree(const or_graph *g, int64_t v) { return g->off[v + 1] - g->off[v]; }

struct Move {
  int32_t v, from, to;
};

// The block of every vertex as one search sees it: the snapshot plus the search's own moves.
struct View {
  const int32_t *part;
  std::unordered_map<int32_t, int32_t> changed;
  int32_t block(int32_t u) const {
    auto it = changed.find(u);
    return it == changed.end() ? part[u] : it->second;
  }
};

struct Choice {
  bool movable = false;
  int32_t to = -1;
  int64_t gain = 0;
};

template <class BlockOf>
Choice best_move(const or_graph *g, int32_t w, BlockOf block_of, const std::vector<int64_t> &bw, int64_t lmax,
                 uint64_t s) {
  std::map<int32_t, int64_t> conn;
  for (int64_t e = g->off[w]; e < g->off[w + 1]; e++) conn[block_of(g->adj[e])] += eweight(g, e);
  const int32_t a = block_of(w);
  const int64_t cw = vweight(g, w);
  const int64_t own = conn.count(a) ? conn[a] : 0;
  Choice c;
  int64_t best_conn = 0;
  uint64_t best_h = 0;
  for (const auto &kv : conn) {
    const int32_t b = kv.first;
    if (b == a || bw[b] + cw > lmax) continue;
    const uint64_t h = or_hash3(s, (uint64_t)w, (uint64_t)b);
    bool better;
    if (!c.movable) better = true;
    else if (kv.second != best_conn) better = kv.second > best_conn;
    else if (h != best_h) better = h > best_h;
    else better = b < c.to;
    if (better) {
      c.movable = true;
      c.to = b;
      best_conn = kv.second;
      best_h = h;
    }
  }
  if (c.movable) c.gain = best_conn - own;
  return c;
}

// Queue key: larger gain first, then larger H(s, w), then smaller w.
typedef std::tuple<int64_t, uint64_t, int32_t> Key;  // (-gain, ~h, w): std::set ascending
Key key_of(int64_t gain, uint64_t h, int32_t w) { return Key(-gain, ~h, w); }

std::vector<Move> perform_moves(const or_graph *g, int32_t v, const int32_t *part, const std::vector<int64_t> &bw0,
                                int64_t lmax, uint64_t s, const or_mls_params &p) {
  std::vector<Move> moves;
  if (degree(g, v) > p.max_degree || degree(g, v) == 0) return moves;
  View view;
  view.part = part;
  std::vector<int64_t> bw = bw0;
  auto block_of = [&](int32_t u) { return view.block(u); };
  std::set<Key> pq;
  std::unordered_map<int32_t, Key> queued;  // vertex -> its key while queued
  std::set<int32_t> done;                   // moved by this search
  auto try_insert = [&](int32_t x) {
    if (queued.count(x) || done.count(x) || degree(g, x) > p.max_degree) return;
    if ((int64_t)queued.size() >= p.queue_cap) return;
    const Choice c = best_move(g, x, block_of, bw, lmax, s);
    if (!c.movable) return;
    const Key k = key_of(c.gain, or_hash3(s, (uint64_t)x, 0), x);
    pq.insert(k);
    queued[x] = k;
  };
  try_insert(v);
  for (int64_t e = g->off[v]; e < g->off[v + 1]; e++) try_insert(g->adj[e]);
  int64_t cum = 0, best = 0, best_len = 0, fruitless = 0;
  while (!pq.empty() && (int64_t)moves.size() < p.max_moves) {
    const int32_t x = std::get<2>(*pq.begin());
    pq.erase(pq.begin());
    queued.erase(x);
    const Choice c = best_move(g, x, block_of, bw, lmax, s);
    if (!c.movable) continue;
    const int32_t a = view.block(x);
    const int64_t cx = vweight(g, x);
    view.changed[x] = c.to;
    bw[a] -= cx;
    bw[c.to] += cx;
    done.insert(x);
    moves.push_back({x, a, c.to});
    cum += c.gain;
    if (cum > best) {
      best = cum;
      best_len = (int64_t)moves.size();
      fruitless = 0;
    } else if (++fruitless >= p.fruitless) {
      break;
    }
    for (int64_t e = g->off[x]; e < g->off[x + 1]; e++) {
      const int32_t u = g->adj[e];
      if (done.count(u) || degree(g, u) > p.max_degree) continue;
      auto it = queued.find(u);
      if (it != queued.end()) {
        pq.erase(it->second);
        queued.erase(it);
        const Choice cu = best_move(g, u, block_of, bw, lmax, s);
        if (cu.movable) {
          const Key k = key_of(cu.gain, or_hash3(s, (uint64_t)u, 0), u);
          pq.insert(k);
          queued[u] = k;
        }
      } else {
        try_insert(u);
      }
    }
  }
  if (best <= 0) return {};
  moves.resize(best_len);
  return moves;
}

int64_t gain_now(const or_graph *g, const int32_t *part, int32_t w, int32_t from, int32_t to) {
  int64_t g_to = 0, g_from = 0;
  for (int64_t e = g->off[w]; e < g->off[w + 1]; e++) {
    const int32_t b = part[g->adj[e]];
    if (b == to) g_to += eweight(g, e);
    if (b == from) g_from += eweight(g, e);
  }
  return g_to - g_from;
}

// todo order: H(s, v) ascending, then v
void order_todo(std::vector<int32_t> &todo, uint64_t s) {
  std::sort(todo.begin(), todo.end(), [&](int32_t x, int32_t y) {
    const uint64_t hx = or_hash3(s, (uint64_t)x, 1), hy = or_hash3(s, (uint64_t)y, 1);
    return hx != hy ? hx < hy : x < y;
  });
}

}  // namespace

extern "C" void or_mls_default_params(or_mls_params *p) {
  p->global_iters = 3;
  p->alpha_pct = 10;
  p->max_local = 16;
  p->max_moves = 64;
  p->fruitless = 16;
  p->queue_cap = 256;
  p->max_degree = 1024;
}

extern "C" int64_t or_mls(const or_graph *g, int64_t k, int64_t lmax, uint64_t seed, const or_mls_params *pp,
                          int32_t *part, or_mls_stats *st) {
  or_mls_params p;
  if (pp) p = *pp;
  else or_mls_default_params(&p);
  const int64_t n = g->n;
  std::vector<int64_t> bw(k, 0);
  for (int64_t v = 0; v < n; v++) bw[part[v]] += vweight(g, v);
  or_mls_stats s = {0, 0, 0, 0};
  int64_t total_all = 0;
  for (int64_t gi = 0; gi < p.global_iters; gi++) {
    uint64_t sl = or_hash3(seed, (uint64_t)gi, 5);
    std::vector<int32_t> todo;
    for (int64_t v = 0; v < n; v++) {
      if (degree(g, v) > p.max_degree) continue;
      for (int64_t e = g->off[v]; e < g->off[v + 1]; e++)
        if (part[g->adj[e]] != part[v]) {
          todo.push_back((int32_t)v);
          break;
        }
    }
    order_todo(todo, sl);
    int64_t total = 0;
    for (int64_t li = 0; li < p.max_local && !todo.empty(); li++) {
      // PerformMoves: every search on the partition of the local iteration's start
      std::vector<std::vector<Move>> seqs(todo.size());
      for (size_t i = 0; i < todo.size(); i++) seqs[i] = perform_moves(g, todo[i], part, bw, lmax, sl, p);
      s.searches += (int64_t)todo.size();
      // ApplyMoves: in todo order, gains recomputed, best prefix applied
      std::vector<char> moved(n, 0);
      std::vector<int32_t> next;
      int64_t gain = 0;
      for (const auto &seq : seqs) {
        std::vector<Move> applied;
        int64_t cum = 0, best = 0, best_len = 0;
        for (const Move &m : seq) {
          if (moved[m.v] || part[m.v] != m.from) break;
          const int64_t cv = vweight(g, m.v);
          if (bw[m.to] + cv > lmax) break;
          cum += gain_now(g, part, m.v, m.from, m.to);
          part[m.v] = m.to;
          bw[m.from] -= cv;
          bw[m.to] += cv;
          applied.push_back(m);
          if (cum > best) {
            best = cum;
            best_len = (int64_t)applied.size();
          }
        }
        for (int64_t j = (int64_t)applied.size() - 1; j >= best_len; j--) {
          const Move &m = applied[j];
          const int64_t cv = vweight(g, m.v);
          part[m.v] = m.from;
          bw[m.to] -= cv;
          bw[m.from] += cv;
        }
        for (int64_t j = 0; j < best_len; j++) {
          moved[applied[j].v] = 1;
          next.push_back(applied[j].v);
        }
        gain += best;
        s.moves += best_len;
      }
      s.local_iters++;
      if (!(gain > 0 && 100 * gain > p.alpha_pct * total)) {
        total += gain;
        break;
      }
      total += gain;
      todo.swap(next);
      sl = or_hash3(sl, (uint64_t)li + 1, 6);  // the next local iteration's seed
      order_todo(todo, sl);
    }
    total_all += total;
  }
  s.gain = total_all;
  if (st) *st = s;
  return total_all;
}
