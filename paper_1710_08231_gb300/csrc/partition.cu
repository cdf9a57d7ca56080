// partition.cu -- multilevel driver and the C ABI of the partitioner library.
//
// Multilevel scheme (Section I, Section III): coarsen by LP clustering + contraction until the
// graph is small (Section III-A, IV-A), partition the coarsest graph several times and keep the best
// (Section III-B, IV-B), then project and refine with LP under U = Lmax level by level
// (Section III-C, IV-C). Parameters: 10 coarsening and 25 refinement LP rounds, 4 tries
// (Section VI "Algorithm Configuration"); Lmax = (1+eps) ceil(c(V)/k) (Section II-A).
// Per-phase seeds: coarsening LP at level l uses H(seed, l, 1); refinement at level l uses
// H(seed, l, 2); try t on the coarsest level c uses s_try = H(seed, c, 4 + t) and refines with
// H(s_try, c, 3).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "contract.cuh"
#include "gp_internal.cuh"
#include "ip.cuh"
#include "lp.cuh"
#include "lp_async.cuh"
#include "match.cuh"
#include "mls.cuh"
#include "mlp.cuh"

namespace gp {
void set_allocator(gp_alloc_fn a, gp_free_fn f, void *ctx);
const char *last_error();
int prof_enable(int on);
int prof_read(gp_profile_entry *out, int max_entries, int reset);
long long launch_count(int reset);

namespace {

int64_t lmax_of(int64_t total, int64_t k, double eps) {
  const int64_t ceil_avg = (total + k - 1) / k;
  return (int64_t)((1.0 + eps) * (double)ceil_avg);
}

__global__ void k_iota(int32_t *x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (int32_t)i;
}

__global__ void k_vw_to_i64(DGraph g, int64_t *out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = g.vweight(v);
}

// CSR validation; err bits: 1 offsets, 2 range, 4 self-loop, 8 order/duplicate, 16 weight <= 0,
// 32 missing reverse entry, 64 asymmetric weight.
__global__ void k_validate(DGraph g, int *err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = g.row_begin(v), e = g.row_begin(v + 1);
    if (e < b || b < 0 || e > g.m) {
      atomicOr(err, 1);
      continue;
    }
    if (g.vw && g.vweight(v) <= 0) atomicOr(err, 16);
    for (int64_t j = b; j < e; j++) {
      const int u = g.adj[j];
      if (u < 0 || u >= g.n) {
        atomicOr(err, 2);
        continue;
      }
      if (u == v) atomicOr(err, 4);
      if (j > b && g.adj[j - 1] >= u) atomicOr(err, 8);
      const int64_t w = g.eweight(j);
      if (w <= 0) atomicOr(err, 16);
      int64_t lo = g.row_begin(u), hi = g.row_begin(u + 1);
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (g.adj[mid] < v) lo = mid + 1;
        else hi = mid;
      }
      if (lo >= g.row_begin(u + 1) || g.adj[lo] != v) atomicOr(err, 32);
      else if (g.eweight(lo) != w) atomicOr(err, 64);
    }
  }
}

// Doubled cut of every try partition (parts: tries * n): cut2[t] += weight of each entry whose ends
// lie in different blocks of try t.
__global__ void k_tries_cut(DGraph g, const int32_t *parts, int tries, unsigned long long *cut2) {
  for (int t = 0; t < tries; t++) {
    const int32_t *p = parts + (size_t)t * g.n;
    unsigned long long c = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
      const int pv = p[v];
      for (int64_t j = g.row_begin(v); j < g.row_begin(v + 1); j++)
        if (p[g.adj[j]] != pv) c += (unsigned long long)g.eweight(j);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cut2[t], c);
  }
}

gp_params g_schedule = {};
int g_keep_pct = 0;  // stale threshold of kept hub tables (0: default)

LpConfig schedule_for(const gp_params *p) {
  gp_params q = g_schedule;
  if (p && p->deg_warp > 0) q.deg_warp = p->deg_warp;
  if (p && p->deg_cta > 0) q.deg_cta = p->deg_cta;
  if (p && p->hub_batch_slots > 0) q.hub_batch_slots = p->hub_batch_slots;
  if (p && p->verts_per_block > 0) q.verts_per_block = p->verts_per_block;
  if (p && p->hub_keep_slots != 0) q.hub_keep_slots = p->hub_keep_slots;
  LpConfig c = lp_config_from(&q);
  if (g_keep_pct > 0) c.hub_keep_pct = std::max(1, std::min(g_keep_pct, 95));
  return c;
}

int grid_n(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, num_sms() * 8)); }

int check_graph_desc(const gp_graph *g) {
  if (!g || g->n < 0 || g->m_dir < 0 || (g->n > 0 && (!g->offsets || (g->m_dir > 0 && !g->adj)))) {
    set_error("graph descriptor is NULL or incomplete");
    return GP_ERR_INVALID_ARG;
  }
  if (g->n >= ((int64_t)1 << 31) - 1) {
    set_error("graphs must have n < 2^31 - 1");
    return GP_ERR_UNSUPPORTED;
  }
  return GP_OK;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Level {
  OwnedGraph g;
  int32_t *f2c = nullptr;  // fine (previous level) -> this level
  size_t f2c_bytes = 0;
};

struct Hierarchy {
  cudaStream_t s;
  std::vector<Level> levels;  // levels[0] unused graph slot (level 0 is the stripped input)
  ~Hierarchy() {
    for (auto &l : levels) {
      l.g.release(s);
      dev_free(l.f2c, l.f2c_bytes, s);
    }
  }
};

}  // namespace

LpConfig schedule_for_batch(const gp_params *p) { return schedule_for(p); }

// ------------------------------------------------------------------------------------------ driver
int partition_device(const gp_graph *gin, int32_t k, double eps, uint64_t seed, const gp_params *pp,
                     int32_t *part_out, gp_result *res, cudaStream_t s) {
  const double t0 = now_ms();
  GP_TRY(check_graph_desc(gin));
  if (!res || !part_out) {
    set_error("gp_partition needs part_out and res");
    return GP_ERR_INVALID_ARG;
  }
  gp_params p;
  if (pp) p = *pp;
  else gp_default_params(&p);
  if (k < 1 || k > gin->n || !(eps >= 0.0) || p.ip_tries < 1 || p.ip_tries > 16 || p.cluster_div < 1 ||
      p.rounds_coarsen < 0 || p.rounds_refine < 0 || p.max_levels < 0 || p.max_levels > 64) {
    set_error("gp_partition: k, eps or params out of range");
    return GP_ERR_INVALID_ARG;
  }
  const bool learned = p.mode == GP_MODE_LEARNED;
  if (p.lp_async && p.mode != GP_MODE_PLAIN) {
    set_error("gp_partition: asynchronous LP needs plain mode");
    return GP_ERR_INVALID_ARG;
  }
  if (p.mls_global_iters < 0 || (p.mls_global_iters > 0 && (p.mode != GP_MODE_PLAIN || k > 256))) {
    set_error("gp_partition: multi-try local search needs plain mode and k <= 256");
    return GP_ERR_INVALID_ARG;
  }
  if (p.coarsen != GP_COARSEN_LP && (p.coarsen != GP_COARSEN_MATCHING || p.mode != GP_MODE_PLAIN)) {
    set_error("gp_partition: coarsen must be GP_COARSEN_LP, or GP_COARSEN_MATCHING in plain mode");
    return GP_ERR_INVALID_ARG;
  }
  if ((p.mode == GP_MODE_LEARNED || p.mode == GP_MODE_BEST_OF) && !p.mlp) {
    set_error("learned modes need params.mlp");
    return GP_ERR_INVALID_ARG;
  }
  if (p.mode == GP_MODE_BEST_OF) {
    gp_params q = p;
    q.mode = GP_MODE_PLAIN;
    Workspace ws(s);
    int32_t *alt;
    GP_TRY(ws.get(&alt, (size_t)gin->n));
    gp_result r_plain, r_learned;
    GP_TRY(partition_device(gin, k, eps, seed, &q, part_out, &r_plain, s));
    q.mode = GP_MODE_LEARNED;
    GP_TRY(partition_device(gin, k, eps, seed, &q, alt, &r_learned, s));
    // keep the lower cut; ties and imbalanced learned results keep the plain partition
    const bool use_learned = r_learned.imbalanced <= r_plain.imbalanced && r_learned.cut < r_plain.cut;
    *res = use_learned ? r_learned : r_plain;
    if (use_learned)
      GP_CUDA(cudaMemcpyAsync(part_out, alt, sizeof(int32_t) * (size_t)gin->n, cudaMemcpyDeviceToDevice, s));
    res->plain_cut = r_plain.cut;
    res->learned_cut = r_learned.cut;
    res->lp_edges = r_plain.lp_edges + r_learned.lp_edges;
    res->ms_total = now_ms() - t0;
    GP_CUDA(cudaStreamSynchronize(s));
    return GP_OK;
  }
  std::memset(res, 0, sizeof(*res));
  const LpConfig cfg = schedule_for(&p);
  const DGraph g = make_dgraph(gin);
  Workspace ws(s);
  // degree-0 vertices are set aside; the same read back gives the total weight and the largest weight
  // of a kept vertex (the level-0 graph's max c(v))
  int64_t W = 0, maxc0 = 0;
  Stripped st;
  std::vector<LpClassInfo> level_cls((size_t)p.max_levels + 1);
  GP_TRY(strip_isolated(g, &st, ws, s, &W, &maxc0, &cfg, &level_cls[0]));
  const int64_t lmax = lmax_of(W, k, eps);
  res->lmax = lmax;
  res->n_isolated = st.n_iso;
  Hierarchy H;
  H.s = s;
  std::vector<DGraph> G{st.g0};
  std::vector<const int32_t *> f2c;
  int32_t *cur = nullptr;  // partition of the current level (device, from ws)
  int64_t lp_edges = 0, lp_moves = 0;
  // LP counters stay on the device until the end (one read back for the whole partition), and each
  // level's degree classes computed by its coarsening call are reused by its refinement call
  LpDeferred lpdef;
  lpdef.capacity = 2 * (int)p.max_levels + (int)p.ip_tries + 4;
  {
    unsigned char *buf;
    GP_TRY(ws.get(&buf, lp_counters_bytes() * (size_t)lpdef.capacity));
    lpdef.dev = buf;
  }
  const double t_coarse0 = now_ms();
  if (st.n0 > 0) {
    const int64_t T = std::max<int64_t>(p.coarse_min, p.coarse_per_k * (int64_t)k);
    int32_t *labels;
    int64_t *lw;
    GP_TRY(ws.get(&labels, (size_t)st.n0));
    GP_TRY(ws.get(&lw, (size_t)st.n0));
    int32_t *q = nullptr;
    if (learned) GP_TRY(ws.get(&q, (size_t)std::max<int64_t>(st.g0.m, 1)));
    while (G.back().n > T && (int64_t)f2c.size() < p.max_levels) {
      const int l = (int)f2c.size();
      const DGraph &gl = G.back();
      // (level 0: from the strip's read back; later levels: reported by the contraction)
      const int64_t maxc = l == 0 ? maxc0 : H.levels.back().g.max_vw;
      const int64_t U = std::max<int64_t>(maxc, lmax / p.cluster_div);
      (::gp::count_launch(), k_iota<<<grid_n(gl.n), 256, 0, s>>>(labels, gl.n));
      (::gp::count_launch(), k_vw_to_i64<<<grid_n(gl.n), 256, 0, s>>>(gl, lw));
      GP_LAUNCH_CHECK();
      if (learned) GP_TRY(mlp_score(gl, l, static_cast<const gp_mlp *>(p.mlp), nullptr, q, s));
      if (p.coarsen == GP_COARSEN_MATCHING)
        GP_TRY(run_match(gl, U, (int)p.rounds_coarsen, hash3(seed, (uint64_t)l, 1), labels, nullptr, s, false));
      else if (p.lp_async)
        GP_TRY(run_lp_async(gl, labels, lw, gl.n, U, (int)p.rounds_coarsen, hash3(seed, (uint64_t)l, 1), false,
                            nullptr, s));
      else
        GP_TRY(run_lp(gl, learned ? q : nullptr, labels, lw, gl.n, U, (int)p.rounds_coarsen,
                      hash3(seed, (uint64_t)l, 1), nullptr, s, cfg, true, &level_cls[l], &lpdef,
                      l == 0 ? "lp_persistent_level0" : "lp_persistent"));
      Level lev;
      lev.f2c_bytes = sizeof(int32_t) * (size_t)gl.n;
      lev.f2c = (int32_t *)dev_alloc(lev.f2c_bytes, s);
      if (!lev.f2c) {
        set_error("allocation of a level map failed");
        return GP_ERR_OOM;
      }
      H.levels.push_back(lev);
      GP_TRY(contract_graph(gl, labels, gl.n, &H.levels.back().g, H.levels.back().f2c, s, &cfg, &level_cls[l + 1]));
      const int64_t n_before = gl.n;
      G.push_back(H.levels.back().g.view());
      f2c.push_back(H.levels.back().f2c);
      if (100 * G.back().n > p.stall_pct * n_before) break;
    }
    const int levels = (int)f2c.size();
    res->levels = levels;
    const double t_ip0 = now_ms();
    res->ms_coarsen = t_ip0 - t_coarse0;
    // initial partitioning: tries in parallel, then LP refinement and evaluation of each
    const DGraph &gc = G.back();
    const int tries = (int)p.ip_tries;
    int32_t *parts;
    int64_t *bw;
    GP_TRY(ws.get(&parts, (size_t)tries * (size_t)gc.n));
    GP_TRY(ws.get(&bw, (size_t)k));
    int *ip_err;  // read back with the tries' cuts
    GP_TRY(ws.zeros(&ip_err, 1));
    GP_TRY(initial_partition(gc, k, lmax, seed, levels, tries, (int)p.repair_rounds, parts, s, ip_err));
    int best = -1;
    int64_t best_cut = 0, best_imb = 0;
    // the tries' LP refinements run as independent problems of one launch
    int64_t *bws;
    GP_TRY(ws.get(&bws, (size_t)tries * k));
    std::vector<LpJob> jobs(tries);

    for (int t = 0; t < tries; t++) {
      int32_t *pt = parts + (size_t)t * gc.n;
      const uint64_t s_try = hash3(seed, (uint64_t)levels, (uint64_t)(4 + t));
      GP_TRY(block_weights(gc, pt, k, bws + (size_t)t * k, nullptr, s));
      jobs[t].g = gc;
      jobs[t].labels = pt;
      jobs[t].lw = bws + (size_t)t * k;
      jobs[t].nl = k;
      jobs[t].U = lmax;
      jobs[t].rounds = (int)p.rounds_refine;
      jobs[t].seed = hash3(s_try, (uint64_t)levels, 3);
      // degree classes of the coarsest graph from the contraction that built it (if any)
      jobs[t].classes = level_cls[levels].valid ? &level_cls[levels] : nullptr;
      jobs[t].prof = "lp_persistent_ip";
    }
    if (gc.n > 0 && p.rounds_refine > 0 && p.lp_async) {
      for (int t = 0; t < tries; t++)
        GP_TRY(run_lp_async(gc, jobs[t].labels, jobs[t].lw, k, lmax, (int)p.rounds_refine, jobs[t].seed, false,
                            nullptr, s));
    } else if (gc.n > 0 && p.rounds_refine > 0) {
      GP_TRY(run_lp_multi(jobs.data(), tries, s, cfg, &lpdef));
    }
    // cuts of all tries in one pass; their block weights are the label weights the refinement kept
    std::vector<unsigned long long> hcut2(tries);
    std::vector<int64_t> hbws((size_t)tries * k);
    {
      unsigned long long *cut2;
      GP_TRY(ws.zeros(&cut2, (size_t)tries));
      if (gc.n > 0) {
        (::gp::count_launch(), k_tries_cut<<<grid_n(gc.n), 256, 0, s>>>(gc, parts, tries, cut2));
        GP_LAUNCH_CHECK();
      }
      int herr = 0;
      Readback rb;
      rb.add(hcut2.data(), cut2, sizeof(unsigned long long) * tries);
      rb.add(hbws.data(), bws, sizeof(int64_t) * (size_t)tries * k);
      rb.add(&herr, ip_err, sizeof(int));
      GP_TRY(rb.run(s));
      if (herr) {
        set_error("initial partitioning: gain range too wide for the repair sort keys");
        return herr;
      }
    }
    for (int t = 0; t < tries; t++) {
      const int64_t cut = (int64_t)(hcut2[t] / 2);
      const int64_t imb =
          *std::max_element(hbws.begin() + (size_t)t * k, hbws.begin() + (size_t)(t + 1) * k) > lmax ? 1 : 0;
      res->try_cut[t] = cut;
      res->try_imbalanced[t] = imb;
      if (best < 0 || cut < best_cut || (cut == best_cut && imb < best_imb)) {
        best = t;
        best_cut = cut;
        best_imb = imb;
      }
    }
    res->best_try = best;
    cur = parts + (size_t)best * gc.n;
    const double t_ref0 = now_ms();
    res->ms_initial = t_ref0 - t_ip0;
    // uncoarsening
    int32_t *bufA, *bufB;
    GP_TRY(ws.get(&bufA, (size_t)st.n0));
    GP_TRY(ws.get(&bufB, (size_t)st.n0));
    // projection keeps every block's weight (a coarse vertex weighs what its members weigh), so the
    // block weights an LP refinement ends with are those the next finer level starts with
    GP_CUDA(cudaMemcpyAsync(bw, bws + (size_t)best * k, sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToDevice, s));
    MlsParams mp;
    mls_default_params(&mp);
    mp.global_iters = p.mls_global_iters;
    if (mp.global_iters > 0) {
      GP_TRY(run_mls(gc, k, lmax, hash3(seed, (uint64_t)levels, 7), mp, cur, nullptr, s));
      GP_TRY(block_weights(gc, cur, k, bw, nullptr, s));
    }
    for (int l = levels - 1; l >= 0; l--) {
      int32_t *fine = (cur == bufA) ? bufB : bufA;
      GP_TRY(project(cur, f2c[l], G[l].n, fine, s));
      if (p.lp_async)
        GP_TRY(run_lp_async(G[l], fine, bw, k, lmax, (int)p.rounds_refine, hash3(seed, (uint64_t)l, 2), false, nullptr, s));
      else
        GP_TRY(run_lp(G[l], nullptr, fine, bw, k, lmax, (int)p.rounds_refine, hash3(seed, (uint64_t)l, 2), nullptr, s,
                      cfg, false, &level_cls[l], &lpdef, "lp_persistent_refine"));
      if (mp.global_iters > 0) {
        GP_TRY(run_mls(G[l], k, lmax, hash3(seed, (uint64_t)l, 7), mp, fine, nullptr, s));
        GP_TRY(block_weights(G[l], fine, k, bw, nullptr, s));
      }
      cur = fine;
    }
    res->ms_refine = now_ms() - t_ref0;
  }
  for (size_t l = 0; l < G.size() && l < 65; l++) {
    res->level_n[l] = G[l].n;
    res->level_m[l] = G[l].m;
  }
  // degree-0 vertices, final evaluation on the input graph
  int32_t *empty = nullptr;
  if (!cur) {
    GP_TRY(ws.get(&empty, 1));
    cur = empty;
  }
  GP_TRY(place_isolated(g, st, cur, k, part_out, s));
  int64_t *bw_final;
  GP_TRY(ws.get(&bw_final, (size_t)k));
  // cut, block weights and the LP counters of the whole partition in one read back
  unsigned long long *cut_acc;
  GP_TRY(ws.get(&cut_acc, 1));
  GP_TRY(eval_cut_launch(g, part_out, k, cut_acc, bw_final, s));
  unsigned long long cut2 = 0;
  std::vector<int64_t> hbw(k);
  Readback rb;
  rb.add(&cut2, cut_acc, sizeof(cut2));
  rb.add(hbw.data(), bw_final, sizeof(int64_t) * k);
  GP_TRY(lp_collect(lpdef, s, &lp_edges, &lp_moves, &rb));
  const int64_t cut = (int64_t)(cut2 / 2);
  res->cut = cut;
  res->max_block_weight = *std::max_element(hbw.begin(), hbw.end());
  res->imbalanced = res->max_block_weight > lmax ? 1 : 0;
  res->lp_edges = lp_edges;
  res->lp_moves = lp_moves;
  if (learned) res->learned_cut = cut;
  else res->plain_cut = cut;
  GP_TRY(prof_flush(s));
  res->ms_total = now_ms() - t0;
  return GP_OK;
}

}  // namespace gp

struct gp_coarse {
  gp::OwnedGraph g;
  gp_graph desc;
  cudaStream_t s;
};

using namespace gp;

extern "C" {

const char *gp_version(void) { return "gpart 0.1.0 (sm_103a)"; }

const char *gp_status_string(int st) {
  switch (st) {
    case GP_OK: return "ok";
    case GP_ERR_INVALID_ARG: return "invalid argument";
    case GP_ERR_BAD_GRAPH: return "malformed graph";
    case GP_ERR_OOM: return "out of device memory";
    case GP_ERR_CUDA: return "CUDA error";
    case GP_ERR_TIMEOUT: return "device wait timed out";
    case GP_ERR_INTERNAL: return "internal invariant violated";
    case GP_ERR_UNSUPPORTED: return "unsupported size";
    default: return "unknown status";
  }
}

const char *gp_last_error(void) { return gp::last_error(); }

int gp_set_allocator(gp_alloc_fn alloc, gp_free_fn release, void *ctx) {
  gp::set_allocator(alloc, release, ctx);
  return GP_OK;
}

void gp_default_params(gp_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->cluster_div = 14;
  p->rounds_coarsen = 10;
  p->rounds_refine = 25;
  p->coarse_min = 2000;
  p->coarse_per_k = 64;
  p->stall_pct = 95;
  p->max_levels = 64;
  p->ip_tries = 4;
  p->repair_rounds = 16;
  p->mode = GP_MODE_PLAIN;
}

int64_t gp_lmax(int64_t total_weight, int64_t k, double eps) {
  if (k < 1) return -1;
  return lmax_of(total_weight, k, eps);
}

int gp_validate_graph(const gp_graph *gd, gp_stream stream) {
  GP_TRY(check_graph_desc(gd));
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws(s);
  int *err;
  GP_TRY(ws.zeros(&err, 1));
  const DGraph g = make_dgraph(gd);
  if (g.n > 0) {
    (::gp::count_launch(), k_validate<<<grid_n(g.n), 256, 0, s>>>(g, err));
    GP_LAUNCH_CHECK();
  }
  int h = 0;
  int64_t first = 0, last = 0;
  GP_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (g.n >= 0) {
    if (g.off64) {
      GP_CUDA(cudaMemcpyAsync(&first, g.off, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaMemcpyAsync(&last, (const int64_t *)g.off + g.n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    } else {
      int32_t a = 0, b = 0;
      GP_CUDA(cudaMemcpyAsync(&a, g.off, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaMemcpyAsync(&b, (const int32_t *)g.off + g.n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      GP_CUDA(cudaStreamSynchronize(s));
      first = a;
      last = b;
    }
  }
  GP_CUDA(cudaStreamSynchronize(s));
  if (h || first != 0 || last != g.m) {
    set_error("graph check failed (code " + std::to_string(h) + ")");
    return GP_ERR_BAD_GRAPH;
  }
  return GP_OK;
}

int gp_lp_cluster(const gp_graph *gd, int64_t U, int32_t rounds, uint64_t seed, const int32_t *edge_q,
                  int32_t *labels_out, gp_lp_stats *stats, gp_stream stream) {
  GP_TRY(check_graph_desc(gd));
  if ((!labels_out && gd->n > 0) || rounds < 0 || U < 1) {
    set_error("gp_lp_cluster: labels_out, rounds or U out of range");
    return GP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DGraph g = make_dgraph(gd);
  Workspace ws(s);
  int64_t maxc = 0;
  GP_TRY(vertex_weight_stats(g, &maxc, nullptr, s));
  if (maxc > U) {
    set_error("gp_lp_cluster: U is below the largest vertex weight");
    return GP_ERR_INVALID_ARG;
  }
  int64_t *lw;
  GP_TRY(ws.get(&lw, (size_t)std::max<int64_t>(g.n, 1)));
  if (g.n > 0) {
    (::gp::count_launch(), k_iota<<<grid_n(g.n), 256, 0, s>>>(labels_out, g.n));
    (::gp::count_launch(), k_vw_to_i64<<<grid_n(g.n), 256, 0, s>>>(g, lw));
    GP_LAUNCH_CHECK();
  }
  GP_TRY(run_lp(g, edge_q, labels_out, lw, g.n, U, rounds, seed, stats, s, schedule_for(nullptr), true));
  GP_TRY(prof_flush(s));
  GP_CUDA(cudaStreamSynchronize(s));
  return GP_OK;
}

int gp_lp_cluster_async(const gp_graph *gd, int64_t U, int32_t rounds, uint64_t seed, int32_t single_warp,
                        int32_t *labels_out, gp_lp_stats *stats, gp_stream stream) {
  GP_TRY(check_graph_desc(gd));
  if ((!labels_out && gd->n > 0) || rounds < 0 || U < 1) {
    set_error("gp_lp_cluster_async: labels_out, rounds or U out of range");
    return GP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DGraph g = make_dgraph(gd);
  Workspace ws(s);
  int64_t maxc = 0;
  GP_TRY(vertex_weight_stats(g, &maxc, nullptr, s));
  if (maxc > U) {
    set_error("gp_lp_cluster_async: U is below the largest vertex weight");
    return GP_ERR_INVALID_ARG;
  }
  int64_t *lw;
  GP_TRY(ws.get(&lw, (size_t)std::max<int64_t>(g.n, 1)));
  if (g.n > 0) {
    (::gp::count_launch(), k_iota<<<grid_n(g.n), 256, 0, s>>>(labels_out, g.n));
    (::gp::count_launch(), k_vw_to_i64<<<grid_n(g.n), 256, 0, s>>>(g, lw));
    GP_LAUNCH_CHECK();
  }
  GP_TRY(run_lp_async(g, labels_out, lw, g.n, U, rounds, seed, single_warp != 0, stats, s));
  GP_CUDA(cudaStreamSynchronize(s));
  return GP_OK;
}

int gp_match(const gp_graph *gd, int64_t U, int32_t rounds, uint64_t seed, int32_t *labels_out,
             gp_match_stats *stats, gp_stream stream) {
  GP_TRY(check_graph_desc(gd));
  if ((!labels_out && gd->n > 0) || rounds < 0 || U < 1) {
    set_error("gp_match: labels_out, rounds or U out of range");
    return GP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DGraph g = make_dgraph(gd);
  MatchStats m;
  GP_TRY(run_match(g, U, rounds, seed, labels_out, &m, s, stats != nullptr));
  if (stats) {
    stats->rounds = m.rounds;
    stats->pairs = m.pairs;
    stats->visits = m.visits;
    stats->edges = m.edges;
  }
  GP_CUDA(cudaStreamSynchronize(s));
  return GP_OK;
}

void gp_mls_default_params(gp_mls_params *q) {
  if (!q) return;
  MlsParams m;
  mls_default_params(&m);
  q->global_iters = m.global_iters;
  q->alpha_pct = m.alpha_pct;
  q->max_local = m.max_local;
  q->max_moves = m.max_moves;
  q->fruitless = m.fruitless;
  q->queue_cap = m.queue_cap;
  q->max_degree = m.max_degree;
}

int gp_mls(const gp_graph *gd, int32_t k, int64_t lmax, uint64_t seed, const gp_mls_params *params, int32_t *part,
           gp_mls_stats *stats, gp_stream stream) {
  GP_TRY(check_graph_desc(gd));
  if ((!part && gd->n > 0) || k < 1 || lmax < 0) {
    set_error("gp_mls: part, k or lmax out of range");
    return GP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DGraph g = make_dgraph(gd);
  {
    Workspace ws(s);
    int64_t *bw;
    int *bad;
    GP_TRY(ws.get(&bw, (size_t)k));
    GP_TRY(ws.zeros(&bad, 1));
    GP_TRY(block_weights(g, part, k, bw, bad, s));
    int hbad = 0;
    GP_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
      set_error("gp_mls: a block id is outside [0, k)");
      return GP_ERR_INVALID_ARG;
    }
  }
  MlsParams mp;
  mls_default_params(&mp);
  if (params) {
    mp.global_iters = params->global_iters;
    mp.alpha_pct = params->alpha_pct;
    mp.max_local = params->max_local;
    mp.max_moves = params->max_moves;
    mp.fruitless = params->fruitless;
    mp.queue_cap = params->queue_cap;
    mp.max_degree = params->max_degree;
  }
  MlsStats m;
  GP_TRY(run_mls(g, k, lmax, seed, mp, part, &m, s));
  if (stats) {
    stats->gain = m.gain;
    stats->moves = m.moves;
    stats->searches = m.searches;
    stats->local_iters = m.local_iters;
  }
  GP_CUDA(cudaStreamSynchronize(s));
  return GP_OK;
}

int gp_lp_refine(const gp_graph *gd, int32_t k, int64_t lmax, int32_t rounds, uint64_t seed, int32_t *part,
                 int64_t *block_w_out, gp_lp_stats *stats, gp_stream stream) {
  GP_TRY(check_graph_desc(gd));
  if ((!part && gd->n > 0) || k < 1 || rounds < 0 || lmax < 0) {
    set_error("gp_lp_refine: part, k, rounds or lmax out of range");
    return GP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DGraph g = make_dgraph(gd);
  Workspace ws(s);
  int64_t *bw;
  int *bad;
  GP_TRY(ws.get(&bw, (size_t)k));
  GP_TRY(ws.zeros(&bad, 1));
  GP_TRY(block_weights(g, part, k, bw, bad, s));
  int hbad = 0;
  GP_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  if (hbad) {
    set_error("gp_lp_refine: a block id is outside [0, k)");
    return GP_ERR_INVALID_ARG;
  }
  GP_TRY(run_lp(g, nullptr, part, bw, k, lmax, rounds, seed, stats, s, schedule_for(nullptr)));
  if (block_w_out) GP_CUDA(cudaMemcpyAsync(block_w_out, bw, sizeof(int64_t) * k, cudaMemcpyDeviceToDevice, s));
  GP_TRY(prof_flush(s));
  GP_CUDA(cudaStreamSynchronize(s));
  return GP_OK;
}

int gp_contract(const gp_graph *gd, const int32_t *labels, gp_coarse **coarse, int32_t *f2c_out, gp_stream stream) {
  GP_TRY(check_graph_desc(gd));
  if ((!labels && gd->n > 0) || !coarse) {
    set_error("gp_contract: labels (unless n = 0) and coarse are required");
    return GP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  gp_coarse *c = new gp_coarse();
  c->s = s;
  const int st = contract_graph(make_dgraph(gd), labels, gd->n, &c->g, f2c_out, s);
  if (st != GP_OK) {
    delete c;
    return st;
  }
  c->desc.n = c->g.n;
  c->desc.m_dir = c->g.m;
  c->desc.offsets = c->g.off;
  c->desc.adj = c->g.adj;
  c->desc.vwgt = c->g.vw;
  c->desc.ewgt = c->g.ew;
  c->desc.offsets_64 = 1;
  c->desc.vwgt_64 = 1;
  c->desc.ewgt_64 = 1;
  c->desc.reserved = 0;
  GP_TRY(prof_flush(s));
  *coarse = c;
  return GP_OK;
}

const gp_graph *gp_coarse_graph(const gp_coarse *c) { return c ? &c->desc : nullptr; }

void gp_coarse_free(gp_coarse *c, gp_stream stream) {
  if (!c) return;
  c->g.release((cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  delete c;
}

int gp_partition(const gp_graph *g, int32_t k, double eps, uint64_t seed, const gp_params *params, int32_t *part_out,
                 gp_result *res, gp_stream stream) {
  const int st = partition_device(g, k, eps, seed, params, part_out, res, (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  return st;
}

int gp_partition_host(const gp_graph *hg, int32_t k, double eps, uint64_t seed, const gp_params *params,
                      int32_t *part_out_host, gp_result *res, gp_stream stream) {
  GP_TRY(check_graph_desc(hg));
  if (!part_out_host) {
    set_error("gp_partition_host: part_out_host is required");
    return GP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws(s);
  const size_t ob = hg->offsets_64 ? 8 : 4, vb = hg->vwgt_64 ? 8 : 4, eb = hg->ewgt_64 ? 8 : 4;
  unsigned char *off, *vw = nullptr, *ew = nullptr;
  int32_t *adj, *part;
  GP_TRY(ws.get(&off, ob * (size_t)(hg->n + 1)));
  GP_TRY(ws.get(&adj, (size_t)std::max<int64_t>(hg->m_dir, 1)));
  GP_TRY(ws.get(&part, (size_t)std::max<int64_t>(hg->n, 1)));
  GP_CUDA(cudaMemcpyAsync(off, hg->offsets, ob * (size_t)(hg->n + 1), cudaMemcpyHostToDevice, s));
  if (hg->m_dir) GP_CUDA(cudaMemcpyAsync(adj, hg->adj, sizeof(int32_t) * (size_t)hg->m_dir, cudaMemcpyHostToDevice, s));
  if (hg->vwgt) {
    GP_TRY(ws.get(&vw, vb * (size_t)hg->n));
    GP_CUDA(cudaMemcpyAsync(vw, hg->vwgt, vb * (size_t)hg->n, cudaMemcpyHostToDevice, s));
  }
  if (hg->ewgt) {
    GP_TRY(ws.get(&ew, eb * (size_t)hg->m_dir));
    GP_CUDA(cudaMemcpyAsync(ew, hg->ewgt, eb * (size_t)hg->m_dir, cudaMemcpyHostToDevice, s));
  }
  gp_graph dg = *hg;
  dg.offsets = off;
  dg.adj = adj;
  dg.vwgt = vw;
  dg.ewgt = ew;
  GP_TRY(partition_device(&dg, k, eps, seed, params, part, res, s));
  GP_CUDA(cudaMemcpyAsync(part_out_host, part, sizeof(int32_t) * (size_t)hg->n, cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  return GP_OK;
}

int gp_lp_set_schedule(int32_t deg_warp, int32_t deg_cta) {
  if (deg_warp < 0 || deg_cta < 0) {
    set_error("gp_lp_set_schedule: thresholds must be >= 0");
    return GP_ERR_INVALID_ARG;
  }
  g_schedule.deg_warp = deg_warp;
  g_schedule.deg_cta = deg_cta;
  return GP_OK;
}

int gp_lp_set_tiles(int64_t hub_batch_slots, int64_t verts_per_block) {
  if (hub_batch_slots < 0 || verts_per_block < 0) {
    set_error("gp_lp_set_tiles: tile sizes must be >= 0");
    return GP_ERR_INVALID_ARG;
  }
  g_schedule.hub_batch_slots = hub_batch_slots;
  g_schedule.verts_per_block = verts_per_block;
  return GP_OK;
}

int gp_lp_set_hub_keep(int64_t slots, int32_t max_load_pct) {
  if (max_load_pct < 0 || max_load_pct > 95) {
    set_error("gp_lp_set_hub_keep: max_load_pct must be in [0, 95]");
    return GP_ERR_INVALID_ARG;
  }
  g_schedule.hub_keep_slots = slots;
  g_keep_pct = max_load_pct;
  return GP_OK;
}

int gp_set_wait_limit(uint64_t ns) {
  gp::set_wait_limit_ns(ns);
  return GP_OK;
}

int64_t gp_pinned_stage_allocs(void) { return gp::pinned_stage_allocs(); }

int64_t gp_launch_count(int reset) { return gp::launch_count(reset); }

void gp_free_cached(void) { gp::free_cached(); }

// Times three LP rounds of g from singletons under each candidate configuration (the first sweep
// warms up) and returns the index of the fastest; *best_ms receives its time.
static int time_candidates(const DGraph &g, const std::vector<gp_params> &cand, int *best, double *best_ms,
                           cudaStream_t s) {
  Workspace ws(s);
  int32_t *labels;
  int64_t *lw;
  GP_TRY(ws.get(&labels, (size_t)std::max<int64_t>(g.n, 1)));
  GP_TRY(ws.get(&lw, (size_t)std::max<int64_t>(g.n, 1)));
  int64_t maxc = 0, W = 0;
  GP_TRY(vertex_weight_stats(g, &maxc, &W, s));
  const int64_t U = std::max<int64_t>(maxc, std::max<int64_t>(W / 32, 1));
  cudaEvent_t a, b;
  GP_CUDA(cudaEventCreate(&a));
  GP_CUDA(cudaEventCreate(&b));
  *best_ms = -1;
  *best = 0;
  for (int rep = 0; rep < 2; rep++) {
    for (size_t c = 0; c < cand.size(); c++) {
      const LpConfig cfg = lp_config_from(&cand[c]);
      if (g.n > 0) {
        (::gp::count_launch(), k_iota<<<grid_n(g.n), 256, 0, s>>>(labels, g.n));
        (::gp::count_launch(), k_vw_to_i64<<<grid_n(g.n), 256, 0, s>>>(g, lw));
      }
      int st = cudaEventRecord(a, s) == cudaSuccess ? GP_OK : GP_ERR_CUDA;
      if (st == GP_OK) st = run_lp(g, nullptr, labels, lw, g.n, U, 3, 0x5eedULL, nullptr, s, cfg, true);
      float ms = 0;
      if (st == GP_OK && (cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
        st = GP_ERR_CUDA;
      if (st != GP_OK) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (st == GP_ERR_CUDA) set_error("autotune: CUDA event timing failed");
        return st;
      }
      if (rep == 1 && (*best_ms < 0 || ms < *best_ms)) {
        *best_ms = ms;
        *best = (int)c;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return GP_OK;
}

int gp_autotune_schedule(const gp_graph *gd, int32_t *deg_warp_out, int32_t *deg_cta_out, double *ms_out,
                         gp_stream stream) {
  GP_TRY(check_graph_desc(gd));
  if (!deg_warp_out || !deg_cta_out) {
    set_error("gp_autotune_schedule: outputs are required");
    return GP_ERR_INVALID_ARG;
  }
  static const int cand[][2] = {{32, 256}, {64, 256}, {64, 512}, {128, 512}, {128, 1024}, {32, 1024},
                                {128, 2048}, {256, 2048}};
  std::vector<gp_params> cs;
  for (const auto &c : cand) {
    gp_params pr;
    gp_default_params(&pr);
    pr.deg_warp = c[0];
    pr.deg_cta = c[1];
    cs.push_back(pr);
  }
  int best = 0;
  double ms = 0;
  GP_TRY(time_candidates(make_dgraph(gd), cs, &best, &ms, (cudaStream_t)stream));
  *deg_warp_out = (int32_t)cs[best].deg_warp;
  *deg_cta_out = (int32_t)cs[best].deg_cta;
  if (ms_out) *ms_out = ms;
  return GP_OK;
}

int gp_autotune(const gp_graph *gd, gp_params *params, double *ms_out, gp_stream stream) {
  GP_TRY(check_graph_desc(gd));
  if (!params) {
    set_error("gp_autotune: params is required");
    return GP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int32_t dw = 0, dc = 0;
  double ms = 0;
  GP_TRY(gp_autotune_schedule(gd, &dw, &dc, &ms, stream));
  const DGraph g = make_dgraph(gd);
  // hubs under the chosen bins decide whether the hub batch size matters
  gp_params base;
  gp_default_params(&base);
  base.deg_warp = dw;
  base.deg_cta = dc;
  LpClassInfo ci;
  {
    Workspace ws(s);
    unsigned long long *words;
    GP_TRY(ws.get(&words, kLpClassWords));
    const LpConfig cfg = lp_config_from(&base);
    GP_TRY(lp_classes_launch(g, cfg, words, ws));
    unsigned long long hw[kLpClassWords];
    GP_CUDA(cudaMemcpyAsync(hw, words, sizeof(hw), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    lp_classes_from(hw, cfg, &ci);
  }
  std::vector<gp_params> cs;
  static const int64_t vpb[] = {32, 64, 128, 256};
  static const int64_t hbs[] = {int64_t(1) << 22, int64_t(1) << 24, int64_t(1) << 26};
  const bool hubs = ci.cls[6] > 0;
  for (int64_t v : vpb)
    for (int h = 0; h < (hubs ? 3 : 1); h++) {
      gp_params pr = base;
      pr.verts_per_block = v;
      pr.hub_batch_slots = hubs ? hbs[h] : 0;
      cs.push_back(pr);
    }
  int best = 0;
  GP_TRY(time_candidates(g, cs, &best, &ms, s));
  params->deg_warp = dw;
  params->deg_cta = dc;
  params->verts_per_block = cs[best].verts_per_block;
  params->hub_batch_slots = cs[best].hub_batch_slots;
  if (ms_out) *ms_out = ms;
  return GP_OK;
}

int gp_profile_enable(int on) { return gp::prof_enable(on); }
int gp_profile_read(gp_profile_entry *out, int max_entries, int reset) {
  return gp::prof_read(out, max_entries, reset);
}

}  // extern "C"
