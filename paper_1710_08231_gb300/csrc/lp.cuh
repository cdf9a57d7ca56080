// lp.cuh -- size-constrained label propagation engine (clustering and refinement).
#pragma once

#include <vector>

#include "gp_internal.cuh"

namespace gp {

struct LpConfig {
  int deg_warp = 128;   // 32 < d <= deg_warp: one warp per vertex, shared-memory hash (<= 256; 128 with scores)
  int deg_cta = 2048;   // deg_warp < d <= deg_cta: one CTA per vertex, shared-memory hash (<= 2048; 1024 with
                        // scores or without a vertex of degree above 1024)
                        // d > deg_cta: several CTAs per vertex, global-memory hash
  // tile sizes: hub table slots per batch (the hub tables of one batch are reused by the next) and the
  // fewest vertices per block of a problem
  int64_t hub_batch_slots = int64_t(1) << 26;
  int64_t verts_per_block = 64;
  // hub tables are kept across sub-rounds (updated by the moves) when all hubs' tables of a launch take
  // at most this many slots; 0: never
  int64_t hub_keep_slots = int64_t(1) << 32;
  int hub_keep_pct = 75;  // a kept table goes stale (rebuilt at the hub's next activation) past this load
};
constexpr int64_t kMinHubBatchSlots = 4096, kMaxHubBatchSlots = int64_t(1) << 28;
constexpr int64_t kMinVertsPerBlock = 16, kMaxVertsPerBlock = 4096;

// Degree classes of a graph under one schedule (vertices per bin, CSR entries, largest hub table and
// the sum of hub tables). run_lp_multi fills it when `valid` is false and a later call on the same
// graph and schedule reuses it, skipping the class kernel and its copy back.
struct LpClassInfo {
  bool valid = false;
  int deg_warp = 0, deg_cta = 0;
  unsigned cls[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  unsigned long long entries = 0, hub_max_cap = 0, hub_cap_sum = 0;
  unsigned long long wide = 0;  // vertices of degree above 1024 (they need the larger shared tables)
};

// Degree classes of one graph computed without a read back: lp_classes_launch writes kLpClassWords
// words into words_dev (device, caller-owned) on the workspace's stream; after the caller has read
// them to the host, lp_classes_from fills the LpClassInfo.
constexpr int kLpClassWords = 9;
int lp_classes_launch(const DGraph &g, const LpConfig &cfg, unsigned long long *words_dev, Workspace &ws);
void lp_classes_from(const unsigned long long *words, const LpConfig &cfg, LpClassInfo *ci);

// Counters of several LP calls kept on the device and read back once (lp_collect) instead of after
// every call. `dev` holds `capacity` counter blocks (lp_counters_bytes() each, from the caller).
struct LpDeferred {
  void *dev = nullptr;
  int capacity = 0, count = 0;
  std::vector<int64_t> visit_bytes, entry_bytes;  // algorithmic bytes per visit and per entry, by job
  std::vector<const char *> names;                // profile entry of each job
};
size_t lp_counters_bytes();
// Reads every deferred counter block back (one synchronisation, shared with the caller's pending
// reads in `extra` when given), checks the device error flags and returns the summed LP edges and
// admitted moves; adds the LP profile entries when profiling.
int lp_collect(LpDeferred &def, cudaStream_t s, int64_t *edges, int64_t *moves, Readback *extra = nullptr);

// One LP run for run_lp_multi. With vbase/lbase != 0 the job is one graph of a disjoint union:
// g is its view (g.n local vertices, offsets and vertex weights shifted to its first vertex, adjacency
// and edge weights of the union), labels/lw are the union's arrays (labels hold global label ids
// lbase .. lbase + nl - 1) and hashes use local ids, so the result equals a run on the graph alone.
struct LpJob {
  DGraph g;
  int64_t vbase = 0, lbase = 0;
  const int32_t *q = nullptr;
  int32_t *labels = nullptr;
  int64_t *lw = nullptr;
  int64_t nl = 0, U = 0;
  int rounds = 0;
  uint64_t seed = 0;
  gp_lp_stats *stats = nullptr;
  // labels start as singletons (vertex v in label lbase + v): in the first sub-round every neighbour
  // label is distinct and no neighbour carries the own label, so connections need no aggregation
  bool singletons = false;
  LpClassInfo *classes = nullptr;  // optional cache of the graph's degree classes (see LpClassInfo)
  // profile entry the job's counts go to (static string); the launch is timed under jobs[0]'s
  const char *prof = "lp_persistent";
};

// Several independent LP runs in one cooperative launch; they must share the edge-weight type and
// whether scores are given.
int run_lp_multi(const LpJob *jobs, int njobs, cudaStream_t s, const LpConfig &cfg, LpDeferred *deferred = nullptr);

LpConfig lp_config_from(const gp_params *p);

// One LP run from (labels, lw). labels[n] in [0,nl) and lw[nl] (int64 label weights, equal to the
// vertex-weight sums) are device arrays updated in place. q: NULL or per-entry scores.
// seed is the run's hash seed. stats (host) may be NULL.
int run_lp(const DGraph &g, const int32_t *q, int32_t *labels, int64_t *lw, int64_t nl, int64_t U,
           int rounds, uint64_t seed, gp_lp_stats *stats, cudaStream_t s, const LpConfig &cfg,
           bool singletons = false, LpClassInfo *classes = nullptr, LpDeferred *deferred = nullptr,
           const char *prof = "lp_persistent");

// Block weights of a partition: bw[k] = sum of c(v) over part[v] = b (device). Sets *bad_dev
// (device int, may be NULL) when a block id is outside [0,k).
int block_weights(const DGraph &g, const int32_t *part, int64_t k, int64_t *bw, int *bad_dev,
                  cudaStream_t s);

}  // namespace gp
