/*
 * gpart.h -- C ABI of the GB300 multilevel graph partitioner (label propagation hot path).
 *
 * Method: "High-Quality Shared-Memory Graph Partitioning" (Akhremtsev, Sanders, Schulz).
 *   - size-constrained label propagation (LP) clustering: Section III-A "Clustering",
 *     parallel form in Section IV-A "Parallel Size-Constraint Label Propagation";
 *   - contraction into the weighted quotient graph: Section III-A, Section IV-A
 *     "Parallel Contraction";
 *   - initial partitioning of the coarsest graph, best of several tries: Section III-B, IV-B;
 *   - projection and LP refinement with U = Lmax: Section III-C, Section IV-C;
 *   - balance bound Lmax = (1+eps) * ceil(c(V)/k) and the cut objective: Section II-A.
 *
 * Conventions shared by every entry point:
 *   - All graph arrays and all output arrays are DEVICE pointers owned by the caller unless the
 *     entry point says otherwise. Inputs are read-only.
 *   - A graph is undirected and stored as a symmetric CSR: row v lists N(v) in ascending order,
 *     both directions of an edge carry the same weight, there are no self-loops and no duplicate
 *     entries, and every weight is >= 1. n < 2^31. Vertex ids are int32.
 *   - Work is issued on `stream` (NULL = legacy default stream). Every entry point returns after
 *     its results are complete on the device and its host-side outputs are written (it
 *     synchronises `stream`).
 *   - Temporary device memory comes from the allocator installed with gp_set_allocator (by
 *     default cudaMallocAsync on `stream`) and is released before the call returns, except for
 *     the coarse graph returned by gp_contract.
 *   - Results are deterministic: for equal inputs and seed, every output is bit-identical across
 *     runs, launch configurations and degree-bin schedules.
 *   - Errors are returned as a gp_status code; nothing aborts and no exception crosses the ABI.
 *     gp_last_error() gives a one-line message for the last failing call on this thread. An
 *     imbalanced partition is a result (gp_result.imbalanced = 1), not an error.
 */
#ifndef GPART_H
#define GPART_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gp_stream; /* same type as cudaStream_t */

typedef enum gp_status {
  GP_OK = 0,
  GP_ERR_INVALID_ARG = 1, /* a scalar argument is out of range or a required pointer is NULL */
  GP_ERR_BAD_GRAPH = 2,   /* the CSR breaks the conventions above (checked by gp_validate_graph) */
  GP_ERR_OOM = 3,         /* the allocator returned NULL */
  GP_ERR_CUDA = 4,        /* a CUDA runtime call failed; gp_last_error() names it */
  GP_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  GP_ERR_INTERNAL = 6,    /* a device-side invariant check failed */
  GP_ERR_UNSUPPORTED = 7  /* the input exceeds a documented size limit */
} gp_status;

/* Graph descriptor. offsets: n+1 entries, int64 when offsets_64 != 0, else int32.
 * vwgt: n vertex weights c(v) (int64 when vwgt_64, else int32), NULL = unit weights.
 * ewgt: m_dir edge weights omega(e) (int64 when ewgt_64, else int32), NULL = unit weights.
 * m_dir is the number of CSR entries, 2|E|. */
typedef struct gp_graph {
  int64_t n;
  int64_t m_dir;
  const void *offsets;
  const int32_t *adj;
  const void *vwgt;
  const void *ewgt;
  int32_t offsets_64;
  int32_t vwgt_64;
  int32_t ewgt_64;
  int32_t reserved;
} gp_graph;

/* Statistics of one LP run. */
typedef struct gp_lp_stats {
  int64_t rounds;  /* rounds executed (stops early after a round without moves) */
  int64_t moves;   /* admitted moves */
  int64_t visits;  /* active-vertex visits */
  int64_t edges;   /* CSR entries scanned by those visits (the LP's traversed edges) */
  int64_t movers;  /* moves proposed before admission */
} gp_lp_stats;

/* Partitioning parameters; gp_default_params fills the values used by the paper where it gives
 * them (10 coarsening and 25 refinement LP iterations, 4 initial-partitioning tries: Section VI
 * "Algorithm Configuration") and this library's readings elsewhere. */
typedef struct gp_params {
  int64_t cluster_div;    /* f: cluster bound U = max(max c(v), floor(Lmax / f)); 14 */
  int64_t rounds_coarsen; /* 10 */
  int64_t rounds_refine;  /* 25 */
  int64_t coarse_min;     /* coarsening stops at n <= max(coarse_min, coarse_per_k * k); 2000 */
  int64_t coarse_per_k;   /* 64 */
  int64_t stall_pct;      /* ... or when a level keeps more than stall_pct % of the vertices; 95 */
  int64_t max_levels;     /* ... or after this many contractions; 64 */
  int64_t ip_tries;       /* initial-partitioning tries, 1..16; 4 */
  int64_t repair_rounds;  /* balance-repair rounds after bisection; 16 */
  int32_t mode;           /* GP_MODE_PLAIN, GP_MODE_LEARNED or GP_MODE_BEST_OF */
  int32_t deg_warp;       /* degree-bin thresholds (0 = default); see gp_lp_cluster */
  int32_t deg_cta;
  int32_t coarsen;        /* GP_COARSEN_LP (the paper's clustering, default) or GP_COARSEN_MATCHING */
  const void *mlp;        /* device pointer to a gp_mlp (learned modes), else NULL */
  /* LP tile sizes (0 = default; never change results): hub table slots per batch of the multi-CTA
   * hub path (default 64M, clamped to [4096, 2^28]) and the fewest vertices per CTA of one LP problem
   * (default 64, clamped to [16, 4096]) */
  int64_t hub_batch_slots;
  int64_t verts_per_block;
  /* multi-try k-way local search after the LP refinement of every level (gp_mls with its default
   * parameters and this many global iterations; 0 = off, the default; the paper's configuration uses 3).
   * Plain mode, k <= 256. */
  int64_t mls_global_iters;
  /* 1: every LP run of the partition (coarsening, the tries' refinement, uncoarsening) uses
   * gp_lp_cluster_async's asynchronous order instead of the deterministic Jacobi rounds: the paper's
   * own scheme, non-deterministic, a comparator for what determinism costs (plain mode). */
  int64_t lp_async;
  /* Hub tables (vertices above deg_cta) kept across LP sub-rounds and updated by the moves, instead of
   * re-accumulated from the hubs' rows every sub-round, when the tables of all hubs of one LP call take
   * at most this many slots (12 bytes each, 20 with scores). 0 = default 2^32,
   * negative = never. Never changes results. */
  int64_t hub_keep_slots;
} gp_params;

enum { GP_MODE_PLAIN = 0, GP_MODE_LEARNED = 1, GP_MODE_BEST_OF = 2 };
/* Clustering of the coarsening phase: size-constrained LP, or matching (clusters of one or two
 * vertices, see gp_match; plain mode only). */
enum { GP_COARSEN_LP = 0, GP_COARSEN_MATCHING = 1 };

/* Result of gp_partition (host struct, written by the call). */
typedef struct gp_result {
  int64_t cut;              /* total weight of cut edges, each undirected edge once */
  int64_t max_block_weight;
  int64_t lmax;             /* Lmax = floor((1+eps) * ceil(c(V)/k)) as int64 */
  int64_t imbalanced;       /* 1 when max_block_weight > lmax */
  int64_t levels;           /* contractions performed */
  int64_t best_try;         /* index of the initial-partitioning try kept */
  int64_t n_isolated;       /* degree-0 vertices set aside before coarsening */
  int64_t level_n[65];      /* vertices of each level graph (level 0 = input minus isolated) */
  int64_t level_m[65];      /* CSR entries of each level graph */
  int64_t try_cut[16];
  int64_t try_imbalanced[16];
  int64_t lp_edges;         /* CSR entries scanned by all LP runs of the call */
  int64_t lp_moves;
  int64_t plain_cut;        /* GP_MODE_BEST_OF: cut of the plain run */
  int64_t learned_cut;      /* GP_MODE_BEST_OF / LEARNED: cut of the learned run */
  double ms_total;          /* host wall time of the call */
  double ms_coarsen, ms_initial, ms_refine;
} gp_result;

/* Learned edge scorer: 8 features -> 32 hidden (ReLU) -> 1 (sigmoid). Stored in device memory as
 * this struct; weights are bfloat16 bit patterns (uint16), biases float. w1 is row-major
 * [32][8] (w1[j*8+i] multiplies feature i for hidden unit j). */
typedef struct gp_mlp {
  uint16_t w1[256];
  uint16_t w2[32];
  float b1[32];
  float b2;
  float pad[7];
} gp_mlp;

/* ---------------------------------------------------------------------------------------- */
/* Library */

const char *gp_version(void);
const char *gp_status_string(int status);
/* One-line description of the last error on the calling thread ("" when none). */
const char *gp_last_error(void);

/* Install the temporary-memory allocator. alloc(bytes, stream, ctx) returns device memory usable
 * in stream order on `stream` (or NULL on failure); release(ptr, bytes, stream, ctx) gives it back.
 * Passing alloc = NULL restores the default (cudaMallocAsync / cudaFreeAsync). Not thread-safe with
 * respect to concurrent calls. */
typedef void *(*gp_alloc_fn)(size_t bytes, gp_stream stream, void *ctx);
typedef void (*gp_free_fn)(void *ptr, size_t bytes, gp_stream stream, void *ctx);
int gp_set_allocator(gp_alloc_fn alloc, gp_free_fn release, void *ctx);

/* Freed device blocks of up to 64 MiB are kept by the library (at most 1 GiB in all) and reused for
 * allocations of exactly the same size on the same stream, so repeated calls on graphs of one shape
 * make no allocator calls after the first. gp_free_cached returns every kept block to the allocator
 * (stream-ordered on the stream that freed it). gp_set_allocator does the same before switching. */
void gp_free_cached(void);

void gp_default_params(gp_params *params);

/* Check the CSR conventions on the device. Returns GP_OK or GP_ERR_BAD_GRAPH. */
int gp_validate_graph(const gp_graph *g, gp_stream stream);

/* Lmax = floor((1+eps) * ceil(W/k)) for total vertex weight W (Section II-A). Host function. */
int64_t gp_lmax(int64_t total_weight, int64_t k, double eps);

/* ---------------------------------------------------------------------------------------- */
/* Hot-path calls */

/* Size-constrained LP clustering (Section III-A "Clustering", Section IV-A): starts from
 * C[v] = v and runs `rounds` rounds (stopping after a round without moves). Each round has two
 * Jacobi sub-rounds; vertex v takes part in sub-round H(seed, r, v) >> 63 of round r (all
 * vertices in round 0, afterwards only neighbours of vertices moved in the previous round). A
 * vertex proposes the eligible label (cluster weight + c(v) <= U) of largest connection
 * omega({(v,u) : C[u] = L}); its own label wins ties; among others the larger sum of edge_q
 * (when given), then the larger H(seed, v, L), then the smaller L wins. Proposals to one label are
 * admitted in (gain desc, edge_q sum desc, v asc) order while the label's weight at the start of
 * the sub-round plus the admitted weight stays <= U.
 *   g         : input graph (device arrays)
 *   U         : cluster weight bound, >= max c(v)
 *   rounds    : >= 0
 *   seed      : hash seed of this run (the partitioner passes H(seed, level, 1))
 *   edge_q    : NULL, or m_dir int32 per-entry scores (learned tie-break; symmetric)
 *   labels_out: n int32, caller-allocated; receives C[v] in [0, n) (may be NULL when n = 0)
 *   stats     : NULL or host struct receiving counters
 * Degree bins (thread group, warp, CTA or multi-CTA per vertex) change the schedule only. */
int gp_lp_cluster(const gp_graph *g, int64_t U, int32_t rounds, uint64_t seed,
                  const int32_t *edge_q, int32_t *labels_out, gp_lp_stats *stats,
                  gp_stream stream);

/* The paper's asynchronous size-constrained LP (Section III-A order, Section IV-A parallel form) from
 * C[v] = v: vertices in increasing order of degree (ties: id) are taken in packets of 32 by warps;
 * each vertex moves at once to the eligible cluster of strongest connection (own label on ties, then
 * larger H(seed, v, L), then smaller L), reading labels and cluster weights as they are at that moment,
 * the target's weight reserved by compare-and-swap so that no cluster exceeds U; neighbours of moved
 * vertices are queued for the next round. Not deterministic: a comparator for gp_lp_cluster's Jacobi
 * rounds. With single_warp != 0 one warp runs everything in the sequential order (deterministic).
 * Arguments as gp_lp_cluster. A vertex may have at most 256 distinct neighbouring labels: graphs of
 * maximum degree above 256 return GP_ERR_UNSUPPORTED. */
int gp_lp_cluster_async(const gp_graph *g, int64_t U, int32_t rounds, uint64_t seed, int32_t single_warp,
                        int32_t *labels_out, gp_lp_stats *stats, gp_stream stream);

/* gp_lp_cluster without any device allocation, for callers that cannot allocate device memory
 * while they run (no cudaMalloc, no caching allocator, no allocator callback). The paper has no
 * counterpart; this is a deployment variant of gp_lp_cluster with identical results.
 *   Arguments, layout and results are those of gp_lp_cluster; the caller still owns the graph,
 *   labels_out and stats.
 *   Temporary buffers come from one fixed 16 MiB device array inside the library, which every
 *   process that loads the library holds on each GPU it uses until exit. Graphs with
 *   n > 32768 vertices or m_dir > 131072 CSR entries are rejected with GP_ERR_UNSUPPORTED.
 *   The call makes no pinned host allocation either (cudaMallocHost): its few read-backs of counters
 *   go straight into ordinary host memory. gp_pinned_stage_allocs() lets a caller check this.
 *   The first call on a device looks the array's device address up (with that device current); make
 *   that first call before any stream capture.
 *   All calls share the array and it keeps the last call's contents (every call clears what must
 *   start at zero), so calls whose GPU work overlaps (other threads, other streams) race: serialise
 *   them. */
int gp_lp_cluster_noalloc(const gp_graph *g, int64_t U, int32_t rounds, uint64_t seed,
                          const int32_t *edge_q, int32_t *labels_out, gp_lp_stats *stats,
                          gp_stream stream);

/* Matching-based clustering (Section III-A names matchings, clusters of size two, as the other family
 * of clusterings; Section VII plans a parallel matching for the coarsening of mesh-like graphs). The
 * library's reading: deterministic handshake matching. Each round, every unmatched vertex v proposes
 * to its unmatched neighbour u with c(v) + c(u) <= U of largest rating omega(v,u)^2 / (c(v) c(u))
 * (compared exactly in 128-bit integers), ties to the larger H(seed, min(u,v), max(u,v)), then the
 * smaller u; two vertices proposing to each other are matched. Rounds stop after one without a new
 * pair or after `rounds`. Run to convergence this is the greedy matching in decreasing rating order.
 *   labels_out: n int32 (device, caller-allocated): min(v, mate(v)) for matched v, else v
 *   stats     : NULL or host struct
 * Exact for omega < 2^44 and c < 2^40 (128-bit products). */
typedef struct gp_match_stats {
  int64_t rounds;  /* rounds run */
  int64_t pairs;   /* matched pairs */
  int64_t visits;  /* unmatched-vertex visits */
  int64_t edges;   /* CSR entries scanned */
} gp_match_stats;
int gp_match(const gp_graph *g, int64_t U, int32_t rounds, uint64_t seed, int32_t *labels_out,
             gp_match_stats *stats, gp_stream stream);

/* Degree-bin schedule of gp_lp_cluster and gp_lp_refine (process-wide): vertices with
 * 32 < d <= deg_warp are handled by one warp, deg_warp < d <= deg_cta by one CTA, larger ones by
 * several CTAs. 0 restores the defaults (128, 2048). deg_warp is clamped to [32, 256] and deg_cta to
 * [deg_warp, 2048] (runs with scores: [32, 128] and [deg_warp, 1024]). The schedule never changes
 * results. gp_partition uses params.deg_warp/deg_cta
 * when non-zero, else this schedule. */
int gp_lp_set_schedule(int32_t deg_warp, int32_t deg_cta);

/* LP tile sizes of gp_lp_cluster and gp_lp_refine (process-wide), as gp_params.hub_batch_slots and
 * gp_params.verts_per_block; 0 restores a default. Tile sizes never change results: a small
 * hub_batch_slots splits the hubs of one sub-round into many batches (each with its own table pass),
 * which the tests use to compare the multi-batch hub path with the oracle on small graphs. */
int gp_lp_set_tiles(int64_t hub_batch_slots, int64_t verts_per_block);

/* Kept hub tables (process-wide). slots: as gp_params.hub_keep_slots for gp_lp_cluster and
 * gp_lp_refine (0 restores the default, negative re-accumulates every hub in every sub-round).
 * max_load_pct (every LP call, gp_partition's too): a kept table whose key bound would pass this share
 * of its slots goes stale and is accumulated again at the hub's next activation; 0 restores the
 * default 75, 1 makes every table go stale at its first new label (the tests use both to compare the
 * update and rebuild paths with the oracle). Range [0, 95]. Never changes results. */
int gp_lp_set_hub_keep(int64_t slots, int32_t max_load_pct);

/* LP refinement of a k-way partition (Section III-C, Section IV-C): the same rounds with labels
 * = blocks 0..k-1 and U = lmax.
 *   part_inout : n int32 block ids in [0,k) (device), improved in place (may be NULL when n = 0)
 *   block_w_out: NULL or k int64 (device) receiving the final block weights
 * Returns GP_ERR_INVALID_ARG when a block id is out of range. */
int gp_lp_refine(const gp_graph *g, int32_t k, int64_t lmax, int32_t rounds, uint64_t seed,
                 int32_t *part_inout, int64_t *block_w_out, gp_lp_stats *stats, gp_stream stream);

/* Multi-try k-way local search, MLS (Section III-C; parallel form Section IV-C, Algorithm 1), on a k-way
 * partition. Global iterations start from all boundary vertices; in every local iteration one search
 * per todo vertex (one warp each) runs on the partition of the iteration's start: it queues the start
 * vertex and its neighbours by gain, moves the vertex of largest gain (negative gains allowed), queues
 * the neighbours of moved vertices and keeps its best prefix (PerformMoves); the recorded sequences are
 * then applied in todo order with every gain recomputed on the current partition, each up to its best
 * prefix (ApplyMoves). Local iterations continue on the moved vertices while their gain exceeds
 * alpha_pct % of the global iteration's gain. The library's readings where the paper is open: todo
 * lists ordered by H(s, v, 1); queue order (gain, H(s, w, 0), -w); targets the best adjacent block under
 * lmax by (connection, H(s, w, b), -b); the adaptive stopping rule replaced by max_moves and fruitless;
 * vertices of degree > max_degree never move. The cut never grows and no block ends above lmax unless
 * it started there.
 *   part_inout: n int32 in [0, k) (device); k <= 256
 *   params    : NULL for gp_mls_default_params (3 global iterations, alpha 10 %, 16 local iterations,
 *               64 moves, 16 fruitless moves, a queue of 256, degree bound 1024); max_moves <= 64,
 *               queue_cap <= 256, else GP_ERR_UNSUPPORTED
 *   stats     : NULL or host struct */
typedef struct gp_mls_params {
  int64_t global_iters, alpha_pct, max_local, max_moves, fruitless, queue_cap, max_degree;
} gp_mls_params;
typedef struct gp_mls_stats {
  int64_t gain;         /* cut reduction */
  int64_t moves;        /* applied moves */
  int64_t searches;     /* searches run */
  int64_t local_iters;  /* local iterations */
} gp_mls_stats;
void gp_mls_default_params(gp_mls_params *params);
int gp_mls(const gp_graph *g, int32_t k, int64_t lmax, uint64_t seed, const gp_mls_params *params,
           int32_t *part_inout, gp_mls_stats *stats, gp_stream stream);

/* Contraction of a clustering (Section III-A; Section IV-A "Parallel Contraction"): cluster ids
 * are renumbered by their rank among the used ids (prefix sum over a used-flag array), the coarse
 * vertex weight is the cluster weight, and the coarse edge (a,b), a != b, weighs the total weight
 * of fine edges between clusters a and b. Rows of the coarse CSR are sorted by neighbour id.
 *   labels : n int32 in [0, n) (device; may be NULL when n = 0)
 *   coarse : receives a library-owned coarse graph (int64 offsets, int64 vertex and edge weights);
 *            release it with gp_coarse_free
 *   f2c_out: NULL or n int32 (device) receiving the coarse id of every fine vertex */
typedef struct gp_coarse gp_coarse;
int gp_contract(const gp_graph *g, const int32_t *labels, gp_coarse **coarse, int32_t *f2c_out,
                gp_stream stream);
const gp_graph *gp_coarse_graph(const gp_coarse *c);
void gp_coarse_free(gp_coarse *c, gp_stream stream);

/* Full multilevel partition into k blocks (Section III, Section IV): strip degree-0 vertices,
 * coarsen by LP clustering + contraction, partition the coarsest graph `ip_tries` times by
 * recursive bisection + balance repair + LP refinement and keep the best (cut, imbalanced, try),
 * then project and LP-refine level by level, and give degree-0 vertices to the lightest blocks.
 *   k        : 1 <= k <= n
 *   eps      : >= 0
 *   params   : NULL for gp_default_params
 *   part_out : n int32 (device), caller-allocated
 *   res      : host struct (required) */
int gp_partition(const gp_graph *g, int32_t k, double eps, uint64_t seed, const gp_params *params,
                 int32_t *part_out, gp_result *res, gp_stream stream);

/* gp_partition on HOST arrays: the graph arrays and part_out are host pointers; the call copies
 * the graph to the device, partitions it and copies the partition back. */
int gp_partition_host(const gp_graph *host_g, int32_t k, double eps, uint64_t seed,
                      const gp_params *params, int32_t *part_out_host, gp_result *res,
                      gp_stream stream);

/* Learned scorer inference on every CSR entry of g (device):
 *   s_out: NULL or m_dir float scores in [0,1];  q_out: NULL or m_dir int32 round-half-even(s*2^15)
 *   level: coarsening level (feature 7 is level/16) */
int gp_mlp_score(const gp_graph *g, int32_t level, const gp_mlp *mlp, float *s_out,
                 int32_t *q_out, gp_stream stream);

/* Learned scorer features (8 float per CSR entry, row-major [m_dir][8]) into feat_out (device). */
int gp_edge_features(const gp_graph *g, int32_t level, float *feat_out, gp_stream stream);

/* Training of the scorer with Adam on (features, labels): feat [m][8] float and y [m] float in
 * {0,1} (device), `steps` full-batch steps of mean binary cross-entropy; mlp is updated in place
 * (device). loss_out: NULL or host array of `steps` floats receiving the loss before each step. */
int gp_mlp_train(const float *feat, const float *y, int64_t m, gp_mlp *mlp, int32_t steps,
                 float lr, float *loss_out, gp_stream stream);

/* Loss and gradients of the scorer on (feat, y) without an update, in FP32 accumulation from the
 * bf16 weights (device in, host out): grad_out[0..255] = dW1, [256..287] = db1, [288..319] = dW2,
 * [320] = db2. Returns the mean loss through *loss_out. */
int gp_mlp_grad(const float *feat, const float *y, int64_t m, const gp_mlp *mlp, float *loss_out,
                float *grad_out, gp_stream stream);

/* ---------------------------------------------------------------------------------------- */
/* Batched partitioning of many independent graphs (one call, persistent device schedule). */

typedef struct gp_batch_item {
  gp_graph g;         /* device arrays of graph i */
  int32_t k;
  int32_t reserved;
  double eps;
  uint64_t seed;
  int32_t *part_out;  /* device, g.n entries */
} gp_batch_item;

/* Partition `count` graphs in one call. Every graph is partitioned exactly as gp_partition would
 * partition it alone (same seeds, bounds and result); the work of all graphs is shared: one
 * cooperative LP launch per level covers every graph (each an independent problem), one contraction
 * runs on the disjoint union of the level graphs, and one launch does the initial partitioning of
 * every graph and try. Modes: GP_MODE_PLAIN or GP_MODE_LEARNED. The union of the graphs must have
 * fewer than 2^31 - 1 vertices. res: host array of `count` results (times are for the whole call). */
int gp_partition_batch(const gp_batch_item *items, int32_t count, const gp_params *params,
                       gp_result *res, gp_stream stream);

/* Degree-bin schedule autotuner: times three LP rounds of g under a fixed set of (deg_warp, deg_cta)
 * candidates (32..256, 256..2048) and returns the fastest (results never depend on the schedule). ms_out: NULL or the
 * best time. Pass the result in gp_params.deg_warp/deg_cta or to gp_lp_set_schedule. */
int gp_autotune_schedule(const gp_graph *g, int32_t *deg_warp_out, int32_t *deg_cta_out, double *ms_out,
                         gp_stream stream);

/* Schedule and tile-size autotuner: as gp_autotune_schedule, then, with the best degree bins, times
 * three LP rounds under candidate tile sizes (verts_per_block in {32, 64, 128, 256}; when g has
 * vertices of degree > deg_cta, hub_batch_slots in {4M, 16M, 64M}) and writes the fastest into
 * params->deg_warp, deg_cta, verts_per_block and hub_batch_slots (other fields are left as they are).
 * params: host struct (required), typically from gp_default_params. */
int gp_autotune(const gp_graph *g, gp_params *params, double *ms_out, gp_stream stream);

/* ---------------------------------------------------------------------------------------- */
/* Profiling: when enabled, the library records CUDA events on the caller's stream around each
 * launch of its named hot kernels (the LP aggregate+choose kernels of every degree bin, the
 * contraction row kernels) and accumulates per name: launches, summed device time, items
 * processed, CSR entries scanned and algorithmic bytes (CSR, labels and weights the method must
 * touch; implementation scratch is not counted). Enabling adds two event records per launch. */
typedef struct gp_profile_entry {
  char name[40];
  int64_t launches;
  double ms;
  int64_t items;
  int64_t edges;
  int64_t bytes;
} gp_profile_entry;
int gp_profile_enable(int on);
/* Limit of every bounded device-side wait (the grid barriers of the LP kernel), in nanoseconds of the
 * GPU's global timer; 0 restores the default of 20 s. A wait that runs out makes the call return
 * GP_ERR_TIMEOUT after every CTA of the kernel has returned (the CUDA context stays usable). The limit is
 * process-wide and read when a call launches its kernels. */
int gp_set_wait_limit(uint64_t ns);
/* Number of pinned host staging buffers (cudaMallocHost) the library has allocated for its device-to-
 * host read-backs since load. gp_lp_cluster_noalloc never adds to it. */
int64_t gp_pinned_stage_allocs(void);
/* Number of kernel launches the library has issued since load (or since the last reset != 0). */
int64_t gp_launch_count(int reset);
/* Copies up to max_entries entries into out and returns how many were written; reset != 0 clears
 * the accumulated entries. Launches recorded by the calls are resolved here (this call waits for
 * them); the calls themselves only record CUDA events on their stream. */
int gp_profile_read(gp_profile_entry *out, int max_entries, int reset);

#ifdef __cplusplus
}
#endif
#endif /* GPART_H */
