/*
 * oracle.h -- C ABI of the CPU oracle (test infrastructure only).
 *
 * The oracle is a plain, slow, single-threaded restatement of the method of
 * "High-Quality Shared-Memory Graph Partitioning" (Akhremtsev, Sanders, Schulz): size-constrained
 * label propagation (Section III-A "Clustering", Section IV-A), contraction (Section III-A,
 * Section IV-A "Parallel Contraction"), initial partitioning by recursive bisection (Section III-B),
 * projection and label-propagation refinement (Section III-C, Section IV-C), with the deterministic
 * readings of the points the paper leaves open. It shares no code with the GPU library and is used
 * only by the tests, the smoke check and the CPU-baseline leg of the benchmark.
 *
 * All arrays are host memory owned by the caller. Offsets, vertex weights and edge weights are
 * int64 here (the Python wrapper widens narrower inputs); a NULL weight array means unit weights.
 */
#ifndef GP_ORACLE_H
#define GP_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_graph {
  int64_t n;
  int64_t m_dir;          /* directed CSR entries (2|E|) */
  const int64_t *off;     /* n+1 */
  const int32_t *adj;     /* m_dir, rows ascending */
  const int64_t *vw;      /* n or NULL */
  const int64_t *ew;      /* m_dir or NULL */
} or_graph;

typedef struct or_lp_stats {
  int64_t rounds;         /* rounds executed */
  int64_t moves;          /* admitted moves over all rounds */
  int64_t visits;         /* active-vertex visits */
  int64_t edges;          /* CSR entries scanned by visits */
  int64_t movers;         /* movers proposed (before admission) */
} or_lp_stats;

typedef struct or_params {
  int64_t cluster_div;        /* f: U = max(max c(v), floor(Lmax / f)) */
  int64_t rounds_coarsen;     /* l = 10 */
  int64_t rounds_refine;      /* 25 */
  int64_t coarse_min;         /* T = max(coarse_min, coarse_per_k * k) */
  int64_t coarse_per_k;
  int64_t stall_pct;          /* stop when 100 n' > stall_pct n */
  int64_t max_levels;
  int64_t ip_tries;
  int64_t repair_rounds;
  int64_t coarsen_mode;       /* 0: LP clustering (the paper's), 1: matching (or_match) */
  int64_t mls;                /* 0: off; else MLS with this many global iterations (other parameters
                                 default) after the LP refinement of every level, seed H(seed, level, 7) */
  int64_t lp_async;           /* 1: every LP run (coarsening, tries, refinement) in or_lp_async's order */
} or_params;

typedef struct or_match_stats {
  int64_t rounds;             /* rounds run */
  int64_t pairs;              /* matched pairs */
} or_match_stats;

typedef struct or_result {
  int64_t cut;
  int64_t max_block_weight;
  int64_t lmax;
  int64_t imbalanced;
  int64_t levels;             /* contractions performed */
  int64_t best_try;
  int64_t n_isolated;
  int64_t level_n[65];        /* n of each level graph (after isolated vertices are removed) */
  int64_t level_m[65];        /* m_dir of each level graph */
  int64_t try_cut[16];
  int64_t try_imbalanced[16];
  int64_t lp_edges;           /* CSR entries scanned by all LP runs */
} or_result;

/* SplitMix64 output function and the keyed hash H(a,b,c) = mix(mix(mix(a)^b)^c). */
uint64_t or_mix64(uint64_t z);
uint64_t or_hash3(uint64_t a, uint64_t b, uint64_t c);

/* Lmax = floor((1+eps) * ceil(W/k)), Section II-A. */
int64_t or_lmax(int64_t total_weight, int64_t k, double eps);

/* One size-constrained LP run (clustering or refinement). labels[n] and lw[nl] are in/out;
 * q (per CSR entry, or NULL) adds the learned tie-break and admission key. Returns 0 or -1. */
int or_lp(const or_graph *g, const int32_t *q, int32_t *labels, int64_t *lw, int64_t nl, int64_t U,
          int64_t rounds, uint64_t seed, or_lp_stats *st);

/* The paper's sequential, in-place LP order (Section III-A; the order of Section IV-A's asynchronous
 * form): vertices in (degree, id) order, moves applied at once. labels[n], lw[nl] in/out. */
int or_lp_async(const or_graph *g, int32_t *labels, int64_t *lw, int64_t nl, int64_t U, int64_t rounds,
                uint64_t seed, or_lp_stats *st);

/* Matching-based clustering (clusters of one or two vertices, Section III-A, Section VII): rounds of
 * deterministic handshake matching under the bound c(u) + c(v) <= U. labels[n] out. */
int or_match(const or_graph *g, int64_t U, int64_t rounds, uint64_t seed, int32_t *labels,
             or_match_stats *st);

/* Multi-try k-way local search (Section III-C, Section IV-C, Algorithm 1) on a k-way partition,
 * part[n] in/out; never violates lmax on blocks that satisfy it. Parameters and readings: mls.cpp. */
typedef struct or_mls_params {
  int64_t global_iters;  /* 3 (Section VI) */
  int64_t alpha_pct;     /* 10: a local iteration follows while its gain > 10% of the global one's */
  int64_t max_local;     /* cap on local iterations per global iteration (16) */
  int64_t max_moves;     /* moves per search (64) */
  int64_t fruitless;     /* a search stops after this many moves without a new best prefix (16) */
  int64_t queue_cap;     /* queued vertices per search (256) */
  int64_t max_degree;    /* vertices of larger degree are never moved (1024) */
} or_mls_params;
typedef struct or_mls_stats {
  int64_t gain;          /* cut reduction */
  int64_t moves;         /* applied moves */
  int64_t searches;      /* searches started */
  int64_t local_iters;   /* local iterations run */
} or_mls_stats;
void or_mls_default_params(or_mls_params *p);
int64_t or_mls(const or_graph *g, int64_t k, int64_t lmax, uint64_t seed, const or_mls_params *p, int32_t *part,
               or_mls_stats *st);

/* Contraction of labels[n] (values in [0,nl)). Outputs sized for the worst case:
 * off_out[n+1], adj_out[m_dir], vw_out[n], ew_out[m_dir], f2c[n]. Writes n' and m' to *n_out, *m_out. */
int or_contract(const or_graph *g, const int32_t *labels, int64_t nl, int64_t *n_out, int64_t *m_out,
                int64_t *off_out, int32_t *adj_out, int64_t *vw_out, int64_t *ew_out, int32_t *f2c);

/* Recursive bisection of one initial-partitioning try (no refinement). part[n] out. */
int or_bisect(const or_graph *g, int64_t k, uint64_t s_try, int32_t *part);

/* Balance repair rounds; part in/out. Returns the number of rounds run. */
int64_t or_repair(const or_graph *g, int64_t k, int64_t lmax, int64_t max_rounds, int32_t *part);

/* cut (each undirected edge once) and block weights bw[k]. */
int64_t or_cut(const or_graph *g, const int32_t *part, int64_t k, int64_t *bw);

/* Full multilevel partition. q_levels: NULL (plain) or one q array per coarsening level. */
void or_default_params(or_params *p);
int or_partition(const or_graph *g, int64_t k, double eps, uint64_t seed, const or_params *p,
                 const int32_t *const *q_levels, int64_t n_q_levels, int32_t *part, or_result *res);

/* Learned edge scorer, FP64: features (8 per CSR entry) and the 8->32->1 MLP. */
void or_edge_features(const or_graph *g, int64_t level, double *feat);
void or_mlp_forward(int64_t m, const double *x, const double *w1, const double *b1,
                    const double *w2, double b2, double *s_out);
/* Mean binary cross-entropy over m rows and its gradients. */
double or_mlp_loss_grad(int64_t m, const double *x, const double *y, const double *w1,
                        const double *b1, const double *w2, double b2, double *gw1, double *gb1,
                        double *gw2, double *gb2);

#ifdef __cplusplus
}
#endif
#endif
