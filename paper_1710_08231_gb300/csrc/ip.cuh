// ip.cuh -- initial partitioning, evaluation, projection and degree-0 vertex handling.
#pragma once

#include "contract.cuh"
#include "gp_internal.cuh"

namespace gp {

// Recursive bisection of `tries` independent tries (try t uses s_try = H(seed, level, 4 + t)),
// followed by balance repair. parts: tries * n int32 (device) receives the k-way partitions.
// err_dev (device int, may be NULL): see initial_partition_multi.
int initial_partition(const DGraph &g, int k, int64_t lmax, uint64_t seed, int level, int tries,
                      int repair_rounds, int32_t *parts, cudaStream_t s, int *err_dev = nullptr);

// The same for several graphs of a disjoint union in one launch (one CTA per graph and try).
struct IpJob {
  DGraph g;            // local view of the graph
  int64_t vbase = 0;   // adjacency values minus vbase are local ids
  int k = 1;
  int64_t lmax = 0;
  uint64_t seed = 0;
  int level = 0;
  int32_t *parts = nullptr;  // tries * g.n
};
// err_dev (device int, may be NULL): when given, the repair's error flag is copied there instead of
// being read back here (the caller reads it later, with other results), so the call does not wait.
int initial_partition_multi(const IpJob *jobs, int njobs, int tries, int repair_rounds, cudaStream_t s,
                            int *err_dev = nullptr);

// The kernels of eval_cut without the read back: *acc_dev (device) receives twice the cut.
int eval_cut_launch(const DGraph &g, const int32_t *part, int64_t k, unsigned long long *acc_dev, int64_t *bw_dev,
                    cudaStream_t s);

// cut (each undirected edge once) of part on g; also block weights into bw[k] when bw != NULL.
int eval_cut(const DGraph &g, const int32_t *part, int64_t k, int64_t *cut_host, int64_t *bw_dev,
             cudaStream_t s);

// fine[v] = coarse[f2c[v]]
int project(const int32_t *coarse, const int32_t *f2c, int64_t n, int32_t *fine, cudaStream_t s);

// Degree-0 vertices: rank[v] = new id of a vertex with neighbours, -1 otherwise. g0 is the graph
// induced by the vertices with neighbours, with the input's weight types (arrays from ws); when no
// vertex has degree 0, g0 is the input itself.
struct Stripped {
  int64_t n_iso = 0;
  int64_t n0 = 0;
  int32_t *rank = nullptr;  // n entries (device), NULL when n_iso == 0
  DGraph g0;
};
// With W_out / maxc_kept_out (host, may be NULL) it also returns the total vertex weight and the
// largest weight of a vertex with neighbours, from the same read back; with cfg and cls it fills *cls
// with g's LP degree classes when no vertex is stripped (then g is the level-0 graph).
int strip_isolated(const DGraph &g, Stripped *out, Workspace &ws, cudaStream_t s, int64_t *W_out = nullptr,
                   int64_t *maxc_kept_out = nullptr, const LpConfig *cfg = nullptr, LpClassInfo *cls = nullptr);

// part_full[v] = part0[rank[v]] for kept vertices; degree-0 vertices in ascending id order go
// to the block of minimum weight (ties: smaller id) given bw (block weights of the kept vertices).
int place_isolated(const DGraph &g, const Stripped &st, const int32_t *part0, int64_t k, int32_t *part_full,
                   cudaStream_t s);

// max over v of c(v), and sum over v of c(v) (host results)
int vertex_weight_stats(const DGraph &g, int64_t *maxc, int64_t *total, cudaStream_t s);

}  // namespace gp
