// contract.cuh -- contraction of a clustering into the weighted quotient graph.
#pragma once

#include "gp_internal.cuh"

namespace gp {

// A device-resident coarse graph: int64 offsets, int32 adjacency, int64 vertex and edge weights.
struct OwnedGraph {
  int64_t n = 0, m = 0;
  int64_t max_vw = 0;  // largest vertex weight (filled by contract_graph)
  int64_t *off = nullptr;
  int32_t *adj = nullptr;
  int64_t *vw = nullptr;
  int64_t *ew = nullptr;
  size_t off_bytes = 0, adj_bytes = 0, vw_bytes = 0, ew_bytes = 0;
  DGraph view() const {
    DGraph d;
    d.n = n;
    d.m = m;
    d.off = off;
    d.adj = adj;
    d.vw = vw;
    d.ew = ew;
    d.off64 = 1;
    d.vw64 = 1;
    d.ew64 = 1;
    return d;
  }
  void release(cudaStream_t s) {
    dev_free(off, off_bytes, s);
    dev_free(adj, adj_bytes, s);
    dev_free(vw, vw_bytes, s);
    dev_free(ew, ew_bytes, s);
    off = nullptr;
    adj = nullptr;
    vw = nullptr;
    ew = nullptr;
  }
};

int alloc_graph(OwnedGraph *g, int64_t n, int64_t m, cudaStream_t s);

struct LpConfig;
struct LpClassInfo;

// labels[n] in [0, nl). Writes the coarse graph into *out (allocated here) and f2c[n] (device,
// caller-allocated, may be NULL). With cfg and cls (may be NULL) it also fills *cls with the coarse
// graph's LP degree classes under cfg, read back together with the coarse sizes.
int contract_graph(const DGraph &g, const int32_t *labels, int64_t nl, OwnedGraph *out, int32_t *f2c,
                   cudaStream_t s, const LpConfig *cfg = nullptr, LpClassInfo *cls = nullptr);

}  // namespace gp
