// match.cuh -- matching-based clustering (clusters of one or two vertices) for the coarsening phase.
#pragma once

#include "gp_internal.cuh"

namespace gp {

struct MatchStats {
  int64_t rounds = 0;  // rounds run (the last one matched nothing, unless the cap was reached)
  int64_t pairs = 0;   // matched pairs
  int64_t visits = 0;  // unmatched-vertex visits
  int64_t edges = 0;   // CSR entries scanned by those visits
};

// Handshake matching of g under c(u) + c(v) <= U, at most `rounds` rounds, seeded by `seed`;
// labels[n] (device) receives min(v, mate(v)) or v. Statistics are read back (one synchronisation)
// only when read_stats is set or profiling is on.
int run_match(const DGraph &g, int64_t U, int rounds, uint64_t seed, int32_t *labels, MatchStats *out,
              cudaStream_t s, bool read_stats);

}  // namespace gp
