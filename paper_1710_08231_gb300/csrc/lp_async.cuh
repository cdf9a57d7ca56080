// lp_async.cuh -- asynchronous label propagation (Section IV-A), a non-deterministic comparator.
#pragma once

#include "gp_internal.cuh"

namespace gp {

// LP from (labels, lw) in the (degree, id) order with moves applied at once; single_warp runs one
// warp (the sequential order). A vertex may have at most 256 distinct neighbouring labels
// (GP_ERR_UNSUPPORTED otherwise).
int run_lp_async(const DGraph &g, int32_t *labels, int64_t *lw, int64_t nl, int64_t U, int rounds, uint64_t seed,
                 bool single_warp, gp_lp_stats *stats, cudaStream_t s);

}  // namespace gp
