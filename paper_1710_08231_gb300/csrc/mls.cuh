// mls.cuh -- multi-try k-way local search (Section III-C, Section IV-C).
#pragma once

#include "gp_internal.cuh"

namespace gp {

struct MlsParams {
  int64_t global_iters, alpha_pct, max_local, max_moves, fruitless, queue_cap, max_degree;
};
struct MlsStats {
  int64_t gain = 0, moves = 0, searches = 0, local_iters = 0;
};
void mls_default_params(MlsParams *p);

// MLS on the k-way partition part[n] (device, in/out) of g under lmax. k <= 256, max_moves <= 64,
// queue_cap <= 256 (else GP_ERR_UNSUPPORTED).
int run_mls(const DGraph &g, int k, int64_t lmax, uint64_t seed, const MlsParams &p, int32_t *part, MlsStats *out,
            cudaStream_t s);

}  // namespace gp
