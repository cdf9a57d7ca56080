// mlp.cuh -- learned edge scorer: features, BF16 tensor-core inference and training.
#pragma once

#include "gp_internal.cuh"

namespace gp {

// Scores of every CSR entry of g: s_out (float, may be NULL) and q_out = round-half-even(s * 2^15)
// (int32, may be NULL). mlp is a device pointer.
int mlp_score(const DGraph &g, int level, const gp_mlp *mlp, float *s_out, int32_t *q_out, cudaStream_t s);

}  // namespace gp
