// mlp.cu -- learned edge scorer (placeholder until the tensor-core kernels land).
#include "mlp.cuh"

namespace gp {
int mlp_score(const DGraph &, int, const gp_mlp *, float *, int32_t *, cudaStream_t) {
  set_error("learned scoring is not available in this build");
  return GP_ERR_UNSUPPORTED;
}
}  // namespace gp

extern "C" {
int gp_mlp_score(const gp_graph *, int32_t, const gp_mlp *, float *, int32_t *, gp_stream) {
  return GP_ERR_UNSUPPORTED;
}
int gp_edge_features(const gp_graph *, int32_t, float *, gp_stream) { return GP_ERR_UNSUPPORTED; }
int gp_mlp_train(const float *, const float *, int64_t, gp_mlp *, int32_t, float, float *, gp_stream) {
  return GP_ERR_UNSUPPORTED;
}
int gp_mlp_grad(const float *, const float *, int64_t, const gp_mlp *, float *, float *, gp_stream) {
  return GP_ERR_UNSUPPORTED;
}
int gp_partition_batch(const gp_batch_item *items, int32_t count, const gp_params *params, gp_result *res,
                       gp_stream stream) {
  if (count < 0 || (count > 0 && (!items || !res))) return GP_ERR_INVALID_ARG;
  for (int32_t i = 0; i < count; i++) {
    const int st = gp_partition(&items[i].g, items[i].k, items[i].eps, items[i].seed, params, items[i].part_out,
                                &res[i], stream);
    if (st != GP_OK) return st;
  }
  return GP_OK;
}
}
