// noalloc.cu -- label-propagation clustering for callers that cannot allocate device memory.
//
// gp_lp_cluster obtains its temporary device buffers (degree bins, mover records, admission keys,
// active flags, label weights) from an allocator on every call. Some callers cannot allow that: code
// that must not call cudaMalloc or a caching allocator while it runs (for example a real-time loop
// or a process whose device memory is fully reserved up front). gp_lp_cluster_noalloc runs the same
// kernels on the same inputs and outputs, but every temporary buffer is carved from the file-scope
// array below, which every process that loads this library keeps on each GPU it uses until exit.
#include <mutex>

#include "gp_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int64_t kMaxVertices = 32768;
constexpr int64_t kMaxEntries = 131072;

static __device__ __align__(256) unsigned char g_lp_scratch[kScratchBytes];

// Device address of g_lp_scratch per device, looked up once with that device current.
std::mutex g_mu;
void *g_scratch_addr[64] = {};

}  // namespace

extern "C" int gp_lp_cluster_noalloc(const gp_graph *g, int64_t U, int32_t rounds, uint64_t seed,
                                     const int32_t *edge_q, int32_t *labels_out, gp_lp_stats *stats,
                                     gp_stream stream) {
  if (!g) {
    gp::set_error("gp_lp_cluster_noalloc: graph descriptor is NULL");
    return GP_ERR_INVALID_ARG;
  }
  if (g->n > kMaxVertices || g->m_dir > kMaxEntries) {
    gp::set_error("gp_lp_cluster_noalloc: graph exceeds the fixed scratch limits (n <= 32768 vertices, "
                  "m_dir <= 131072 CSR entries)");
    return GP_ERR_UNSUPPORTED;
  }
  int dev = 0;
  GP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    gp::set_error("gp_lp_cluster_noalloc: device index out of range");
    return GP_ERR_UNSUPPORTED;
  }
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      // In host code the array's name is only a stand-in; the device address must be looked up.
      GP_CUDA(cudaGetSymbolAddress(&g_scratch_addr[dev], g_lp_scratch));
    }
    base = g_scratch_addr[dev];
  }
  gp::ScratchArena arena{static_cast<unsigned char *>(base), kScratchBytes, 0, 0};
  gp::set_thread_arena(&arena);
  const int st = gp_lp_cluster(g, U, rounds, seed, edge_q, labels_out, stats, stream);
  gp::set_thread_arena(nullptr);
  if (st == GP_ERR_OOM)
    gp::set_error("gp_lp_cluster_noalloc: the fixed 16 MiB scratch array is too small for this graph");
  return st;
}
