// gp_internal.cuh -- shared device/host utilities of the GB300 partitioner library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gpart.h"

namespace gp {

// ------------------------------------------------------------------------------------------ status
void set_error(const std::string &msg);

#define GP_TRY(...)                               \
  do {                                            \
    int _st = (__VA_ARGS__);                      \
    if (_st != GP_OK) return _st;                 \
  } while (0)

#define GP_CUDA(expr)                                                                      \
  do {                                                                                     \
    cudaError_t _e = (expr);                                                               \
    if (_e != cudaSuccess) {                                                               \
      ::gp::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e) + " at " +       \
                      __FILE__ + ":" + std::to_string(__LINE__));                          \
      return GP_ERR_CUDA;                                                                  \
    }                                                                                      \
  } while (0)

#define GP_LAUNCH_CHECK() GP_CUDA(cudaGetLastError())

// ------------------------------------------------------------------------------------------ memory
struct ScratchArena {
  unsigned char *base;
  size_t size;
  size_t used;
  size_t high;
};
void set_thread_arena(ScratchArena *a);
bool arena_active();
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, size_t bytes, cudaStream_t s);
void free_cached();  // returns the blocks the library keeps for reuse to the allocator
long long pinned_stage_allocs();  // pinned host staging allocations made by Readback so far

// Several device ranges read to host memory with one synchronisation of the stream: the copies go
// through the calling thread's pinned staging buffer (so they are queued without blocking) and are
// scattered to their host destinations after the single cudaStreamSynchronize.
struct Readback {
  struct Item {
    void *host;
    const void *dev;
    size_t bytes, off;
  };
  std::vector<Item> items;
  size_t total = 0;
  void add(void *host, const void *dev, size_t bytes) {
    items.push_back({host, dev, bytes, total});
    total += (bytes + 15) & ~size_t(15);
  }
  int run(cudaStream_t s);
};

// Scoped set of temporary allocations, released in stream order when the scope ends.
class Workspace {
 public:
  explicit Workspace(cudaStream_t s) : s_(s) {}
  ~Workspace() { release(); }
  Workspace(const Workspace &) = delete;
  Workspace &operator=(const Workspace &) = delete;
  // Buffers of up to kChunk bytes are carved out of kChunk-byte chunks (one allocator call per
  // chunk); larger ones get an allocation of their own. Every buffer starts on a 256-byte boundary.
  // With a scratch arena active, every buffer is allocated exactly (no chunk slack).
  template <class T>
  int get(T **out, size_t count) {
    size_t bytes = (count ? count : 1) * sizeof(T);
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (bytes <= kChunk && !arena_active()) {
      if (chunk_left_ < bytes) {
        void *c = dev_alloc(kChunk, s_);
        if (!c) {
          set_error("device allocation of " + std::to_string(kChunk) + " bytes failed");
          return GP_ERR_OOM;
        }
        items_.push_back({c, kChunk});
        chunk_ptr_ = static_cast<char *>(c);
        chunk_left_ = kChunk;
      }
      p = chunk_ptr_;
      chunk_ptr_ += bytes;
      chunk_left_ -= bytes;
    } else {
      p = dev_alloc(bytes, s_);
      if (!p) {
        set_error("device allocation of " + std::to_string(bytes) + " bytes failed");
        return GP_ERR_OOM;
      }
      items_.push_back({p, bytes});
    }
    *out = static_cast<T *>(p);
    return GP_OK;
  }
  template <class T>
  int zeros(T **out, size_t count) {
    GP_TRY(get(out, count));
    GP_CUDA(cudaMemsetAsync(*out, 0, (count ? count : 1) * sizeof(T), s_));
    return GP_OK;
  }
  void release() {
    for (auto it = items_.rbegin(); it != items_.rend(); ++it) dev_free(it->p, it->bytes, s_);
    items_.clear();
    chunk_ptr_ = nullptr;
    chunk_left_ = 0;
  }
  cudaStream_t stream() const { return s_; }

 private:
  static constexpr size_t kChunk = size_t(2) << 20;
  struct Item {
    void *p;
    size_t bytes;
  };
  cudaStream_t s_;
  std::vector<Item> items_;
  char *chunk_ptr_ = nullptr;
  size_t chunk_left_ = 0;
};

// ------------------------------------------------------------------------------------------ hash
// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014) and the keyed hash
// H(a,b,c) = mix(mix(mix(a) ^ b) ^ c) that decides sub-rounds and ties.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t hash3(uint64_t a, uint64_t b, uint64_t c) {
  return mix64(mix64(mix64(a) ^ b) ^ c);
}

// Slot hash for open-addressing tables: the 32-bit finalizer of MurmurHash3 (Appleby), a bijection
// whose low bits depend on every input bit. Vertex ids of skewed generators (R-MAT) share their low
// bits far more often than uniform ids, so a table index must not be taken from them directly.
__host__ __device__ __forceinline__ unsigned mix32(unsigned h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// ------------------------------------------------------------------------------------------ graph
// Device view of a CSR graph with runtime-typed offsets and weights.
struct DGraph {
  int64_t n = 0, m = 0;
  const void *off = nullptr;
  const int32_t *adj = nullptr;
  const void *vw = nullptr;
  const void *ew = nullptr;
  int off64 = 0, vw64 = 0, ew64 = 0;

  __device__ __forceinline__ int64_t row_begin(int64_t v) const {
    return off64 ? static_cast<const int64_t *>(off)[v] : (int64_t) static_cast<const int32_t *>(off)[v];
  }
  __device__ __forceinline__ int64_t vweight(int64_t v) const {
    if (!vw) return 1;
    return vw64 ? static_cast<const int64_t *>(vw)[v] : (int64_t) static_cast<const int32_t *>(vw)[v];
  }
  __device__ __forceinline__ int64_t eweight(int64_t e) const {
    if (!ew) return 1;
    return ew64 ? static_cast<const int64_t *>(ew)[e] : (int64_t) static_cast<const int32_t *>(ew)[e];
  }
  // edge-weight mode: 0 unit, 1 int32, 2 int64
  int ew_mode() const { return ew ? (ew64 ? 2 : 1) : 0; }
  int64_t offset_bytes() const { return off64 ? 8 : 4; }
  int64_t vw_bytes() const { return vw ? (vw64 ? 8 : 4) : 0; }
  int64_t ew_bytes() const { return ew ? (ew64 ? 8 : 4) : 0; }
};

inline DGraph make_dgraph(const gp_graph *g) {
  DGraph d;
  d.n = g->n;
  d.m = g->m_dir;
  d.off = g->offsets;
  d.adj = g->adj;
  d.vw = g->vwgt;
  d.ew = g->ewgt;
  d.off64 = g->offsets_64 ? 1 : 0;
  d.vw64 = g->vwgt_64 ? 1 : 0;
  d.ew64 = g->ewgt_64 ? 1 : 0;
  return d;
}

// Typed edge-weight load selected at compile time: EW = 0 unit, 1 int32, 2 int64.
template <int EW>
__device__ __forceinline__ int64_t load_ew(const void *ew, int64_t e) {
  if constexpr (EW == 0) return 1;
  else if constexpr (EW == 1) return (int64_t)__ldg(static_cast<const int32_t *>(ew) + e);
  else return (int64_t)__ldg(reinterpret_cast<const long long *>(ew) + e);
}

// ------------------------------------------------------------------------------------------ device
int num_sms();
int device_id();

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int64_t warp_sum64(int64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Block-wide exclusive scan of int64 (blockDim.x <= 1024, multiple of 32). `tmp` holds 32 entries.
template <class T>
__device__ __forceinline__ T block_excl_scan64(T x, T *tmp, T *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) tmp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? tmp[lane] : 0;
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nw) tmp[lane] = wi - w;
    if (lane == nw - 1 && total) *total = wi;
  }
  __syncthreads();
  T r = tmp[wid] + inc - x;
  __syncthreads();
  return r;
}

// Bounded barrier over `nblocks` blocks of a cooperatively launched kernel (all blocks co-resident).
// One word per barrier, zero-initialised. At every barrier thread 0 of each block adds to it with one
// acquire-release atomic (its release covers the writes of the whole block, ordered before it by the
// preceding __syncthreads): block rank 0 adds 2^31 - (nblocks - 1), every other block adds 1. The
// additions of one barrier sum to exactly 2^31, and the low 31 bits start at zero, so bit 31 flips when,
// and only when, the last block has arrived; each block polls the word with acquire loads until bit 31
// differs from the value its own addition returned. A block that moves on to the next barrier adds
// again, but bit 31 cannot flip back before every block has arrived there too. A problem of one block
// needs only __syncthreads.
// The wait is bounded in time: a block that has polled for more than `wait_us` microseconds of the
// global timer (or that sees another block's timeout) stores GP_ERR_TIMEOUT in `err` and returns false,
// and so does every other waiting block once it sees the flag, so the kernel ends with every block
// returned and the host reads the status.
constexpr unsigned kBarrierStride = 32;
inline unsigned barrier_words(unsigned) { return kBarrierStride; }
constexpr unsigned long long kDefaultWaitNs = 20ull * 1000 * 1000 * 1000;  // 20 s
// Process-wide limit of every bounded device wait (host setting, copied into each launch's arguments).
unsigned long long wait_limit_ns();
void set_wait_limit_ns(unsigned long long ns);  // 0 restores kDefaultWaitNs

struct GridBarrier {
  unsigned int *count;  // barrier_words(nblocks) words, zero-initialised
  int *err;
  unsigned int nblocks;
  unsigned int rank;    // this block's index among the nblocks
  unsigned int wait_us; // limit of one wait in microseconds
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool grid_sync(const GridBarrier &b) {
  __shared__ int s_ok;
  if (b.nblocks <= 1) {
    __syncthreads();
    return true;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_ok = 1;
    const unsigned inc = b.rank == 0 ? 0x80000000u - (b.nblocks - 1) : 1u;
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(b.count), "r"(inc) : "memory");
    const unsigned long long t0 = global_ns();
    while (((ld_acquire_u32(b.count) ^ old) & 0x80000000u) == 0) {
      if (global_ns() - t0 > 1000ull * b.wait_us || *(volatile int *)b.err == GP_ERR_TIMEOUT) {
        atomicExch(b.err, GP_ERR_TIMEOUT);
        s_ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------------------------------------ scans
// Device-wide exclusive scan of `n` int64 values (in may alias out); total -> *total_dev.
int scan_excl_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev, Workspace &ws);
// Same for uint32 flags producing int32 ranks.
int scan_excl_u32(const uint32_t *in, int32_t *out, int64_t n, int64_t *total_dev, Workspace &ws);

// ------------------------------------------------------------------------------------------ profile
// Counts every kernel launch the library issues (read with gp_launch_count).
void count_launch();
bool profiling();
struct ProfScope {
  // Records start/stop events on `s` around a launch when profiling is on.
  ProfScope(const char *name, cudaStream_t s);
  ~ProfScope();
  const char *name;
  cudaStream_t s;
  int slot;
};
void prof_add_counts(const char *name, int64_t items, int64_t edges, int64_t bytes);
void prof_add_time(const char *name, double ms);  // device time measured inside a kernel
int prof_flush(cudaStream_t s);  // kept for call sites; events are resolved by prof_read

}  // namespace gp
