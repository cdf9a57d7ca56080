// common.cu -- errors, allocator, device-wide scans and kernel profiling of the partitioner library.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gp_internal.cuh"

namespace gp {

// ------------------------------------------------------------------------------------------ errors
static thread_local std::string t_last_error;
void set_error(const std::string &msg) { t_last_error = msg; }
const char *last_error() { return t_last_error.c_str(); }

// ------------------------------------------------------------------------------------------ memory
static gp_alloc_fn g_alloc = nullptr;
static gp_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

static void *raw_alloc(size_t bytes, cudaStream_t s) {
  if (g_alloc) return g_alloc(bytes, s, g_alloc_ctx);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void raw_free(void *p, size_t bytes, cudaStream_t s) {
  if (g_alloc) {
    if (g_free) g_free(p, bytes, s, g_alloc_ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

// Freed blocks of up to kCacheMaxBlock bytes are kept (at most kCacheMaxTotal bytes in all) and
// handed out again for an allocation of exactly the same size on the same stream, so repeated calls
// on graphs of one shape make no allocator calls after the first; reuse on the freeing stream keeps
// it stream-ordered. free_cached() returns them all to the allocator.
struct CachedBlock {
  void *p;
  size_t bytes;
  cudaStream_t s;
};
static std::mutex g_cache_mu;
static std::vector<CachedBlock> g_cache;
static size_t g_cache_bytes = 0;
constexpr size_t kCacheMaxBlock = size_t(64) << 20;
constexpr size_t kCacheMaxTotal = size_t(1) << 30;

// The calling thread's pinned staging buffer for Readback (grown on demand, kept until the thread
// exits).
namespace {
struct PinnedStage {
  unsigned char *p = nullptr;
  size_t cap = 0;
  ~PinnedStage() {
    if (p) cudaFreeHost(p);
  }
};
thread_local PinnedStage t_stage;
}  // namespace

static std::atomic<long long> g_stage_allocs{0};
long long pinned_stage_allocs() { return g_stage_allocs.load(); }
static thread_local ScratchArena *t_arena = nullptr;

int Readback::run(cudaStream_t s) {
  if (items.empty()) return GP_OK;
  if (t_arena) {
    // A caller that allocates nothing gets no pinned host stage either: the copies go straight to
    // the (pageable) host destinations, still with a single synchronisation at the end.
    for (const Item &it : items)
      if (it.bytes) GP_CUDA(cudaMemcpyAsync(it.host, it.dev, it.bytes, cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    items.clear();
    total = 0;
    return GP_OK;
  }
  if (t_stage.cap < total) {
    if (t_stage.p) cudaFreeHost(t_stage.p);
    t_stage.p = nullptr;
    t_stage.cap = 0;
    const size_t cap = std::max<size_t>(total, 64 * 1024);
    void *h = nullptr;
    GP_CUDA(cudaMallocHost(&h, cap));
    g_stage_allocs.fetch_add(1);
    t_stage.p = static_cast<unsigned char *>(h);
    t_stage.cap = cap;
  }
  for (const Item &it : items)
    if (it.bytes) GP_CUDA(cudaMemcpyAsync(t_stage.p + it.off, it.dev, it.bytes, cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  for (const Item &it : items)
    if (it.bytes) std::memcpy(it.host, t_stage.p + it.off, it.bytes);
  items.clear();
  total = 0;
  return GP_OK;
}

void free_cached() {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (const CachedBlock &b : g_cache) raw_free(b.p, b.bytes, b.s);
  g_cache.clear();
  g_cache_bytes = 0;
}

void set_allocator(gp_alloc_fn a, gp_free_fn f, void *ctx) {
  free_cached();  // cached blocks belong to the allocator being replaced
  g_alloc = a;
  g_free = a ? f : nullptr;
  g_alloc_ctx = a ? ctx : nullptr;
}

// While a thread has an arena installed, its temporary allocations are carved from that fixed
// device buffer (bump allocation, released all at once by the caller) instead of an allocator.
void set_thread_arena(ScratchArena *a) { t_arena = a; }
bool arena_active() { return t_arena != nullptr; }

void *dev_alloc(size_t bytes, cudaStream_t s) {
  if (t_arena) {
    const size_t off = (t_arena->used + 255) & ~size_t(255);
    if (off + bytes > t_arena->size) return nullptr;
    t_arena->used = off + bytes;
    if (t_arena->used > t_arena->high) t_arena->high = t_arena->used;
    return t_arena->base + off;
  }
  if (bytes <= kCacheMaxBlock) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (size_t i = g_cache.size(); i-- > 0;) {
      if (g_cache[i].bytes == bytes && g_cache[i].s == s) {
        void *p = g_cache[i].p;
        g_cache[i] = g_cache.back();
        g_cache.pop_back();
        g_cache_bytes -= bytes;
        return p;
      }
    }
  }
  return raw_alloc(bytes, s);
}

void dev_free(void *p, size_t bytes, cudaStream_t s) {
  if (!p || t_arena) return;
  if (bytes <= kCacheMaxBlock) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (g_cache_bytes + bytes <= kCacheMaxTotal) {
      g_cache.push_back({p, bytes, s});
      g_cache_bytes += bytes;
      return;
    }
  }
  raw_free(p, bytes, s);
}

// ------------------------------------------------------------------------------------------ waits
static std::atomic<unsigned long long> g_wait_ns{kDefaultWaitNs};
unsigned long long wait_limit_ns() { return g_wait_ns.load(); }
void set_wait_limit_ns(unsigned long long ns) { g_wait_ns.store(ns ? ns : kDefaultWaitNs); }

// ------------------------------------------------------------------------------------------ device
int device_id() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

int num_sms() {
  static int cached[64] = {0};
  const int d = device_id();
  if (d < 0 || d >= 64) return 148;
  if (!cached[d]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    cached[d] = v > 0 ? v : 148;
  }
  return cached[d];
}

// ------------------------------------------------------------------------------------------ scans
// Three-phase scan: per-block totals, a single-block scan of the totals, per-block rescan.
namespace {
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

template <class In>
__global__ void k_scan_reduce(const In *in, int64_t n, int64_t *block_tot) {
  __shared__ int64_t tmp[32];
  __shared__ int64_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
  for (int k = 0; k < kScanItems; k++) {
    const int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    if (i < n) s += (int64_t)in[i];
  }
  block_excl_scan64(s, tmp, &tot);
  if (threadIdx.x == 0) block_tot[blockIdx.x] = tot;
}

__global__ void k_scan_tops(int64_t *block_tot, int64_t nb, int64_t *total_dev) {
  __shared__ int64_t tmp[32];
  __shared__ int64_t tot;
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t x = i < nb ? block_tot[i] : 0;
    const int64_t ex = block_excl_scan64(x, tmp, &tot);
    if (i < nb) block_tot[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total_dev) *total_dev = carry;
}

// block_off NULL: a single tile (one block), whose total goes to *total_dev (may be NULL).
template <class In, class Out>
__global__ void k_scan_final(const In *in, Out *out, int64_t n, const int64_t *block_off, int64_t *total_dev) {
  __shared__ int64_t tmp[32];
  __shared__ int64_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  In vals[kScanItems];
  int64_t s = 0;
  for (int k = 0; k < kScanItems; k++) {
    const int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    vals[k] = i < n ? in[i] : (In)0;
    s += (int64_t)vals[k];
  }
  int64_t run = block_excl_scan64(s, tmp, &tot) + (block_off ? block_off[blockIdx.x] : 0);
  if (!block_off && total_dev && threadIdx.x == 0) *total_dev = tot;
  for (int k = 0; k < kScanItems; k++) {
    const int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    if (i < n) out[i] = (Out)run;
    run += (int64_t)vals[k];
  }
}

template <class In, class Out>
int scan_impl(const In *in, Out *out, int64_t n, int64_t *total_dev, Workspace &ws) {
  cudaStream_t s = ws.stream();
  if (n <= 0) {
    if (total_dev) GP_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s));
    return GP_OK;
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    // one tile: one launch
    (::gp::count_launch(), k_scan_final<In, Out><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total_dev));
    GP_LAUNCH_CHECK();
    return GP_OK;
  }
  int64_t *bt;
  GP_TRY(ws.get(&bt, (size_t)nb));
  (::gp::count_launch(), k_scan_reduce<In><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, bt));
  (::gp::count_launch(), k_scan_tops<<<1, 1024, 0, s>>>(bt, nb, total_dev));
  (::gp::count_launch(), k_scan_final<In, Out><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, bt, nullptr));
  GP_LAUNCH_CHECK();
  return GP_OK;
}
}  // namespace

int scan_excl_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev, Workspace &ws) {
  return scan_impl<int64_t, int64_t>(in, out, n, total_dev, ws);
}
int scan_excl_u32(const uint32_t *in, int32_t *out, int64_t n, int64_t *total_dev, Workspace &ws) {
  return scan_impl<uint32_t, int32_t>(in, out, n, total_dev, ws);
}

// ------------------------------------------------------------------------------------------ profile
namespace {
struct ProfEntry {
  std::string name;
  int64_t launches = 0;
  double ms = 0;
  int64_t items = 0, edges = 0, bytes = 0;
};
struct Pending {
  int entry;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfEntry> g_entries;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_event_pool;

int entry_index(const char *name) {
  for (size_t i = 0; i < g_entries.size(); i++)
    if (g_entries[i].name == name) return (int)i;
  g_entries.push_back(ProfEntry());
  g_entries.back().name = name;
  return (int)g_entries.size() - 1;
}

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

std::atomic<long long> g_launches{0};

bool profiling() { return g_prof_on; }

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

long long launch_count(int reset) {
  return reset ? g_launches.exchange(0) : g_launches.load();
}

ProfScope::ProfScope(const char *nm, cudaStream_t st) : name(nm), s(st), slot(-1) {
  if (!g_prof_on || t_arena) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  Pending p;
  p.entry = entry_index(nm);
  p.a = take_event();
  p.b = take_event();
  cudaEventRecord(p.a, s);
  g_pending.push_back(p);
  slot = (int)g_pending.size() - 1;
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(g_pending[slot].b, s);
}

void prof_add_counts(const char *name, int64_t items, int64_t edges, int64_t bytes) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfEntry &e = g_entries[entry_index(name)];
  e.items += items;
  e.edges += edges;
  e.bytes += bytes;
}

void prof_add_time(const char *name, double ms) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfEntry &e = g_entries[entry_index(name)];
  e.ms += ms;
  e.launches += 1;
}

// Recorded launches are resolved lazily: a call only records its events, and prof_read waits for
// them, so profiling adds no synchronisation to the calls it measures.
int prof_flush(cudaStream_t) { return GP_OK; }

static void resolve_pending() {
  for (const Pending &p : g_pending) {
    cudaEventSynchronize(p.b);
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_entries[p.entry].ms += ms;
      g_entries[p.entry].launches += 1;
    } else {
      cudaGetLastError();
    }
    g_event_pool.push_back(p.a);
    g_event_pool.push_back(p.b);
  }
  g_pending.clear();
}

int prof_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  // events are created here, not inside the calls being measured
  while (g_prof_on && g_event_pool.size() + 2 * g_pending.size() < 4096) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    g_event_pool.push_back(e);
  }
  return GP_OK;
}

int prof_read(gp_profile_entry *out, int max_entries, int reset) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  resolve_pending();
  int n = 0;
  for (const ProfEntry &e : g_entries) {
    if (n >= max_entries) break;
    gp_profile_entry &o = out[n++];
    std::memset(&o, 0, sizeof(o));
    std::strncpy(o.name, e.name.c_str(), sizeof(o.name) - 1);
    o.launches = e.launches;
    o.ms = e.ms;
    o.items = e.items;
    o.edges = e.edges;
    o.bytes = e.bytes;
  }
  if (reset) g_entries.clear();
  return n;
}

}  // namespace gp
